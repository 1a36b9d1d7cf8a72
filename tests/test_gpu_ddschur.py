"""Parity of the Section 5 Schur-complement global preconditioner on the GPU
against the oracle: interior/interface layout bit for bit, the union's FP64
factors (interface rows fixed) bit for bit against the oracle's local
factorizations laid out the same way, one application within 1e-9 (the inner
GMRES's dot products run in another order), FGMRES iterations within one, and
the mixed-precision factors within the 10 % iteration budget."""
import math

import numpy as np
import pytest

import oracle
from gpu_helpers import compare_factor, cuda_ok, gpu_compress, rel_fro, torch, vb
from paper_1508_02219_gb300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]

def _colscaled(m, seed):
    """m with its columns multiplied by seeded factors in [0.1, 10]: the Step 2
    column scalings then differ from 1 at the first and at the last level."""
    d = np.exp(np.random.default_rng(seed).uniform(np.log(0.1), np.log(10.0), m.n))
    return synth.CSR(m.n, m.rowptr.copy(), m.colind.copy(), m.val * d[m.colind])


CASES = {
    # name: (matrix, tau, nparts, msteps, nlev, droptol, lfil)
    "s4_m5": (lambda: synth.geometric(3000, 4, seed=31), 0.8, 4, 5, 3, 1e-4, 20),
    "s8_m3": (lambda: _colscaled(synth.geometric(4000, 5, seed=32), 7), 0.8, 8, 3, 2, 1e-4, -1),
    "s16_m8": (lambda: synth.geometric(6000, 6, seed=33), 0.8, 16, 8, 3, 1e-4, 30),
    "grid_s5": (lambda: synth.grid_7pt(12, 12, 12, 4, seed=1, scramble=True), 1.0, 5, 4, 2, 1e-3, 20),
    "one_part": (lambda: synth.geometric(1500, 4, seed=34), 0.8, 1, 3, 2, 1e-3, 20),
    "more_parts_than_rows": (lambda: synth.geometric(40, 3, seed=35), 0.8, 64, 2, 2, 1e-3, -1),
}


def _build(case, precision="fp64"):
    gen, tau, nparts, msteps, nlev, t, lfil = CASES[case]
    m = gen()
    V = vb()
    A = gpu_compress(m, tau)
    c = oracle.compress(m.n, m.rowptr, m.colind, m.val, tau)
    assert np.array_equal(A.export()["perm"], c.perm)
    P = V.vbarms_dd_schur_factor(A, nparts, msteps, nlev, t, lfil, precision=precision)
    D = oracle.DDSchur(c.A, nparts, msteps, nlev, t, lfil)
    return m, V, A, c, P, D


@pytest.mark.parametrize("case", list(CASES))
def test_layout_and_fp64_factors_bit_exact(case):
    m, V, A, c, P, D = _build(case)
    nparts = CASES[case][2]
    lay = V.dd_schur_layout(P)
    part, iface = D.part()
    assert np.array_equal(lay["part"], part), "subdomain of each block row differs"
    assert np.array_equal(lay["iface"], iface), "interface flags differ"
    W = [D.rows(i) for i in range(nparts)]
    assert np.array_equal(lay["rows"], np.concatenate([w for w, _ in W])), "union order differs"
    assert np.array_equal(lay["nint"], [k for _, k in W]), "interior counts differ"
    assert lay["ng"] == D.ng
    nlev, t, lfil = CASES[case][4:]
    fixed = np.concatenate([(np.arange(len(w)) >= k).astype(np.int32) for w, k in W])
    Po = oracle.Prec(oracle.block_diag([D.local(i) for i in range(nparts)]), nlev, t, lfil, fixed=fixed)
    compare_factor(P, Po)


@pytest.mark.parametrize("case", list(CASES))
def test_apply_and_fgmres(case):
    m, V, A, c, P, D = _build(case)
    x = np.random.default_rng(3).standard_normal(m.n)
    yo = np.empty(m.n)
    yo[c.perm] = D.apply(x[c.perm])
    xd = torch.from_numpy(x).cuda()
    yd = torch.zeros(m.n, dtype=torch.float64, device="cuda")
    V.vbarms_apply(P, xd, yd)
    assert rel_fro(yd.cpu().numpy(), yo) <= 1e-9
    # the allocation-free path runs the same kernels in the same order
    ys = torch.zeros_like(yd)
    V.vbarms_apply_static(P, xd, ys)
    assert torch.equal(ys, yd)
    b = synth.ones_rhs(m)
    xs = torch.zeros(m.n, dtype=torch.float64, device="cuda")
    its, rr, st = V.fgmres_solve(A, P, torch.from_numpy(b).cuda(), xs, rtol=1e-8, restart=50, maxit=1000)
    xo, its_o, rr_o, st_o = oracle.fgmres(c.A, D, b[c.perm], rtol=1e-8, restart=50, maxit=1000)
    assert st == V.VB_OK and st_o == oracle.OK
    assert abs(its - its_o) <= 1, f"FGMRES iterations {its} vs oracle {its_o}"
    r = b - m.matvec(xs.cpu().numpy())
    assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(b) * (1 + 1e-6)


def test_zero_vector_and_repeat_apply():
    m, V, A, c, P, D = _build("s4_m5")
    z = torch.zeros(m.n, dtype=torch.float64, device="cuda")
    y = torch.ones_like(z)
    V.vbarms_apply(P, z, y)
    assert torch.count_nonzero(y) == 0
    x = torch.from_numpy(np.random.default_rng(8).standard_normal(m.n)).cuda()
    y1, y2 = torch.zeros_like(x), torch.zeros_like(x)
    V.vbarms_apply(P, x, y1)
    V.vbarms_apply(P, x, y2)
    assert torch.equal(y1, y2)


def test_mixed_precision_within_budget():
    """FP32 mixed local factors: FGMRES within the mixed-precision iteration
    budget of the FP64 oracle's Schur-complement preconditioner."""
    m, V, A, c, P, D = _build("s16_m8", precision="fp32")
    b = synth.ones_rhs(m)
    xs = torch.zeros(m.n, dtype=torch.float64, device="cuda")
    its, rr, st = V.fgmres_solve(A, P, torch.from_numpy(b).cuda(), xs, rtol=1e-8)
    xo, its_o, rr_o, st_o = oracle.fgmres(c.A, D, b[c.perm], rtol=1e-8)
    assert st == V.VB_OK and st_o == oracle.OK and rr <= 1e-8
    assert its <= math.floor(1.10 * its_o), f"mixed {its} vs FP64 oracle {its_o}"


def test_invalid_arguments():
    V = vb()
    A = gpu_compress(synth.geometric(100, 3, seed=36), 0.8)
    for nparts, ms in [(0, 3), (5000, 3), (4, 0), (4, 1001)]:
        with pytest.raises(V.VbarmsError) as e:
            V.vbarms_dd_schur_factor(A, nparts, ms, 2, 1e-3, -1)
        assert e.value.status == V.VB_EINVAL
    P = V.vbarms_factor(A, 2, 1e-3, -1)
    with pytest.raises(V.VbarmsError):
        V.dd_schur_layout(P)
