"""Parity of the Section 5 global preconditioners (block Jacobi, additive
and restricted additive Schwarz with VBARMS local solvers) on the GPU
against the oracle: subdomain layout bit for bit, the union's FP64 factors
bit for bit against the oracle's local factorizations laid out the same way,
the application to 1e-12, FGMRES iterations within one."""
import math

import numpy as np
import pytest

import oracle
from gpu_helpers import compare_factor, cuda_ok, gpu_compress, rel_fro, torch, vb
from paper_1508_02219_gb300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]

CASES = {
    # name: (matrix, tau, nparts, overlap, restricted, nlev, droptol, lfil)
    "bj8": (lambda: synth.geometric(3000, 4, seed=21), 0.8, 8, 0, True, 3, 1e-4, 20),
    "ras4_d1": (lambda: synth.geometric(2500, 5, seed=22), 0.8, 4, 1, True, 2, 1e-3, -1),
    "asm4_d1": (lambda: synth.geometric(2500, 5, seed=22), 0.8, 4, 1, False, 2, 1e-3, -1),
    "ras16_d2": (lambda: synth.geometric(4000, 6, seed=23, dominance=1.5, ill_frac=0.01), 0.8, 16, 2, True, 3,
                 1e-4, 30),
    "grid_ras5": (lambda: synth.grid_7pt(10, 10, 10, 5, seed=0, scramble=True), 1.0, 5, 1, True, 2, 1e-3, 20),
    "more_parts_than_rows": (lambda: synth.geometric(40, 3, seed=24), 0.8, 64, 1, True, 2, 1e-3, -1),
}


def _compress_both(m, tau):
    A = gpu_compress(m, tau)
    c = oracle.compress(m.n, m.rowptr, m.colind, m.val, tau)
    assert np.array_equal(A.export()["perm"], c.perm)
    return A, c


def _build(case, precision="fp64"):
    gen, tau, nparts, ov, restricted, nlev, t, lfil = CASES[case]
    m = gen()
    V = vb()
    A, c = _compress_both(m, tau)
    P = V.vbarms_dd_factor(A, nparts, ov, restricted, nlev, t, lfil, precision=precision)
    D = oracle.DD(c.A, nparts, ov, restricted, nlev, t, lfil)
    return m, V, A, c, P, D


@pytest.mark.parametrize("case", list(CASES))
def test_dd_layout_and_fp64_factors_bit_exact(case):
    m, V, A, c, P, D = _build(case)
    nparts = CASES[case][2]
    part, dstart, rows = V.dd_layout(P)
    assert np.array_equal(part, D.part()), "subdomain of each block row differs"
    W = [D.rows(i) for i in range(nparts)]
    assert np.array_equal(dstart, np.concatenate([[0], np.cumsum([len(w) for w in W])])), "subdomain sizes differ"
    assert np.array_equal(rows, np.concatenate(W)), "overlap sets W_i differ"
    # the oracle factors every A_i on its own; the GPU factors their union
    nlev, t, lfil = CASES[case][5:]
    Po = oracle.Prec(oracle.block_diag([D.local(i) for i in range(nparts)]), nlev, t, lfil)
    compare_factor(P, Po)


@pytest.mark.parametrize("case", list(CASES))
def test_dd_apply_and_fgmres(case):
    m, V, A, c, P, D = _build(case)
    x = np.random.default_rng(3).standard_normal(m.n)
    yo = np.empty(m.n)
    yo[c.perm] = D.apply(x[c.perm])
    xd = torch.from_numpy(x).cuda()
    yd = torch.zeros(m.n, dtype=torch.float64, device="cuda")
    V.vbarms_apply(P, xd, yd)
    assert rel_fro(yd.cpu().numpy(), yo) <= 1e-12
    if m.n <= 500_000:  # the allocation-free path gives the same result
        ys = torch.zeros_like(yd)
        V.vbarms_apply_static(P, xd, ys)
        assert rel_fro(ys.cpu().numpy(), yo) <= 1e-12
    b = synth.ones_rhs(m)
    xs = torch.zeros(m.n, dtype=torch.float64, device="cuda")
    its, rr, st = V.fgmres_solve(A, P, torch.from_numpy(b).cuda(), xs, rtol=1e-8, restart=50, maxit=1000)
    xo, its_o, rr_o, st_o = oracle.fgmres(c.A, D, b[c.perm], rtol=1e-8, restart=50, maxit=1000)
    assert st == V.VB_OK and st_o == oracle.OK
    assert abs(its - its_o) <= 1, f"FGMRES iterations {its} vs oracle {its_o}"
    r = b - m.matvec(xs.cpu().numpy())
    assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(b) * (1 + 1e-6)


def test_one_subdomain_is_plain_vbarms():
    m = synth.geometric(2000, 5, seed=25)
    V = vb()
    A = gpu_compress(m, 0.8)
    P1 = V.vbarms_factor(A, 3, 1e-4, 20)
    x = torch.from_numpy(np.random.default_rng(4).standard_normal(m.n)).cuda()
    y1 = torch.zeros_like(x)
    V.vbarms_apply(P1, x, y1)
    for ov in (0, 2):
        Pd = V.vbarms_dd_factor(A, 1, ov, True, 3, 1e-4, 20)
        yd = torch.zeros_like(x)
        V.vbarms_apply(Pd, x, yd)
        assert torch.equal(yd, y1)


def test_dd_mixed_precision_within_budget():
    """FP32 mixed local factors: FGMRES within the mixed-precision iteration
    budget of the FP64 oracle's RAS."""
    m, V, A, c, P, D = _build("ras16_d2", precision="fp32")
    b = synth.ones_rhs(m)
    xs = torch.zeros(m.n, dtype=torch.float64, device="cuda")
    its, rr, st = V.fgmres_solve(A, P, torch.from_numpy(b).cuda(), xs, rtol=1e-8)
    xo, its_o, rr_o, st_o = oracle.fgmres(c.A, D, b[c.perm], rtol=1e-8)
    assert st == V.VB_OK and st_o == oracle.OK and rr <= 1e-8
    assert its <= math.floor(1.10 * its_o), f"mixed {its} vs FP64 oracle {its_o}"


def test_dd_invalid_arguments():
    V = vb()
    A = gpu_compress(synth.geometric(100, 3, seed=26), 0.8)
    for nparts, ov in [(0, 0), (5000, 0), (4, -1)]:
        with pytest.raises(V.VbarmsError) as e:
            V.vbarms_dd_factor(A, nparts, ov, True, 2, 1e-3, -1)
        assert e.value.status == V.VB_EINVAL
    P = V.vbarms_factor(A, 2, 1e-3, -1)
    with pytest.raises(V.VbarmsError):
        V.dd_layout(P)
