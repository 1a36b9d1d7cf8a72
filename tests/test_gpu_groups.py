"""Parity of grouped levels (Step 3 with groups of up to group_size
supernodes, block-sparse diagonal blocks D_i, eliminated by Section 3.1's two
sweeps inside each group) on the GPU against the oracle: the ordering, the
group boundaries and every FP64 factor (pivot LU after the group
elimination, group multipliers, group part of Ubar, W, G, S, the last level)
bit for bit, the application within 1e-12, FGMRES iterations within one,
and the mixed-precision factors within the 10 % iteration budget."""
import math

import numpy as np
import pytest

import oracle
from gpu_helpers import as_dict, compare_factor, compare_vb, cuda_ok, gpu_compress, rel_fro, torch, vb
from paper_1508_02219_gb300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]

CASES = {
    # name: (matrix, tau, nlev, droptol, lfil, group_size)
    "gs2": (lambda: synth.geometric(2500, 4, seed=41), 0.8, 3, 1e-4, 20, 2),
    "gs4_lfil": (lambda: synth.geometric(3000, 5, seed=42), 0.8, 2, 1e-3, 6, 4),
    "gs8_nodrop": (lambda: synth.geometric(500, 3, seed=43), 0.8, 2, 0.0, -1, 8),
    "gs4_dom": (lambda: synth.geometric(3000, 4, seed=44, dominance=1.5, ill_frac=0.01), 0.8, 3, 1e-4, 30, 4),
    "gs3_grid": (lambda: synth.grid_7pt(10, 10, 10, 4, seed=2), 1.0, 2, 1e-3, 20, 3),
    "gs6_tau09": (lambda: synth.geometric(2000, 6, seed=45), 0.9, 4, 1e-5, 40, 6),
}


def _build(case, precision="fp64"):
    gen, tau, nlev, t, lfil, gs = CASES[case]
    m = gen()
    V = vb()
    A = gpu_compress(m, tau)
    c = oracle.compress(m.n, m.rowptr, m.colind, m.val, tau)
    assert np.array_equal(A.export()["perm"], c.perm)
    P = V.vbarms_factor(A, nlev, t, lfil, precision=precision, group_size=gs)
    Po = oracle.Prec(c.A, nlev, t, lfil, gs=gs)
    return m, V, A, c, P, Po


@pytest.mark.parametrize("case", list(CASES))
def test_grouped_fp64_factors_bit_exact(case):
    m, V, A, c, P, Po = _build(case)
    assert Po.levels >= 1
    compare_factor(P, Po)
    grouped = 0
    for lev in range(Po.levels):
        assert np.array_equal(P.vector(lev, "gptr"), Po.gptr(lev)), f"level {lev}: group boundaries differ"
        for w in ("Lg", "Ug"):
            compare_vb(P.export(lev, w), as_dict(Po.mat(lev, w)), f"level {lev} {w}")
        grouped += int(np.diff(Po.gptr(lev)).max() > 1)
    assert grouped > 0, "no group holds more than one supernode"


@pytest.mark.parametrize("case", list(CASES))
def test_grouped_apply_and_fgmres(case):
    m, V, A, c, P, Po = _build(case)
    x = np.random.default_rng(3).standard_normal(m.n)
    yo = np.empty(m.n)
    yo[c.perm] = Po.apply(x[c.perm])
    xd = torch.from_numpy(x).cuda()
    yd = torch.zeros(m.n, dtype=torch.float64, device="cuda")
    V.vbarms_apply(P, xd, yd)
    assert rel_fro(yd.cpu().numpy(), yo) <= 1e-12
    ys = torch.zeros_like(yd)
    V.vbarms_apply_static(P, xd, ys)
    assert torch.equal(ys, yd)
    b = synth.ones_rhs(m)
    xs = torch.zeros(m.n, dtype=torch.float64, device="cuda")
    its, rr, st = V.fgmres_solve(A, P, torch.from_numpy(b).cuda(), xs, rtol=1e-8, restart=50, maxit=1000)
    xo, its_o, rr_o, st_o = oracle.fgmres(c.A, Po, b[c.perm], rtol=1e-8, restart=50, maxit=1000)
    assert st == V.VB_OK and st_o == oracle.OK
    assert abs(its - its_o) <= 1, f"FGMRES iterations {its} vs oracle {its_o}"


def test_group_size_one_is_the_default_factorization():
    m = synth.geometric(2000, 4, seed=46)
    V = vb()
    A = gpu_compress(m, 0.8)
    P0 = V.vbarms_factor(A, 3, 1e-4, 20)
    P1 = V.vbarms_factor(A, 3, 1e-4, 20, group_size=1)
    x = torch.from_numpy(np.random.default_rng(4).standard_normal(m.n)).cuda()
    y0, y1 = torch.zeros_like(x), torch.zeros_like(x)
    V.vbarms_apply(P0, x, y0)
    V.vbarms_apply(P1, x, y1)
    assert torch.equal(y0, y1)


def test_grouped_mixed_precision_within_budget():
    m, V, A, c, P, Po = _build("gs4_dom", precision="fp32")
    b = synth.ones_rhs(m)
    xs = torch.zeros(m.n, dtype=torch.float64, device="cuda")
    its, rr, st = V.fgmres_solve(A, P, torch.from_numpy(b).cuda(), xs, rtol=1e-8)
    xo, its_o, rr_o, st_o = oracle.fgmres(c.A, Po, b[c.perm], rtol=1e-8)
    assert st == V.VB_OK and st_o == oracle.OK and rr <= 1e-8
    assert its <= math.floor(1.10 * its_o), f"mixed {its} vs FP64 oracle {its_o}"


def test_grouped_schur_complement_preconditioner_and_batch():
    """Groups with fixed interface rows (Schur-complement preconditioner) and
    in a batch: FGMRES converges and the batch equals the single factors."""
    m = synth.geometric(3000, 4, seed=47)
    V = vb()
    A = gpu_compress(m, 0.8)
    P = V.vbarms_dd_schur_factor(A, 4, 5, 2, 1e-4, 20, group_size=4)
    b = torch.from_numpy(synth.ones_rhs(m)).cuda()
    xs = torch.zeros(m.n, dtype=torch.float64, device="cuda")
    its, rr, st = V.fgmres_solve(A, P, b, xs, rtol=1e-8)
    assert st == V.VB_OK and rr <= 1e-8


def test_invalid_group_size():
    V = vb()
    A = gpu_compress(synth.geometric(100, 3, seed=48), 0.8)
    for gs in (0, 65):
        with pytest.raises(V.VbarmsError) as e:
            V.vbarms_factor(A, 2, 1e-3, -1, group_size=gs)
        assert e.value.status == V.VB_EINVAL
