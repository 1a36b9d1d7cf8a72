"""Mixed precision: FP32 factors (FP32 accumulation) with FP64 pivot blocks
where the block is near-singular, inside an FP64 FGMRES.  The per-component
error against the FP64 oracle is reported and bounded; the iteration budget
is at most 10% above the FP64 factor's."""
import math

import numpy as np
import pytest

import oracle
import precision_report
from gpu_helpers import as_dict, cuda_ok, gpu_compress, rel_fro, torch, vb
from paper_1508_02219_gb300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]

CASES = {
    "geo_3lev": (lambda: synth.geometric(2500, 6, seed=7), 0.8, 3, 1e-4, -1),
    "geo_dominance": (lambda: synth.geometric(4000, 6, seed=12, dominance=1.5, ill_frac=0.005), 0.8, 4, 1e-4, 30),
    "grid10_l5": (lambda: synth.grid_7pt(10, 10, 10, 5, seed=0, scramble=True), 1.0, 2, 1e-3, 20),
}


@pytest.mark.parametrize("case", list(CASES))
def test_mixed_factor_iteration_budget(case):
    gen, tau, nlev, t, lfil = CASES[case]
    m = gen()
    V = vb()
    A = gpu_compress(m, tau)
    b = torch.from_numpy(synth.ones_rhs(m)).cuda()
    res = {}
    for prec in ("fp64", "fp32"):
        P = V.vbarms_factor(A, nlev, t, lfil, precision=prec)
        x = torch.zeros(m.n, dtype=torch.float64, device="cuda")
        its, rr, st = V.fgmres_solve(A, P, b, x, rtol=1e-8, restart=50, maxit=1000)
        assert st == V.VB_OK, f"{prec}: FGMRES did not converge (relres {rr:.2e})"
        assert rr <= 1e-8
        true = torch.linalg.norm(x - 1.0).item() / math.sqrt(m.n)
        assert true < 1e-5, f"{prec}: solution error {true:.2e}"
        res[prec] = (its, P)
    its64, its32 = res["fp64"][0], res["fp32"][0]
    # at most 10 % extra iterations: its32 <= floor(1.10 its64)
    assert its32 <= math.floor(1.10 * its64), f"mixed FP32 needs {its32} vs FP64 {its64} iterations"


def test_mixed_factor_error_against_fp64_oracle():
    """Level 1 is ordered from FP64 values, so the FP32 run has the oracle's
    ordering there; its FP32 factors differ from the FP64 oracle by FP32
    rounding only (relative Frobenius error per component reported)."""
    gen, tau, nlev, t, lfil = CASES["geo_dominance"]
    m = gen()
    V = vb()
    A = gpu_compress(m, tau)
    c = oracle.compress(m.n, m.rowptr, m.colind, m.val, tau)
    P = V.vbarms_factor(A, nlev, t, lfil, precision="fp32")
    Po = oracle.Prec(c.A, nlev, t, lfil)
    assert np.array_equal(P.vector(0, "pI"), Po.vec(0, "pI"))
    errs = {}
    for w in ("D", "F", "E", "C"):
        g, o = P.export(0, w), as_dict(Po.mat(0, w))
        assert np.array_equal(g["bcol"], o["bcol"])
        errs[w] = rel_fro(g["val"], o["val"])
    assert errs["D"] == 0.0  # pivot blocks are gathered from the FP64 matrix
    for w in ("F", "E", "C"):
        assert errs[w] <= 1e-7
    for w in ("W", "G", "S"):
        g, o = P.export(0, w), as_dict(Po.mat(0, w))
        if np.array_equal(g["bcol"], o["bcol"]) and np.array_equal(g["bptr"], o["bptr"]):
            errs[w] = rel_fro(g["val"], o["val"])
            assert errs[w] <= 1e-5, f"{w}: {errs[w]:.2e}"
    print("per-component relative error of the FP32 factor vs the FP64 oracle (level 1):", errs)
    # every level's W, G, S, the last level's L and U, one application of the
    # preconditioner and the FGMRES solution, against the FP64 oracle
    rep = precision_report.factor_errors(P, Po)
    flat = precision_report.summary(rep)
    x = np.random.default_rng(5).standard_normal(m.n)
    y = torch.zeros(m.n, dtype=torch.float64, device="cuda")
    V.vbarms_apply(P, torch.from_numpy(x).cuda(), y)
    yo = np.empty(m.n)
    yo[c.perm] = Po.apply(x[c.perm])
    flat["apply"] = precision_report.rel(y.cpu().numpy(), yo)
    b = synth.ones_rhs(m)
    xs = torch.zeros(m.n, dtype=torch.float64, device="cuda")
    V.fgmres_solve(A, P, torch.from_numpy(b).cuda(), xs, rtol=1e-8)
    xo, _, _, _ = oracle.fgmres(c.A, Po, b[c.perm], rtol=1e-8)
    xof = np.empty(m.n)
    xof[c.perm] = xo
    flat["solution"] = precision_report.rel(xs.cpu().numpy(), xof)
    print("relative error of every result of the mixed factor vs the FP64 oracle:",
          {k: f"{v:.2e}" for k, v in flat.items()})
    print("median blockwise relative error per result:",
          {k: f"{v:.2e}" for k, v in precision_report.summary(rep, "block_rel_median").items()})
    print("blocks stored by one side only:", {f"{k}.{n}": (r["blocks_only_gpu"], r["blocks_only_oracle"])
                                             for k, v in rep.items() for n, r in v.items() if isinstance(r, dict)})
    assert all(np.isfinite(v) for v in flat.values())
    assert flat["apply"] <= 1e-2 and flat["solution"] <= 1e-2, flat


def test_near_singular_pivots_are_kept_in_fp64():
    m = synth.geometric(3000, 6, seed=13, dominance=1.5, ill_frac=0.01)
    V = vb()
    A = gpu_compress(m, 0.8)
    P = V.vbarms_factor(A, 3, 1e-4, 30, precision="fp32", fp64_pivot_cond=1e4)
    tags = np.concatenate([P.vector(l, "ptag") for l in range(P.levels + 1)])
    assert tags.sum() >= 1
    assert tags.mean() < 0.2  # most pivot blocks are well conditioned
    P2 = V.vbarms_factor(A, 3, 1e-4, 30, precision="fp32", fp64_pivot_cond=1e300)
    tags2 = np.concatenate([P2.vector(l, "ptag")[:] for l in range(P2.levels + 1)])
    assert tags2.sum() == 0
