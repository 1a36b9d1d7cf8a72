"""Parity at the configured full sizes, through the same C-ABI calls the
bench times: the 360k-unknown FP64 workload bit for bit against the oracle
(compression, every level's factors, the last level), and the 3M-unknown
mixed-precision workload (compression bit for bit, level-1 ordering
identical, FGMRES within the mixed-precision iteration budget of the FP64
oracle).  Each test runs the oracle on the full matrix (tens of seconds)."""
import math

import numpy as np
import pytest

import oracle
import precision_report
from gpu_helpers import as_dict, compare_factor, compare_vb, cuda_ok, gpu_compress, torch, vb
from paper_1508_02219_gb300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow, pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]


def _compress_both(m, tau):
    A = gpu_compress(m, tau, on_device=True)
    c = oracle.compress(m.n, m.rowptr, m.colind, m.val, tau)
    g = A.export()
    assert np.array_equal(g["perm"], c.perm), "P_B differs"
    assert np.array_equal(g["bsz"], c.bsz), "block sizes differ"
    compare_vb(dict(rsz=g["bsz"], csz=g["bsz"], bptr=g["bptr"], bcol=g["bcol"], voff=g["voff"], val=g["val"]),
               as_dict(c.A), "VBSR")
    return A, c


def test_fullsize_geo60k_fp64_bit_exact():
    w = synth.WORKLOADS["geo60k_l6"]
    m = synth.make_workload("geo60k_l6", seed=0)
    assert m.n == 360_000
    V = vb()
    A, c = _compress_both(m, w["tau"])
    P = V.vbarms_factor(A, w["nlev"], w["droptol"], w["lfil"], precision="fp64")
    Po = oracle.Prec(c.A, w["nlev"], w["droptol"], w["lfil"])
    compare_factor(P, Po)
    b = synth.ones_rhs(m)
    x = torch.zeros(m.n, dtype=torch.float64, device="cuda")
    its, rr, st = V.fgmres_solve(A, P, torch.from_numpy(b).cuda(), x, rtol=1e-8)
    xo, its_o, rr_o, st_o = oracle.fgmres(c.A, Po, b[c.perm], rtol=1e-8)
    assert st == V.VB_OK and st_o == oracle.OK
    assert abs(its - its_o) <= 1 and rr <= 1e-8


def test_fullsize_geo500k_mixed():
    w = synth.WORKLOADS["geo500k_l6"]
    m = synth.make_workload("geo500k_l6", seed=0)
    assert m.n == 3_000_000
    V = vb()
    A, c = _compress_both(m, w["tau"])
    P = V.vbarms_factor(A, w["nlev"], w["droptol"], w["lfil"], precision="fp32")
    Po = oracle.Prec(c.A, w["nlev"], w["droptol"], w["lfil"])
    # level 1 is scaled and ordered from the FP64 matrix: identical to the oracle
    for v in ("r", "c", "w"):
        assert np.array_equal(P.vector(0, v), Po.vec(0, v)), f"level 1 {v} differs"
    assert np.array_equal(P.vector(0, "pI"), Po.vec(0, "pI")), "level 1 ordering differs"
    b = synth.ones_rhs(m)
    x = torch.zeros(m.n, dtype=torch.float64, device="cuda")
    its, rr, st = V.fgmres_solve(A, P, torch.from_numpy(b).cuda(), x, rtol=1e-8)
    xo, its_o, rr_o, st_o = oracle.fgmres(c.A, Po, b[c.perm], rtol=1e-8)
    assert st == V.VB_OK and st_o == oracle.OK
    assert rr <= 1e-8
    assert its <= math.floor(1.10 * its_o), f"mixed FGMRES {its} vs FP64 oracle {its_o}"
    # the true residual, recomputed here in FP64
    xg = x.cpu().numpy()
    r = b - m.matvec(xg)
    assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(b) * (1 + 1e-6)
    # the error of every result against the FP64 oracle, reported
    rep = precision_report.factor_errors(P, Po)
    flat = precision_report.summary(rep)
    print("median blockwise relative error per result:",
          {k: f"{v:.2e}" for k, v in precision_report.summary(rep, "block_rel_median").items()})
    xof = np.empty(m.n)
    xof[c.perm] = xo
    flat["solution"] = precision_report.rel(xg, xof)
    print("geo500k_l6 mixed factor, relative error per result vs the FP64 oracle:",
          {k: f"{v:.2e}" for k, v in flat.items()})
    # both solutions meet rtol 1e-8; they differ by up to cond(A) times that
    # (the workload plants pivot blocks of condition 1e6)
    assert all(np.isfinite(v) for v in flat.values()) and flat["solution"] <= 1e-2
