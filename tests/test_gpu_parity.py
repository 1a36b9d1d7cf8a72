"""GPU parity: the CUDA library through its C ABI against the FP64 CPU oracle
on the same seeded inputs (compression, ordering and FP64 factors bit-exact;
solve and FGMRES within the stated tolerances)."""
import numpy as np
import pytest

import oracle
from gpu_helpers import (FP64_REL, as_dict, compare_factor, compare_vb, cuda_ok, gpu_compress, rel_fro, torch, vb)
from paper_1508_02219_gb300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]


def compress_both(m, tau, on_device=False):
    A = gpu_compress(m, tau, on_device=on_device)
    c = oracle.compress(m.n, m.rowptr, m.colind, m.val, tau)
    g = A.export()
    assert np.array_equal(g["perm"], c.perm), "P_B differs"
    assert np.array_equal(g["bsz"], c.bsz), "block sizes differ"
    compare_vb(dict(rsz=g["bsz"], csz=g["bsz"], bptr=g["bptr"], bcol=g["bcol"], voff=g["voff"], val=g["val"]),
               as_dict(c.A), "VBSR")
    q = A.query()
    assert q["av_bd"] == c.av_bd and q["av_bs"] == c.av_bs
    return A, c


@pytest.mark.parametrize("case", ["grid_tau1", "geo_tau08", "geo_tau075_l4", "geo_tau05", "random_empty",
                                  "geo_scrambled"])
def test_compress_bit_exact(case):
    if case == "grid_tau1":
        m, tau = synth.grid_7pt(10, 10, 10, 5, seed=0, scramble=True), 1.0
    elif case == "geo_tau08":
        m, tau = synth.geometric(3000, 6, seed=1), 0.8
    elif case == "geo_tau075_l4":
        m, tau = synth.geometric(2000, 4, seed=2), 0.75
    elif case == "geo_tau05":
        m, tau = synth.geometric(1500, 5, seed=3), 0.5
    elif case == "random_empty":
        m, tau = synth.random_sparse(3000, 0.003, seed=4, empty_rows=40), 0.5
    else:
        m, tau = synth.geometric(1000, 6, seed=5, scramble=True), 0.8
    compress_both(m, tau, on_device=(case == "geo_tau08"))


def test_compress_heavy_rows_and_dense():
    # dense rows/columns exceed the shared-memory tables: global-table path
    rng = np.random.default_rng(0)
    a = (rng.random((1500, 1500)) < 0.002).astype(float) * rng.standard_normal((1500, 1500))
    a[:, 7] = 1.0
    a[11, :] = 2.0
    a[np.arange(1500), np.arange(1500)] += 5.0
    m = synth.from_dense(a)
    compress_both(m, 0.5)
    d = synth.from_dense(rng.standard_normal((300, 300)), keep_zeros=True)
    A, c = compress_both(d, 1.0)
    assert len(c.bsz) == 1


def test_compress_edge_cases():
    V = vb()
    compress_both(synth.from_dense(np.array([[3.0]])), 1.0)
    A = V.vbarms_compress(0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0), 1.0)
    assert A.query()["nblk"] == 0
    m = synth.from_dense(np.eye(5) + np.diag(np.ones(4), 1))
    bad = m.colind.copy()
    bad[0], bad[1] = bad[1], bad[0]  # row 0 becomes [1, 0]
    with pytest.raises(V.VbarmsError) as e:
        V.vbarms_compress(m.n, m.rowptr, bad, m.val, 1.0)
    assert e.value.status == V.VB_EINVAL
    with pytest.raises(V.VbarmsError) as e:
        V.vbarms_compress(m.n, m.rowptr, m.colind, m.val, 0.0)
    assert e.value.status == V.VB_EINVAL
    oob = m.colind.copy()
    oob[-1] = 99
    with pytest.raises(V.VbarmsError):
        V.vbarms_compress(m.n, m.rowptr, oob, m.val, 1.0)


FACTOR_CASES = {
    "grid10_l5": (lambda: synth.grid_7pt(10, 10, 10, 5, seed=0, scramble=True), 1.0, 2, 1e-3, 20),
    "geo_nodrop": (lambda: synth.geometric(1200, 4, seed=6), 0.75, 1, 0.0, -1),
    "geo_3lev": (lambda: synth.geometric(2500, 6, seed=7), 0.8, 3, 1e-4, -1),
    "geo_lfil": (lambda: synth.geometric(2000, 5, seed=8), 0.8, 2, 1e-3, 6),
    "geo_pivoting": (lambda: synth.geometric(1500, 6, seed=9, dominance=1.5, ill_frac=0.01), 0.8, 3, 1e-4, 30),
    "geo_ilut_only": (lambda: synth.geometric(800, 3, seed=10), 0.75, 0, 1e-3, 10),
    # the largest configuration's regime at small size: tau = 0.9 fragments the
    # node blocks (block sizes 1-12), 5 levels, t = 1e-5, lfil 40
    "geo_tau09_l5": (lambda: synth.make_workload("geo2m_l6", seed=3, scale=0.002), 0.9, 5, 1e-5, 40),
}


@pytest.mark.parametrize("case", list(FACTOR_CASES))
def test_fp64_factor_bit_exact(case):
    gen, tau, nlev, t, lfil = FACTOR_CASES[case]
    m = gen()
    V = vb()
    A, c = compress_both(m, tau)
    P = V.vbarms_factor(A, nlev, t, lfil, precision="fp64")
    Po = oracle.Prec(c.A, nlev, t, lfil)
    compare_factor(P, Po)


@pytest.mark.parametrize("case", ["geo_3lev", "geo_pivoting", "geo_tau09_l5"])
def test_fp64_factor_schur_drop_all_bit_exact(case):
    """The ARMS-style variant (threshold on S at every reduction) against the
    oracle's, bit for bit, and its application."""
    gen, tau, nlev, t, lfil = FACTOR_CASES[case]
    m = gen()
    V = vb()
    A, c = compress_both(m, tau)
    P = V.vbarms_factor(A, nlev, t, lfil, precision="fp64", schur_drop_all=True)
    Po = oracle.Prec(c.A, nlev, t, lfil, 0.0, True)
    compare_factor(P, Po)
    x = np.random.default_rng(2).standard_normal(m.n)
    yo = np.empty(m.n)
    yo[c.perm] = Po.apply(x[c.perm])
    yd = torch.zeros(m.n, dtype=torch.float64, device="cuda")
    V.vbarms_apply(P, torch.from_numpy(x).cuda(), yd)
    assert rel_fro(yd.cpu().numpy(), yo) <= 1e-12


@pytest.mark.parametrize("case", ["grid10_l5", "geo_3lev", "geo_pivoting", "geo_tau09_l5"])
def test_apply_and_fgmres_fp64(case):
    gen, tau, nlev, t, lfil = FACTOR_CASES[case]
    m = gen()
    V = vb()
    A, c = compress_both(m, tau)
    P = V.vbarms_factor(A, nlev, t, lfil, precision="fp64")
    Po = oracle.Prec(c.A, nlev, t, lfil)
    rng = np.random.default_rng(1)
    x = rng.standard_normal(m.n)
    # oracle works in the P_B numbering
    yo_p = Po.apply(x[c.perm])
    yo = np.empty(m.n)
    yo[c.perm] = yo_p
    xd = torch.from_numpy(x).cuda()
    yd = torch.zeros(m.n, dtype=torch.float64, device="cuda")
    V.vbarms_apply(P, xd, yd)
    y = yd.cpu().numpy()
    assert rel_fro(y, yo) <= 1e-12
    b = synth.ones_rhs(m)
    bd = torch.from_numpy(b).cuda()
    xs = torch.zeros(m.n, dtype=torch.float64, device="cuda")
    its, rr, st = V.fgmres_solve(A, P, bd, xs, rtol=1e-8, restart=50, maxit=1000)
    xo, its_o, rr_o, st_o = oracle.fgmres(c.A, Po, b[c.perm], rtol=1e-8, restart=50, maxit=1000)
    assert st == V.VB_OK and st_o == oracle.OK
    assert abs(its - its_o) <= 1, f"FGMRES iterations {its} vs oracle {its_o}"
    assert rr <= 1e-8
    xg = xs.cpu().numpy()
    # the true residual is checked in FP64 here too; the solution matches the
    # oracle's to the conditioning of the system
    r = b - m.matvec(xg)
    assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(b) * (1 + 1e-6)
    xo_full = np.empty(m.n)
    xo_full[c.perm] = xo
    assert rel_fro(xg, xo_full) <= 1e-6


def test_no_drop_factor_is_exact_inverse():
    """t = 0, no lfil: M = A, so FGMRES converges in one iteration."""
    V = vb()
    m = synth.geometric(1500, 4, seed=11)
    A = gpu_compress(m, 0.75)
    P = V.vbarms_factor(A, 2, 0.0, -1)
    b = torch.from_numpy(synth.ones_rhs(m)).cuda()
    x = torch.zeros(m.n, dtype=torch.float64, device="cuda")
    its, rr, st = V.fgmres_solve(A, P, b, x, rtol=1e-8)
    assert st == V.VB_OK and its == 1
    assert torch.allclose(x, torch.ones_like(x), atol=1e-8)


def test_singular_pivot_reported():
    V = vb()
    a = np.eye(4)
    a[2:, 2:] = [[1.0, 2.0], [2.0, 4.0]]
    m = synth.from_dense(a, keep_zeros=False)
    # blocks of sizes 2 and 2 from tau = 1 compression (rows 2,3 share a pattern)
    A = gpu_compress(m, 1.0)
    with pytest.raises(V.VbarmsError) as e:
        V.vbarms_factor(A, 1, 0.0, -1)
    assert e.value.status == V.VB_ESINGULAR


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_lean_factorization_applies_like_the_kept_one(precision):
    """keep_factors = 0 releases every level's scaled matrix, F, E, C and S
    once consumed; the factors the solve reads are unchanged, so the
    application is bit-identical, and exporting a released factor fails."""
    V = vb()
    m = synth.geometric(2500, 6, seed=7)
    A = gpu_compress(m, 0.8)
    P = V.vbarms_factor(A, 3, 1e-4, -1, precision=precision)
    Q = V.vbarms_factor(A, 3, 1e-4, -1, precision=precision, keep_factors=False)
    x = torch.from_numpy(np.random.default_rng(9).standard_normal(m.n)).cuda()
    y1 = torch.zeros_like(x)
    y2 = torch.zeros_like(x)
    V.vbarms_apply(P, x, y1)
    V.vbarms_apply(Q, x, y2)
    assert torch.equal(y1, y2)
    for lev, name in [(0, "W"), (0, "G"), (0, "D"), (Q.levels, "L"), (Q.levels, "U")]:
        assert np.array_equal(P.export(lev, name)["val"], Q.export(lev, name)["val"]), (lev, name)
    for name in ("A", "F", "E", "C", "S"):
        with pytest.raises(V.VbarmsError) as e:
            Q.export(0, name)
        assert e.value.status == V.VB_EINVAL


def test_ilut_geometry_is_timed_then_reused_and_results_do_not_depend_on_it():
    """The last-level ILUT's per-warp workspace is chosen by timing the
    candidate shapes on a prefix of the matrix's own rows (large last levels
    only), then reused for matrices of the same class; the factors do not
    depend on it (every element sees the oracle's operation order)."""
    V = vb()
    m = synth.geometric(110000, 3, seed=3)
    A = gpu_compress(m, 0.8)
    P1 = V.vbarms_factor(A, 1, 1e-3, 20)
    g1 = P1.ilut_geometry()
    P2 = V.vbarms_factor(A, 1, 1e-3, 20)
    g2 = P2.ilut_geometry()
    assert P1.shape(P1.levels, "A")["nbr"] >= 65536
    assert g1["source"] in ("timed", "cached") and g2["source"] == "cached"
    assert (g1["slots"], g1["value_bytes"]) == (g2["slots"], g2["value_bytes"]) and g2["warps_per_sm"] >= 1
    for name in ("L", "U", "D"):
        assert np.array_equal(P1.export(P1.levels, name)["val"], P2.export(P2.levels, name)["val"]), name
    b = torch.from_numpy(synth.ones_rhs(m)).cuda()
    x = torch.zeros(m.n, dtype=torch.float64, device="cuda")
    its, rr, st = V.fgmres_solve(A, P1, b, x, rtol=1e-8)
    assert st == V.VB_OK


def test_pivot_phase_size_classes_are_reported_and_factors_unchanged():
    """The pivot phase runs over block-size-class queues: the class counts add
    up to the pivot blocks of the level, every class names its mode, a class
    of 1024 blocks or more is timed once and then taken from the cache, and
    the factors of the timed and the cached run are identical."""
    V = vb()
    m = synth.geometric(60000, 4, seed=11)
    A = gpu_compress(m, 0.8)
    P1 = V.vbarms_factor(A, 2, 1e-3, 20)
    P2 = V.vbarms_factor(A, 2, 1e-3, 20)
    for lev in range(P1.levels):
        t1, t2 = P1.pivot_tiles(lev), P2.pivot_tiles(lev)
        assert sum(t1["counts"]) == P1.shape(lev, "D")["nbr"]
        assert all(md in ("thread", "warp") for md in t1["modes"])
        assert t1["modes"] == t2["modes"] and t2["source"] in ("default", "cached")
        assert np.array_equal(P1.export(lev, "D")["val"], P2.export(lev, "D")["val"])
        assert np.array_equal(P1.vector(lev, "piv"), P2.vector(lev, "piv"))
    assert P1.pivot_tiles(0)["source"] in ("timed", "cached")
    with pytest.raises(V.VbarmsError):
        P1.pivot_tiles(P1.levels)


def test_ilut_wait_chain_bounds_the_kept_l_depth():
    """The ILUT reports its longest chain of waits: every kept L block is a
    wait, so the chain is at least the depth of the kept L pattern (longest
    path computed here on the host), and at most the last level's rows."""
    V = vb()
    m = synth.geometric(8000, 4, seed=12)
    A = gpu_compress(m, 0.8)
    P = V.vbarms_factor(A, 2, 1e-3, 20)
    L = P.export(P.levels, "L")
    depth = np.zeros(len(L["bptr"]) - 1, np.int64)
    for i in range(len(depth)):
        cols = L["bcol"][L["bptr"][i]:L["bptr"][i + 1]]
        depth[i] = 1 + (depth[cols].max() if len(cols) else 0)
    chain = P.ilut_chain()
    assert depth.max() <= chain <= len(depth), (depth.max(), chain, len(depth))
