"""Pins of the oracle's Steps 2-4 (Section 3: scaling, block independent set,
block partial factorization Eq. 4-6, multilevel recursion Eq. 7-8, block ILUT
with dropping, Alg. 3) against dense linear algebra and invariants.  CPU only."""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from paper_1508_02219_gb300 import synth


def _offsets(sizes):
    return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)


def scalar_perm(sizes, order):
    off = _offsets(sizes)
    if len(order) == 0:
        return np.zeros(0, np.int64)
    return np.concatenate([np.arange(off[Y], off[Y + 1]) for Y in order])


def piv_perm(piv):
    """Row order p with A[p] = L U for LAPACK-style interchanges."""
    p = np.arange(len(piv))
    for k, q in enumerate(piv):
        p[[k, q]] = p[[q, k]]
    return p


def lu_parts(lu):
    L = np.tril(lu, -1) + np.eye(lu.shape[0])
    U = np.triu(lu)
    return L, U


def blockdiag_dense(Dm: oracle.VBMat):
    """Dense P^T L U of every GEPP-factored pivot block, as block diagonal."""
    n = int(Dm.rsz.sum())
    out = np.zeros((n, n))
    off = _offsets(Dm.rsz)
    return out, off


def compressed(nodes=60, ell=4, seed=0, tau=0.75, approx=True, dominance=None):
    m = synth.geometric(nodes, ell, seed=seed, approx=approx, dominance=dominance)
    return m, oracle.compress(m.n, m.rowptr, m.colind, m.val, tau)


def test_scaling_matches_numpy():
    m, c = compressed(80, 5, seed=1)
    s, r, cc = oracle.scale(c.A)
    a = c.A.dense()
    rmax = np.abs(a).max(axis=1)
    r_np = np.where(rmax > 0, 1.0 / np.where(rmax > 0, rmax, 1), 1.0)
    b = r_np[:, None] * a
    cmax = np.abs(b).max(axis=0)
    c_np = np.where(cmax > 0, 1.0 / np.where(cmax > 0, cmax, 1), 1.0)
    assert np.array_equal(r, r_np) and np.array_equal(cc, c_np)
    assert np.array_equal(s.dense(), b * c_np[None, :])
    assert np.abs(s.dense()).max() <= 1.0 + 2 ** -52


def test_scaling_zero_rows_and_cols():
    a = np.zeros((4, 4))
    a[0, 0] = 3.0
    a[1, 1] = -0.5
    a[1, 3] = 2.0
    from conftest import vb_from_dense_blocks
    vb = vb_from_dense_blocks(a, [2, 2], drop_zero_blocks=False)
    s, r, c = oracle.scale(vb)
    assert r[2] == 1.0 and r[3] == 1.0 and c[2] == 1.0
    assert r[0] == 1 / 3.0 and r[1] == 0.5


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_independent_set_is_the_greedy_by_weight(seed):
    m, c = compressed(150, 3, seed=seed)
    s, _, _ = oracle.scale(c.A)
    pI, nD, w = oracle.is_order(s)
    p = s.nbr
    # weights: ||A_YY||_F / sum_Z ||A_YZ||_F, recomputed with numpy norms
    for Y in range(p):
        norms = [np.linalg.norm(s.val[s.voff[b]:s.voff[b + 1]]) for b in range(s.bptr[Y], s.bptr[Y + 1])]
        cols = list(s.bcol[s.bptr[Y]:s.bptr[Y + 1]])
        d = norms[cols.index(Y)] if Y in cols else 0.0
        assert w[Y] == pytest.approx(d / sum(norms), rel=1e-14)
    adj = [set() for _ in range(p)]
    for Y in range(p):
        for b in range(s.bptr[Y], s.bptr[Y + 1]):
            Z = int(s.bcol[b])
            if Z != Y:
                adj[Y].add(Z)
                adj[Z].add(Y)
    D = set(pI[:nD].tolist())
    assert list(pI[:nD]) == sorted(D) and list(pI[nD:]) == sorted(set(range(p)) - D)

    def better(u, v):
        return w[u] > w[v] or (w[u] == w[v] and u < v)
    # lexicographically-first MIS in rank order: v in D iff no better neighbour in D
    for v in range(p):
        has_better_D = any(u in D and better(u, v) for u in adj[v])
        assert (v in D) == (not has_better_D)
    # brute-force sequential greedy
    order = sorted(range(p), key=lambda v: (-w[v], v))
    marked, Dg = set(), set()
    for v in order:
        if v in marked:
            continue
        Dg.add(v)
        marked.add(v)
        marked |= adj[v]
    assert Dg == D


def test_ddtol_forces_weak_rows_to_C():
    m, c = compressed(100, 3, seed=7)
    s, _, _ = oracle.scale(c.A)
    pI, nD, w = oracle.is_order(s, ddtol=0.3)
    assert all(w[v] >= 0.3 for v in pI[:nD])


@pytest.mark.parametrize("mm", [1, 2, 5, 6, 12])
def test_gepp_matches_lapack(mm):
    rng = np.random.default_rng(mm)
    a = rng.standard_normal((mm, mm))
    lu, piv = oracle.gepp(a)
    lu_ref, piv_ref = sla.lu_factor(a)
    assert np.array_equal(piv, piv_ref)
    np.testing.assert_allclose(lu, lu_ref, rtol=1e-12, atol=1e-14)
    L, U = lu_parts(lu)
    np.testing.assert_allclose((L @ U), a[piv_perm(piv)], rtol=1e-13, atol=1e-14)


def test_gepp_ties_take_lowest_row_and_singular_is_reported():
    a = np.array([[1.0, 2.0], [-1.0, 5.0]])
    _, piv = oracle.gepp(a)
    assert piv[0] == 0
    with pytest.raises(oracle.OracleError) as e:
        oracle.gepp(np.array([[1.0, 2.0], [2.0, 4.0]]))
    assert e.value.status == oracle.ESINGULAR


def test_drop_rule_straddles_threshold():
    """Section 3: drop B (m x n) iff ||B||_F / (m n) < t."""
    t = 1e-3
    for (mm, nn) in [(1, 1), (2, 3), (6, 6)]:
        thr = t * mm * nn
        b = np.zeros((mm, nn))
        b[0, 0] = thr
        assert not oracle.dropped(b, t)
        b[0, 0] = np.nextafter(thr, 0)
        assert oracle.dropped(b, t)
    assert not oracle.dropped(np.zeros((2, 2)), 0.0)


def level_dense(P: oracle.Prec, lev: int):
    """Dense [[D,F],[E,C]] of level lev (scaled, P_I-permuted), plus parts."""
    A = P.mat(lev, "A")
    pI = P.vec(lev, "pI")
    sp = scalar_perm(A.rsz, pI)
    return A.dense()[np.ix_(sp, sp)]


def level_factor_dense(P: oracle.Prec, lev: int):
    """Dense lower and upper factors [[P^T L, 0], [G, I]] and [[U, W], [0, S]]."""
    Dm, W, G, S = P.mat(lev, "D"), P.mat(lev, "W"), P.mat(lev, "G"), P.mat(lev, "S")
    piv = P.vec(lev, "piv")
    nf, ns = int(Dm.rsz.sum()), int(S.rsz.sum())
    Lo = np.zeros((nf + ns, nf + ns))
    Up = np.zeros((nf + ns, nf + ns))
    off = _offsets(Dm.rsz)
    for y in range(Dm.nbr):
        lu = Dm.val[Dm.voff[Dm.bptr[y]]:Dm.voff[Dm.bptr[y] + 1]].reshape(Dm.rsz[y], Dm.rsz[y])
        L, U = lu_parts(lu)
        pp = piv_perm(piv[off[y]:off[y + 1]])
        Pt = np.eye(len(pp))[:, pp]  # P^T with P = rows pp of I
        Lo[off[y]:off[y + 1], off[y]:off[y + 1]] = Pt @ L
        Up[off[y]:off[y + 1], off[y]:off[y + 1]] = U
    Lo[nf:, :nf] = G.dense()
    Lo[nf:, nf:] = np.eye(ns)
    Up[:nf, nf:] = W.dense()
    Up[nf:, nf:] = S.dense()
    return Lo, Up, nf


@pytest.mark.parametrize("seed", [0, 1])
def test_one_level_no_drop_is_exact_block_lu(seed):
    """t = 0, no lfil: Eq. 5 holds exactly and S = C - E D^{-1} F (Eq. 6)."""
    m, c = compressed(70, 4, seed=seed)
    P = oracle.Prec(c.A, 1, 0.0, -1)
    assert P.levels == 1
    B = level_dense(P, 0)
    Lo, Up, nf = level_factor_dense(P, 0)
    scale = np.linalg.norm(B)
    assert np.linalg.norm(Lo @ Up - B) <= 1e-13 * scale
    Dd, Fd, Ed, Cd = B[:nf, :nf], B[:nf, nf:], B[nf:, :nf], B[nf:, nf:]
    S_ref = Cd - Ed @ np.linalg.solve(Dd, Fd)
    S = P.mat(0, "S").dense()
    assert np.linalg.norm(S - S_ref) <= 1e-12 * np.linalg.norm(S_ref)
    # D is block diagonal: pivot blocks are uncoupled (independent set)
    Dm = P.mat(0, "D")
    off = _offsets(Dm.rsz)
    for y in range(Dm.nbr):
        Dd[off[y]:off[y + 1], off[y]:off[y + 1]] = 0
    assert not Dd.any()
    # the extracted D, F, E, C are the blocks of the permuted matrix
    assert np.array_equal(P.mat(0, "F").dense(), Fd)
    assert np.array_equal(P.mat(0, "E").dense(), Ed)
    assert np.array_equal(P.mat(0, "C").dense(), Cd)


def _block_map(M: oracle.VBMat):
    out = {}
    for I in range(M.nbr):
        for b in range(M.bptr[I], M.bptr[I + 1]):
            J = int(M.bcol[b])
            out[(I, J)] = M.val[M.voff[b]:M.voff[b + 1]].reshape(M.rsz[I], M.csz[J])
    return out


def _blocks_of_dense(a, rs, cs):
    ro, co = _offsets(rs), _offsets(cs)
    out = {}
    for I in range(len(rs)):
        for J in range(len(cs)):
            blk = a[ro[I]:ro[I + 1], co[J]:co[J + 1]]
            if blk.any():
                out[(I, J)] = blk
    return out


@pytest.mark.parametrize("t,lfil", [(1e-3, -1), (1e-2, -1), (1e-3, 3), (5e-3, 2)])
def test_dropping_level_residual_lives_on_dropped_blocks(t, lfil):
    """With dropping, W and G keep exactly the blocks of L^{-1} P F and
    E U^{-1} that pass the threshold (and the lfil largest), and S = C - G W
    with the kept blocks (Eq. 6 with the dropped factors)."""
    m, c = compressed(90, 4, seed=11)
    P = oracle.Prec(c.A, 2, t, lfil)
    for lev in range(P.levels):
        B = level_dense(P, lev)
        Dm = P.mat(lev, "D")
        nf = int(Dm.rsz.sum())
        Lo, Up, _ = level_factor_dense(P, lev)
        Dd, Fd, Ed, Cd = B[:nf, :nf], B[:nf, nf:], B[nf:, :nf], B[nf:, nf:]
        PtL, U = Lo[:nf, :nf], Up[:nf, :nf]
        W_full = np.linalg.solve(PtL, Fd)
        G_full = np.linalg.solve(U.T, Ed.T).T
        W, G, S = P.mat(lev, "W"), P.mat(lev, "G"), P.mat(lev, "S")
        for M, full in [(W, W_full), (G, G_full)]:
            kept = _block_map(M)
            cand = _blocks_of_dense(full, M.rsz, M.csz)
            for key, blk in kept.items():
                np.testing.assert_allclose(blk, full[_offsets(M.rsz)[key[0]]:_offsets(M.rsz)[key[0] + 1],
                                                     _offsets(M.csz)[key[1]]:_offsets(M.csz)[key[1] + 1]],
                                           rtol=1e-11, atol=1e-13)
            for I in range(M.nbr):
                passing = [(np.linalg.norm(b), -J) for (r, J), b in cand.items()
                           if r == I and np.linalg.norm(b) >= t * b.shape[0] * b.shape[1] * (1 + 1e-12)]
                got = sorted(J for (r, J) in kept if r == I)
                if lfil < 0 or len(passing) <= lfil:
                    assert got == sorted(-j for _, j in passing)
                else:
                    assert len(got) == lfil
                    top = sorted(passing, reverse=True)[:lfil]
                    assert got == sorted(-j for _, j in top)
        S_ref = Cd - G.dense() @ W.dense()
        Sd = S.dense()
        if lev < P.levels - 1:
            assert np.linalg.norm(Sd - S_ref) <= 1e-12 * np.linalg.norm(S_ref)
        else:  # last reduction: off-diagonal blocks below threshold dropped
            ro = _offsets(S.rsz)
            for (I, J), blk in _blocks_of_dense(S_ref, S.rsz, S.csz).items():
                got = Sd[ro[I]:ro[I + 1], ro[J]:ro[J + 1]]
                if np.abs(got).any() or I == J:
                    np.testing.assert_allclose(got, blk, rtol=1e-10, atol=1e-14)
                else:
                    assert np.linalg.norm(blk) < t * blk.size * (1 + 1e-12)


def last_level_dense(P: oracle.Prec):
    lev = P.levels
    A, Dg, Lm, Um = P.mat(lev, "A"), P.mat(lev, "D"), P.mat(lev, "L"), P.mat(lev, "U")
    piv = P.vec(lev, "piv")
    n = int(A.rsz.sum())
    off = _offsets(A.rsz)
    Dd = np.zeros((n, n))
    for i in range(Dg.nbr):
        lu = Dg.val[Dg.voff[Dg.bptr[i]]:Dg.voff[Dg.bptr[i] + 1]].reshape(A.rsz[i], A.rsz[i])
        L, U = lu_parts(lu)
        pp = piv_perm(piv[off[i]:off[i + 1]])
        Dd[off[i]:off[i + 1], off[i]:off[i + 1]] = np.eye(len(pp))[:, pp] @ L @ U
    return A, (np.eye(n) + Lm.dense()) @ (Dd + Um.dense()), Lm, Um


@pytest.mark.parametrize("dominance", [None, 1.5])
@pytest.mark.parametrize("t,lfil", [(0.0, -1), (1e-3, -1), (1e-2, 4)])
def test_last_level_ilut_residual(t, lfil, dominance):
    """Block ILUT (Alg. 3 in block form): (I + L)(D + U) - A vanishes on every
    stored block; with t = 0 and no lfil it vanishes everywhere (block LU).
    Random (dominance) pivot blocks make GEPP interchange rows."""
    m, c = compressed(60, 3, seed=4, dominance=dominance)
    P = oracle.Prec(c.A, 0, t, lfil)  # zero reductions: ILUT of the whole matrix
    assert P.levels == 0
    A, LU, Lm, Um = last_level_dense(P)
    Ad = A.dense()
    R = LU - Ad
    if t == 0.0 and lfil < 0:
        assert np.linalg.norm(R) <= 1e-12 * np.linalg.norm(Ad)
    off = _offsets(A.rsz)
    # lfil trims the L part after its multipliers have updated the row (as in
    # pointwise ILUT), so the residual vanishes on stored blocks of the rows
    # whose L part was not trimmed.
    nL = np.diff(Lm.bptr)
    untrimmed = [I for I in range(A.nbr) if lfil < 0 or nL[I] < lfil]
    assert len(untrimmed) >= 5
    for M in (Lm, Um):
        for (I, J) in _block_map(M):
            if I in untrimmed:
                assert np.abs(R[off[I]:off[I + 1], off[J]:off[J + 1]]).max() <= 1e-12
        if lfil >= 0:
            assert max(np.diff(M.bptr)) <= lfil
    for I in untrimmed:
        assert np.abs(R[off[I]:off[I + 1], off[I]:off[I + 1]]).max() <= 1e-12


def test_singular_pivot_block_reported():
    a = np.eye(4)
    a[2:, 2:] = [[1.0, 2.0], [2.0, 4.0]]
    from conftest import vb_from_dense_blocks
    vb = vb_from_dense_blocks(a, [2, 2])
    with pytest.raises(oracle.OracleError) as e:
        oracle.Prec(vb, 1, 0.0, -1)
    assert e.value.status == oracle.ESINGULAR


@pytest.mark.parametrize("t,lfil", [(1e-3, -1), (5e-3, 3)])
def test_schur_drop_all_drops_at_every_reduction(t, lfil):
    """ARMS-style variant (Section 3 applies the threshold to S only at the
    last reduction; the variant applies it at every one): the first level's
    D, W, G are unchanged, its S is the default S less exactly the
    off-diagonal blocks below the threshold, and every level's S keeps
    C - G W on its stored blocks."""
    m, c = compressed(90, 4, seed=11)
    P0 = oracle.Prec(c.A, 3, t, lfil)
    P1 = oracle.Prec(c.A, 3, t, lfil, 0.0, True)
    for name in ("D", "W", "G", "C"):
        a, b = P0.mat(0, name), P1.mat(0, name)
        assert np.array_equal(a.bcol, b.bcol) and np.array_equal(a.val, b.val), name
    S0, S1 = _block_map(P0.mat(0, "S")), _block_map(P1.mat(0, "S"))
    assert set(S1) <= set(S0)
    for key, blk in S0.items():
        keep = key[0] == key[1] or np.linalg.norm(blk) >= t * blk.size
        assert (key in S1) == keep, key
        if keep:
            assert np.array_equal(S1[key], blk)
    assert len(S1) < len(S0), "nothing was dropped: the case pins nothing"
    for lev in range(P1.levels):
        B = level_dense(P1, lev)
        nf = int(P1.mat(lev, "D").rsz.sum())
        Cd = B[nf:, nf:]
        S = P1.mat(lev, "S")
        S_ref = Cd - P1.mat(lev, "G").dense() @ P1.mat(lev, "W").dense()
        Sd, ro = S.dense(), _offsets(S.rsz)
        for (I, J), blk in _blocks_of_dense(S_ref, S.rsz, S.csz).items():
            got = Sd[ro[I]:ro[I + 1], ro[J]:ro[J + 1]]
            if np.abs(got).any() or I == J:
                np.testing.assert_allclose(got, blk, rtol=1e-10, atol=1e-14)
            else:
                assert np.linalg.norm(blk) < t * blk.size * (1 + 1e-12)


def test_schur_drop_all_one_level_is_the_default():
    """With one level the only reduction is the last: the variant changes
    nothing."""
    m, c = compressed(70, 4, seed=2)
    P0 = oracle.Prec(c.A, 1, 1e-3, 4)
    P1 = oracle.Prec(c.A, 1, 1e-3, 4, 0.0, True)
    for lev, name in [(0, "S"), (0, "W"), (1, "L"), (1, "U"), (1, "D")]:
        assert np.array_equal(P0.mat(lev, name).val, P1.mat(lev, name).val), name


GOLDEN = __import__("os").path.join(__import__("os").path.dirname(__file__), "golden")


def test_ilut_hand_derived_three_block_rows():
    """Block ILUT (Section 3 dropping rule, Alg. 3 in block form) on a case
    whose kept and dropped blocks straddle t m n, every value derived by hand
    in tests/golden/ilut_three_block_rows.json."""
    import json
    g = json.load(open(__import__("os").path.join(GOLDEN, "ilut_three_block_rows.json")))
    from conftest import vb_from_dense_blocks
    vb = vb_from_dense_blocks(np.array(g["A"], dtype=float), g["block_sizes"])
    P = oracle.Prec(vb, 0, g["t"], -1)
    assert P.levels == 0
    assert np.array_equal(P.vec(0, "r"), np.ones(4)) and np.array_equal(P.vec(0, "c"), np.ones(4))
    for name in ("L", "U"):
        M = P.mat(0, name)
        assert M.bptr.tolist() == g[name]["bptr"], name
        assert M.bcol.tolist() == g[name]["bcol"], name
        np.testing.assert_allclose(M.val, g[name]["val"], rtol=0, atol=1e-15, err_msg=name)
    from fractions import Fraction
    np.testing.assert_allclose(P.mat(0, "D").val, [float(Fraction(x)) for x in g["D_exact"]], rtol=0, atol=1e-15)
    assert P.vec(0, "piv").tolist() == g["D"]["piv"]


def _pivot_dense(P, lev, A):
    """P^T L U of every last-level pivot block, as a dict of dense blocks."""
    Dg, piv = P.mat(lev, "D"), P.vec(lev, "piv")
    off = _offsets(A.rsz)
    out = {}
    for i in range(Dg.nbr):
        lu = Dg.val[Dg.voff[Dg.bptr[i]]:Dg.voff[Dg.bptr[i] + 1]].reshape(A.rsz[i], A.rsz[i])
        L, U = lu_parts(lu)
        pp = piv_perm(piv[off[i]:off[i + 1]])
        out[i] = np.eye(len(pp))[:, pp] @ L @ U
    return out


@pytest.mark.parametrize("dominance", [None, 1.5])
@pytest.mark.parametrize("t,lfil", [(1e-3, -1), (1e-2, -1), (1e-2, 5), (3e-2, 3)])
def test_ilut_kept_set_row_by_row(t, lfil, dominance):
    """Which blocks the block ILUT keeps (Section 3 dropping rule, Alg. 3):
    with R = (I + L)(D + U) - A, on every row whose L part was not trimmed
    by lfil,
      - a stored U block has ||U_ij||_F >= t n_i n_j, and an unstored U
        position carries the dropped working-row block, ||R_ij||_F < t n_i n_j
        (or, when lfil trimmed the U part, ranks after every stored block by
        norm descending, column ascending);
      - a stored L block has ||L_ik||_F >= t n_i n_k, and at an unstored L
        position the multiplier that was dropped, -R_ik D_k^{-1}, has norm
        < t n_i n_k;
      - the diagonal block and every stored block have R = 0."""
    m, c = compressed(60, 3, seed=4, dominance=dominance)
    P = oracle.Prec(c.A, 0, t, lfil)
    A, LU, Lm, Um = last_level_dense(P)
    R = LU - A.dense()
    off = _offsets(A.rsz)
    Dk = _pivot_dense(P, 0, A)
    Lb, Ub = _block_map(Lm), _block_map(Um)
    nL, nU = np.diff(Lm.bptr), np.diff(Um.bptr)
    slack = 1 + 1e-9
    checked = dropped_u = dropped_m = near_u = near_m = 0
    noise = 1e-13
    for i in range(A.nbr):
        if lfil >= 0 and nL[i] >= lfil:
            continue  # its L part may have been trimmed after use
        checked += 1
        ni = A.rsz[i]
        blk = lambda j: R[off[i]:off[i + 1], off[j]:off[j + 1]]
        assert np.abs(blk(i)).max() <= 1e-12, (i, "diagonal")
        stored_u = []
        for j in range(i + 1, A.nbr):
            thr = t * ni * A.rsz[j]
            if (i, j) in Ub:
                u = Ub[(i, j)]
                assert np.linalg.norm(u) >= thr / slack, (i, j, "stored U below threshold")
                assert np.abs(blk(j)).max() <= 1e-12, (i, j, "stored U block not exact")
                stored_u.append((np.linalg.norm(u), j))
                near_u += np.linalg.norm(u) < 3 * thr
        trimmed_u = lfil >= 0 and nU[i] == lfil
        for j in range(i + 1, A.nbr):
            if (i, j) in Ub:
                continue
            r = np.linalg.norm(blk(j))
            if r <= noise:
                continue
            dropped_u += 1
            thr = t * ni * A.rsz[j]
            if r >= thr * slack:
                assert trimmed_u, (i, j, f"unstored U block of norm {r:.3e} >= {thr:.3e}")
                for (sn, sj) in stored_u:
                    assert sn > r * slack or (abs(sn - r) <= 1e-12 * r and sj < j), (i, j, "lfil rank")
        for k in range(i):
            thr = t * ni * A.rsz[k]
            if (i, k) in Lb:
                lk = Lb[(i, k)]
                assert np.linalg.norm(lk) >= thr / slack, (i, k, "stored multiplier below threshold")
                assert np.abs(blk(k)).max() <= 1e-12, (i, k, "stored L block not exact")
                near_m += np.linalg.norm(lk) < 2 * thr
            else:
                r = blk(k)
                if np.linalg.norm(r) <= noise:
                    continue
                mult = -r @ np.linalg.inv(Dk[k])
                dropped_m += 1
                assert np.linalg.norm(mult) < thr * slack, (i, k, "unstored multiplier above threshold")
    # the case pins something: dropped blocks of both kinds, and kept blocks
    # close enough to the threshold that a threshold 3x (U) or 2x (multiplier)
    # larger would drop them
    print(f"rows {checked}, dropped U {dropped_u}, dropped multipliers {dropped_m}, near U {near_u}, near L {near_m}")
    assert checked >= 20 and dropped_u >= 5 and dropped_m >= 5 and near_u >= 1 and near_m >= 1, \
        (checked, dropped_u, dropped_m, near_u, near_m)
