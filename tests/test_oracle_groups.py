"""Pins of the oracle's group independent sets (Step 3 with the diagonal
blocks D_i of D block sparse) and the grouped partial factorization: the
group ordering against a brute-force replica of the breadth-first greedy, its
invariants, dense block-LU identities of the grouped factors, exactness with
no dropping, the drop and lfil rules, and the grouped code reducing to the
single-supernode factorization bit for bit.  CPU only."""
import numpy as np
import pytest

import oracle
from paper_1508_02219_gb300 import synth


def _offsets(sizes):
    return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)


def _case(nodes=300, ell=3, seed=4, tau=0.8, **kw):
    m = synth.geometric(nodes, ell, seed=seed, **kw)
    return m, oracle.compress(m.n, m.rowptr, m.colind, m.val, tau)


def _adj(A):
    p = A.nbr
    nb = [set() for _ in range(p)]
    for I in range(p):
        for J in A.bcol[A.bptr[I]:A.bptr[I + 1]]:
            if J != I:
                nb[I].add(int(J))
                nb[int(J)].add(I)
    return [sorted(s) for s in nb]


def _groups_replica(A, gs, ddtol=0.0):
    """Breadth-first group greedy written out: weights by is_order, visit by
    (weight desc, index asc), grow by unmarked neighbours in ascending order
    of the members in joining order, then mark every neighbour."""
    _, _, w = oracle.is_order(A, 0.0)
    adj = _adj(A)
    order = sorted(range(A.nbr), key=lambda v: (-w[v], v))
    marked = np.zeros(A.nbr, bool)
    groups = []
    for v in order:
        if marked[v] or w[v] < ddtol:
            continue
        g = [v]
        marked[v] = True
        head = 0
        while head < len(g) and len(g) < gs:
            for z in adj[g[head]]:
                if len(g) >= gs:
                    break
                if not marked[z] and not (w[z] < ddtol):
                    g.append(z)
                    marked[z] = True
            head += 1
        for u in g:
            marked[adj[u]] = True
        groups.append(sorted(g))
    groups.sort(key=lambda g: g[0])
    D = [v for g in groups for v in g]
    C = [v for v in range(A.nbr) if v not in set(D)]
    return np.array(D + C, np.int32), len(D), np.concatenate([[0], np.cumsum([len(g) for g in groups])])


@pytest.mark.parametrize("gs", [1, 2, 3, 5, 8])
@pytest.mark.parametrize("seed", [4, 9])
def test_group_ordering_matches_the_breadth_first_replica(gs, seed):
    m, c = _case(seed=seed)
    P = oracle.Prec(c.A, 1, 1e-3, -1, gs=gs, grouped=True)
    A0 = P.mat(0, "A")  # the scaled level matrix the ordering works on
    pI, nD, gptr = _groups_replica(A0, gs)
    assert np.array_equal(P.vec(0, "pI"), pI)
    assert P.nD(0) == nD
    assert np.array_equal(P.gptr(0), gptr)


@pytest.mark.parametrize("gs", [2, 4, 8])
def test_group_invariants(gs):
    """Groups hold at most gs supernodes, are connected, pairwise uncoupled in
    A + A^T, and maximal: every C supernode touches some group."""
    m, c = _case(500, 4, seed=6)
    P = oracle.Prec(c.A, 2, 1e-3, 20, gs=gs)
    for lev in range(P.levels):
        A = P.mat(lev, "A")
        adj = _adj(A)
        pI, nD, gptr = P.vec(lev, "pI"), P.nD(lev), P.gptr(lev)
        grp = np.full(A.nbr, -1)
        for g in range(len(gptr) - 1):
            mem = pI[gptr[g]:gptr[g + 1]]
            assert 1 <= len(mem) <= gs and np.all(np.diff(mem) > 0)
            grp[mem] = g
            seen, todo = {mem[0]}, [mem[0]]
            while todo:
                u = todo.pop()
                for z in adj[u]:
                    if grp[z] == g and z not in seen:
                        seen.add(z)
                        todo.append(z)
            assert len(seen) == len(mem), "group not connected"
        for u in range(A.nbr):
            for z in adj[u]:
                assert not (grp[u] >= 0 and grp[z] >= 0 and grp[u] != grp[z]), "groups coupled"
        for v in pI[nD:]:
            assert any(grp[z] >= 0 for z in adj[v]), "a C supernode could have started a group"


@pytest.mark.parametrize("t,lfil", [(1e-3, 10), (1e-4, -1), (0.0, -1)])
def test_grouped_code_with_one_supernode_is_the_plain_factorization(t, lfil):
    m, c = _case(400, 4, seed=3)
    P = oracle.Prec(c.A, 3, t, lfil)
    Pg = oracle.Prec(c.A, 3, t, lfil, grouped=True)
    assert P.levels == Pg.levels
    for lev in range(P.levels):
        for k in ("D", "F", "E", "C", "W", "G", "S"):
            a, b = P.mat(lev, k), Pg.mat(lev, k)
            assert np.array_equal(a.bptr, b.bptr) and np.array_equal(a.bcol, b.bcol), (lev, k)
            assert np.array_equal(a.val, b.val), (lev, k)
        assert Pg.mat(lev, "Lg").nnzb == 0 and Pg.mat(lev, "Ug").nnzb == 0
    x = np.random.default_rng(1).standard_normal(c.A.rsz.sum())
    assert np.array_equal(P.apply(x), Pg.apply(x))


def _dense(M, nrows_sizes=None):
    return M.dense()


@pytest.mark.parametrize("gs", [2, 4, 8])
def test_exact_grouped_level_satisfies_the_block_lu_identities(gs):
    """t = 0, no lfil: with Ltilde (multipliers below, P_y^T L_y on the
    diagonal) and Ubar (U_y on the diagonal, the group part above), the
    permuted level matrix [[D, F], [E, C]] gives D = Ltilde Ubar,
    W = Ltilde^{-1} F, G = E Ubar^{-1} and S = C - E D^{-1} F."""
    m, c = _case(300, 3, seed=5)
    P = oracle.Prec(c.A, 1, 0.0, -1, gs=gs)
    A = P.mat(0, "A")
    pI, nD = P.vec(0, "pI"), P.nD(0)
    off = _offsets(A.rsz)
    perm = np.concatenate([np.arange(off[I], off[I + 1]) for I in pI])
    M = A.dense()[np.ix_(perm, perm)]
    nd = int(A.rsz[pI[:nD]].sum())
    Dd, Fd, Ed, Cd = M[:nd, :nd], M[:nd, nd:], M[nd:, :nd], M[nd:, nd:]
    Dp = P.mat(0, "D")
    piv = P.vec(0, "piv")
    Lt = P.mat(0, "Lg").dense()
    Ub = P.mat(0, "Ug").dense()
    doff = _offsets(Dp.rsz)
    for y in range(Dp.nbr):
        a, b = doff[y], doff[y + 1]
        n = b - a
        lu = Dp.val[Dp.voff[Dp.bptr[y]]:Dp.voff[Dp.bptr[y] + 1]].reshape(n, n)
        Lk = np.tril(lu, -1) + np.eye(n)
        Pm = np.eye(n)
        for k in range(n):  # P applies the interchanges in order
            j = piv[a + k]
            Pm[[k, j]] = Pm[[j, k]]
        Lt[a:b, a:b] = Pm.T @ Lk
        Ub[a:b, a:b] = np.triu(lu)
    assert np.abs(Lt @ Ub - Dd).max() <= 1e-12 * np.abs(Dd).max()
    W = P.mat(0, "W").dense()
    G = P.mat(0, "G").dense()
    S = P.mat(0, "S").dense()
    assert np.abs(W - np.linalg.solve(Lt, Fd)).max() <= 1e-12 * max(1.0, np.abs(W).max())
    assert np.abs(G - np.linalg.solve(Ub.T, Ed.T).T).max() <= 1e-12 * max(1.0, np.abs(G).max())
    assert np.abs(S - (Cd - Ed @ np.linalg.solve(Dd, Fd))).max() <= 1e-12 * np.abs(S).max()


@pytest.mark.parametrize("gs,nlev", [(2, 1), (4, 3), (8, 2)])
def test_exact_grouped_factorization_inverts_A(gs, nlev):
    m, c = _case(250, 3, seed=7)
    P = oracle.Prec(c.A, nlev, 0.0, -1, gs=gs)
    assert P.levels == nlev
    x = np.random.default_rng(2).standard_normal(c.A.rsz.sum())
    ref = np.linalg.solve(c.A.dense(), x)
    assert np.linalg.norm(P.apply(x) - ref) <= 1e-12 * np.linalg.norm(ref)


def test_drop_and_lfil_rules_on_the_group_factors():
    """Every stored multiplier, group block of Ubar, W and G block passes the
    threshold (||B||_F >= t m n) and no row keeps more than lfil of them;
    some groups do fill (the group part is not empty)."""
    m, c = _case(600, 4, seed=8)
    t, lfil = 2e-3, 6
    P = oracle.Prec(c.A, 2, t, lfil, gs=6)
    filled = 0
    for lev in range(P.levels):
        for k in ("Lg", "Ug", "W", "G"):
            M = P.mat(lev, k)
            for r in range(M.nbr):
                assert M.bptr[r + 1] - M.bptr[r] <= lfil
                for b in range(M.bptr[r], M.bptr[r + 1]):
                    blk = M.val[M.voff[b]:M.voff[b + 1]]
                    assert np.sqrt((blk * blk).sum()) >= t * M.rsz[r] * M.csz[M.bcol[b]]
            if k in ("Lg", "Ug"):
                filled += M.nnzb
    assert filled > 0


def test_grouped_fgmres_converges_and_gs_grows_the_independent_set():
    m, c = _case(800, 4, seed=11)
    b = synth.ones_rhs(m)[c.perm]
    nd1 = oracle.Prec(c.A, 1, 1e-3, 20).nD(0)
    for gs in (2, 4):
        P = oracle.Prec(c.A, 3, 1e-3, 20, gs=gs)
        assert P.nD(0) > nd1
        x, its, rr, st = oracle.fgmres(c.A, P, b, rtol=1e-8)
        assert st == oracle.OK and rr <= 1e-8


def test_ddtol_rows_never_join_a_group():
    m, c = _case(300, 3, seed=12)
    P = oracle.Prec(c.A, 1, 1e-3, -1, ddtol=0.3, gs=4)
    _, _, w = oracle.is_order(P.mat(0, "A"), 0.0)
    pI, nD = P.vec(0, "pI"), P.nD(0)
    assert np.all(w[pI[:nD]] >= 0.3)
    pr, ndr, gp = _groups_replica(P.mat(0, "A"), 4, ddtol=0.3)
    assert np.array_equal(pI, pr) and np.array_equal(P.gptr(0), gp)
