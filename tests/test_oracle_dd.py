"""Pins of the oracle's Section 5 global preconditioners (block Jacobi,
additive and restricted additive Schwarz with VBARMS local solvers) against
dense linear algebra and brute-force graph reachability.  CPU only."""
import numpy as np
import pytest

import oracle
from paper_1508_02219_gb300 import synth


def _offsets(sizes):
    return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)


def _case(nodes=260, ell=4, seed=3, tau=0.8):
    m = synth.geometric(nodes, ell, seed=seed)
    return oracle.compress(m.n, m.rowptr, m.colind, m.val, tau).A


def _block_graph(A):
    p = A.nbr
    B = np.zeros((p, p), bool)
    for I in range(p):
        B[I, A.bcol[A.bptr[I]:A.bptr[I + 1]]] = True
    return B | B.T


def _scalar_rows(A, blocks):
    off = _offsets(A.rsz)
    if len(blocks) == 0:
        return np.zeros(0, np.int64)
    return np.concatenate([np.arange(off[I], off[I + 1]) for I in blocks])


@pytest.mark.parametrize("nparts", [1, 3, 7])
def test_partition_is_contiguous_and_balanced(nparts):
    A = _case()
    D = oracle.DD(A, nparts, 0, True, 1, 1e-3, -1)
    part = D.part()
    n = int(A.rsz.sum())
    assert np.all(np.diff(part) >= 0) and part[0] == 0 and part[-1] == nparts - 1
    off = _offsets(A.rsz)
    for i in range(nparts):
        rows = np.flatnonzero(part == i)
        size = off[rows[-1] + 1] - off[rows[0]]
        # every range starts at the first block row whose scalar offset reaches i n / N
        assert off[rows[0]] * nparts >= i * n and (rows[0] == 0 or off[rows[0] - 1] * nparts < i * n)
        assert abs(size - n / nparts) <= 2 * A.rsz.max()
        assert np.array_equal(D.rows(i), rows)  # no overlap: W_i^0


def _drop_upper_blocks(A, frac, seed):
    """A with a seeded fraction of its strictly upper blocks removed: an
    unsymmetric block pattern."""
    rng = np.random.default_rng(seed)
    bptr, bcol, voff, vals = [0], [], [0], []
    for I in range(A.nbr):
        for b in range(A.bptr[I], A.bptr[I + 1]):
            J = A.bcol[b]
            if J > I and rng.random() < frac:
                continue
            bcol.append(J)
            vals.append(A.val[A.voff[b]:A.voff[b + 1]])
            voff.append(voff[-1] + len(vals[-1]))
        bptr.append(len(bcol))
    return oracle.VBMat(A.rsz.copy(), A.csz.copy(), np.asarray(bptr, np.int64), np.asarray(bcol, np.int32),
                        np.asarray(voff, np.int64), np.concatenate(vals))


@pytest.mark.parametrize("unsym", [False, True])
@pytest.mark.parametrize("delta", [1, 2, 3])
def test_overlap_sets_are_graph_neighbourhoods(delta, unsym):
    """W_i^delta = the block rows within delta steps of W_i^0 in the graph of
    A + A^T (boolean matrix powers), also for an unsymmetric block pattern."""
    A = _case()
    if unsym:
        A = _drop_upper_blocks(A, 0.5, 9)
        B = np.zeros((A.nbr, A.nbr), bool)
        for I in range(A.nbr):
            B[I, A.bcol[A.bptr[I]:A.bptr[I + 1]]] = True
        assert (B != B.T).any()
    nparts = 4
    D = oracle.DD(A, nparts, delta, True, 1, 1e-3, -1)
    part = D.part()
    Bi = _block_graph(A).astype(np.int64) + np.eye(A.nbr, dtype=np.int64)
    for i in range(nparts):
        v = (part == i).astype(np.int64)
        for _ in range(delta):
            v = (Bi @ v > 0).astype(np.int64)
        assert np.array_equal(D.rows(i), np.flatnonzero(v)), f"subdomain {i}"


@pytest.mark.parametrize("delta", [0, 1])
def test_local_matrices_are_principal_submatrices(delta):
    A = _case()
    Ad = A.dense()
    D = oracle.DD(A, 3, delta, True, 1, 1e-3, -1)
    for i in range(3):
        s = _scalar_rows(A, D.rows(i))
        assert np.array_equal(D.local(i).dense(), Ad[np.ix_(s, s)])


@pytest.mark.parametrize("delta,restricted", [(0, True), (1, True), (1, False), (2, True), (2, False)])
def test_exact_local_solves_match_the_dense_formula(delta, restricted):
    """With t = 0 and no lfil every local VBARMS is an exact LU, so the
    preconditioner is sum_i Q_i^T A_i^{-1} R_i (Q_i = R_i, or the restriction
    to W_i^0 when restricted), computed here with dense solves."""
    A = _case(200, 3, seed=5)
    Ad = A.dense()
    nparts = 4
    D = oracle.DD(A, nparts, delta, restricted, 2, 0.0, -1)
    part = D.part()
    x = np.random.default_rng(0).standard_normal(Ad.shape[0])
    ref = np.zeros_like(x)
    for i in range(nparts):
        W = D.rows(i)
        s = _scalar_rows(A, W)
        z = np.linalg.solve(Ad[np.ix_(s, s)], x[s])
        if restricted:
            keep = np.isin(s, _scalar_rows(A, np.flatnonzero(part == i)))
            ref[s[keep]] += z[keep]
        else:
            ref[s] += z
    y = D.apply(x)
    assert np.linalg.norm(y - ref) <= 1e-10 * np.linalg.norm(ref)
    if delta == 0:  # block Jacobi: M = blockdiag(A_i), so M y = x
        Mb = np.zeros_like(Ad)
        for i in range(nparts):
            s = _scalar_rows(A, D.rows(i))
            Mb[np.ix_(s, s)] = Ad[np.ix_(s, s)]
        assert np.linalg.norm(Mb @ y - x) <= 1e-10 * np.linalg.norm(x)


def test_one_subdomain_is_plain_vbarms():
    A = _case()
    x = np.random.default_rng(1).standard_normal(int(A.rsz.sum()))
    P = oracle.Prec(A, 2, 1e-3, 10)
    for delta in (0, 2):
        D = oracle.DD(A, 1, delta, True, 2, 1e-3, 10)
        assert np.array_equal(D.apply(x), P.apply(x))


def test_covering_overlap_restricted_is_plain_vbarms():
    """When every W_i^delta is the whole matrix, each local solve is the
    global VBARMS solve and the restricted sum takes each row once."""
    A = _case(120, 3, seed=2)
    D = oracle.DD(A, 3, 50, True, 2, 1e-3, 10)
    assert all(len(D.rows(i)) == A.nbr for i in range(3))
    x = np.random.default_rng(2).standard_normal(int(A.rsz.sum()))
    P = oracle.Prec(A, 2, 1e-3, 10)
    assert np.array_equal(D.apply(x), P.apply(x))
    Da = oracle.DD(A, 3, 50, False, 2, 1e-3, 10)
    np.testing.assert_allclose(Da.apply(x), 3 * P.apply(x), rtol=1e-14, atol=0)


def test_dd_fgmres_converges():
    A = _case(400, 4, seed=4)
    b = np.ones(int(A.rsz.sum()))
    for delta, restricted in [(0, True), (1, True), (1, False)]:
        D = oracle.DD(A, 4, delta, restricted, 2, 1e-3, 20)
        x, its, rr, st = oracle.fgmres(A, D, b, rtol=1e-8)
        assert st == oracle.OK and rr <= 1e-8
        assert np.linalg.norm(b - oracle.spmv(A, x)) <= 1e-8 * np.linalg.norm(b) * (1 + 1e-6)


@pytest.mark.parametrize("t,lfil", [(1e-3, 10), (1e-4, -1)])
def test_union_factorization_is_the_local_ones(t, lfil):
    """Every step of the method stays inside a connected component, so one
    factorization of the subdomains' block-diagonal union applies, row for
    row, exactly what the separate local factorizations apply (the layout the
    library factors)."""
    A = _case(300, 4, seed=8)
    D = oracle.DD(A, 5, 1, True, 3, t, lfil)
    locs = [D.local(i) for i in range(5)]
    U = oracle.block_diag(locs)
    Pu = oracle.Prec(U, 3, t, lfil)
    xu = np.random.default_rng(5).standard_normal(int(U.rsz.sum()))
    yu = Pu.apply(xu)
    o = 0
    for i, M in enumerate(locs):
        ni = int(M.rsz.sum())
        assert np.array_equal(yu[o:o + ni], D.local_prec(i).apply(xu[o:o + ni])), f"subdomain {i}"
        o += ni


def test_more_subdomains_than_block_rows():
    """Empty subdomains are skipped; with exact local solves the restricted sum
    over the non-empty ones is the dense formula, and the ranges still cover
    every block row once."""
    A = _case(20, 3, seed=6)
    nparts = 2 * A.nbr
    D = oracle.DD(A, nparts, 1, True, 2, 0.0, -1)
    part = D.part()
    assert len(part) == A.nbr and len(set(part.tolist())) < nparts, "some subdomains are empty"
    assert sum(len(np.flatnonzero(part == i)) for i in range(nparts)) == A.nbr
    Ad = A.dense()
    x = np.random.default_rng(7).standard_normal(Ad.shape[0])
    ref = np.zeros_like(x)
    for i in range(nparts):
        W = D.rows(i)
        if len(W) == 0:
            continue
        s = _scalar_rows(A, W)
        z = np.linalg.solve(Ad[np.ix_(s, s)], x[s])
        keep = np.isin(s, _scalar_rows(A, np.flatnonzero(part == i)))
        ref[s[keep]] += z[keep]
    y = D.apply(x)
    assert np.linalg.norm(y - ref) <= 1e-10 * np.linalg.norm(ref)
