"""Pins of the oracle's Section 5 Schur-complement global preconditioner
(eq. paral, eq. gschur, eq. loc_var_schur): the interior/interface split
against brute force on the block graph, the local Schur complements against
dense C - E B^{-1} F, the inner GMRES steps against least squares over the
Krylov space, and the exact solve when the local factorizations are exact and
the inner iteration runs to the interface dimension.  CPU only."""
import numpy as np
import pytest

import oracle
from paper_1508_02219_gb300 import synth


def _offsets(sizes):
    return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)


def _case(nodes=400, ell=3, seed=5, tau=0.8, unsym=0.0, colscale=False):
    """A compressed geometric matrix; unsym drops that seeded fraction of its
    strictly upper blocks (an unsymmetric block pattern); colscale multiplies
    its columns by seeded factors in [0.05, 20], so that the Step 2 column
    scalings differ from 1 at every level."""
    m = synth.geometric(nodes, ell, seed=seed)
    A = oracle.compress(m.n, m.rowptr, m.colind, m.val, tau).A
    rng = np.random.default_rng(seed + 100)
    bptr, bcol, voff, vals = [0], [], [0], []
    coff = _offsets(A.csz)
    d = np.exp(rng.uniform(np.log(0.05), np.log(20.0), int(coff[-1]))) if colscale else None
    for I in range(A.nbr):
        for b in range(A.bptr[I], A.bptr[I + 1]):
            J = A.bcol[b]
            if J > I and unsym > 0 and rng.random() < unsym:
                continue
            blk = A.val[A.voff[b]:A.voff[b + 1]].reshape(A.rsz[I], A.csz[J])
            if d is not None:
                blk = blk * d[coff[J]:coff[J + 1]][None, :]
            bcol.append(J)
            vals.append(blk.ravel())
            voff.append(voff[-1] + blk.size)
        bptr.append(len(bcol))
    return oracle.VBMat(A.rsz.copy(), A.csz.copy(), np.asarray(bptr, np.int64), np.asarray(bcol, np.int32),
                        np.asarray(voff, np.int64), np.concatenate(vals))


def _scalar_rows(A, blocks):
    off = _offsets(A.rsz)
    if len(blocks) == 0:
        return np.zeros(0, np.int64)
    return np.concatenate([np.arange(off[I], off[I + 1]) for I in blocks])


def _pieces(A, D):
    """Dense B_i, F_i, E_i, C_i of every subdomain (interior rows first), the
    scalar rows of each subdomain in that order, and the global interface
    scalar rows (subdomain by subdomain)."""
    Ad = A.dense()
    out, gam = [], []
    for i in range(D.nparts):
        rows, nint = D.rows(i)
        s = _scalar_rows(A, rows)
        k = int(A.rsz[rows[:nint]].sum())
        M = Ad[np.ix_(s, s)]
        out.append((s, k, M[:k, :k], M[:k, k:], M[k:, :k], M[k:, k:]))
        gam.append(s[k:])
    return Ad, out, np.concatenate(gam) if gam else np.zeros(0, np.int64)


@pytest.mark.parametrize("unsym", [0.0, 0.5])
@pytest.mark.parametrize("nparts", [2, 3, 5])
def test_interface_split_is_the_block_graph_cut(nparts, unsym):
    """D4: a block row is interface iff a stored block couples it (as row or
    column) to another subdomain; each subdomain lists its interior rows, then
    its interface rows, each ascending; A_i is the principal submatrix in that
    order; E holds exactly the blocks between interface rows of different
    subdomains."""
    A = _case(unsym=unsym)
    D = oracle.DDSchur(A, nparts, 3, 2, 1e-3, 10)
    part, iface = D.part()
    ref_part = D.part()[0]
    G = np.zeros((A.nbr, A.nbr), bool)
    for I in range(A.nbr):
        G[I, A.bcol[A.bptr[I]:A.bptr[I + 1]]] = True
    assert unsym == 0.0 or (G != G.T).any()
    cut = G & (part[:, None] != part[None, :])
    assert np.array_equal(iface.astype(bool), cut.any(1) | cut.any(0))
    assert np.array_equal(ref_part, oracle.DD(A, nparts, 0, True, 1, 1e-3, -1).part())  # D1 partition
    Ad = A.dense()
    for i in range(nparts):
        rows, nint = D.rows(i)
        mine = np.flatnonzero(part == i)
        assert np.array_equal(rows[:nint], mine[iface[mine] == 0])
        assert np.array_equal(rows[nint:], mine[iface[mine] == 1])
        # interior rows couple only inside the subdomain
        assert not cut[rows[:nint]].any() and not cut[:, rows[:nint]].any()
        s = _scalar_rows(A, rows)
        assert np.array_equal(D.local(i).dense(), Ad[np.ix_(s, s)])
    gam_blocks = np.concatenate([D.rows(i)[0][D.rows(i)[1]:] for i in range(nparts)])
    g = _scalar_rows(A, gam_blocks)
    Eref = Ad[np.ix_(g, g)].copy()
    gpart = np.repeat(part[gam_blocks], A.rsz[gam_blocks])
    Eref[gpart[:, None] == gpart[None, :]] = 0.0
    assert D.ng == len(g)
    assert np.array_equal(D.coupling().dense(), Eref)


@pytest.mark.parametrize("nlev", [1, 3])
def test_interface_rows_never_enter_an_independent_set(nlev):
    """D5: following the rows through the levels, every D row of every level
    is interior, and the last level ends with the subdomain's interface rows,
    flagged as fixed."""
    A = _case()
    D = oracle.DDSchur(A, 3, 3, nlev, 1e-3, 10)
    for i in range(3):
        rows, nint = D.rows(i)
        P = D.local_prec(i)
        idx = np.arange(len(rows))
        for lev in range(P.levels):
            pI, nD = P.vec(lev, "pI"), P.nD(lev)
            assert nD > 0 and np.all(idx[pI[:nD]] < nint)
            idx = idx[pI[nD:]]
        assert np.array_equal(idx[-(len(rows) - nint):] if len(rows) > nint else idx[:0], np.arange(nint, len(rows)))
        assert np.array_equal(P.last_fixed(), (idx >= nint).astype(np.int32))


@pytest.mark.parametrize("nlev", [0, 1, 3])
def test_exact_factorization_gives_the_local_schur_complements(nlev):
    """D5 with t = 0 and no lfil: the trailing interface factors are the LU of
    S_i = C_i - E_i B_i^{-1} F_i, so blockdiag(S_i)^{-1} v is dense-solvable."""
    A = _case(300, 3, seed=2, colscale=True)
    D = oracle.DDSchur(A, 3, 2, nlev, 0.0, -1)
    P0 = D.local_prec(0)
    # column scalings away from 1 at the first and at the last level
    assert np.abs(P0.vec(0, "c") - 1.0).max() > 0.1 and np.abs(P0.vec(P0.levels, "c") - 1.0).max() > 1e-4
    _, pcs, _ = _pieces(A, D)
    v = np.random.default_rng(1).standard_normal(D.ng)
    ref, o = [], 0
    for s, k, B, F, E, Cm in pcs:
        S = Cm - E @ np.linalg.solve(B, F)
        ng_i = len(s) - k
        ref.append(np.linalg.solve(S, v[o:o + ng_i]))
        o += ng_i
    ref = np.concatenate(ref)
    np.testing.assert_allclose(D.sinv(v), ref, rtol=0, atol=1e-11 * np.abs(ref).max())


def _dense_operator(A, D, pcs, gam):
    """K = I + blockdiag(S_i)^{-1} E and z = blockdiag(S_i)^{-1} g' for exact
    local factorizations, from dense algebra."""
    Ad = A.dense()
    ng = len(gam)
    Sinv = np.zeros((ng, ng))
    o = 0
    for s, k, B, F, E, Cm in pcs:
        ng_i = len(s) - k
        Sinv[o:o + ng_i, o:o + ng_i] = np.linalg.inv(Cm - E @ np.linalg.solve(B, F))
        o += ng_i
    Eg = D.coupling().dense()
    return np.eye(ng) + Sinv @ Eg, Sinv


@pytest.mark.parametrize("colscale", [False, True])
@pytest.mark.parametrize("msteps", [1, 2, 4])
def test_inner_gmres_minimises_over_the_krylov_space(msteps, colscale):
    """D6 with exact local factors: y minimises ||z - K y|| over
    span{z, Kz, ..., K^{m-1} z} (least squares over an explicit Krylov basis),
    and D7 recovers u_i = B_i^{-1} (f_i - F_i y_i)."""
    A = _case(300, 3, seed=2, colscale=colscale, unsym=0.3 if colscale else 0.0)
    D = oracle.DDSchur(A, 3, msteps, 2, 0.0, -1)
    _, pcs, gam = _pieces(A, D)
    K, Sinv = _dense_operator(A, D, pcs, gam)
    x = np.random.default_rng(3).standard_normal(int(A.rsz.sum()))
    gprime = []
    for s, k, B, F, E, Cm in pcs:
        f, g = x[s[:k]], x[s[k:]]
        gprime.append(g - E @ np.linalg.solve(B, f))
    z = Sinv @ np.concatenate(gprime)
    Kry = [z]
    for _ in range(msteps - 1):
        Kry.append(K @ Kry[-1])
    Y = np.stack(Kry, 1)
    c = np.linalg.lstsq(K @ Y, z, rcond=None)[0]
    y = Y @ c
    ref = np.zeros_like(x)
    o = 0
    for s, k, B, F, E, Cm in pcs:
        ng_i = len(s) - k
        yi = y[o:o + ng_i]
        ref[s[k:]] = yi
        ref[s[:k]] = np.linalg.solve(B, x[s[:k]] - F @ yi)
        o += ng_i
    out = D.apply(x)
    assert np.linalg.norm(out - ref) <= 1e-9 * np.linalg.norm(ref)


def test_enough_inner_steps_with_exact_factors_solve_A():
    """With exact local factorizations and as many inner steps as interface
    unknowns, the global Schur system is solved exactly, so one application
    is A^{-1} x."""
    A = _case(160, 3, seed=7, colscale=True)
    D0 = oracle.DDSchur(A, 2, 1, 2, 0.0, -1)
    D = oracle.DDSchur(A, 2, D0.ng, 2, 0.0, -1)
    x = np.random.default_rng(4).standard_normal(int(A.rsz.sum()))
    ref = np.linalg.solve(A.dense(), x)
    assert np.linalg.norm(D.apply(x) - ref) <= 1e-10 * np.linalg.norm(ref)


def test_one_subdomain_is_plain_vbarms():
    """No interface: the application is the plain VBARMS solve."""
    A = _case()
    D = oracle.DDSchur(A, 1, 3, 2, 1e-3, 10)
    assert D.ng == 0
    x = np.random.default_rng(1).standard_normal(int(A.rsz.sum()))
    assert np.array_equal(D.apply(x), oracle.Prec(A, 2, 1e-3, 10).apply(x))


def test_zero_right_hand_side_and_bad_arguments():
    A = _case(200, 3)
    D = oracle.DDSchur(A, 3, 4, 2, 1e-3, 10)
    assert np.array_equal(D.apply(np.zeros(int(A.rsz.sum()))), np.zeros(int(A.rsz.sum())))
    with pytest.raises(oracle.OracleError):
        oracle.DDSchur(A, 3, 0, 2, 1e-3, 10)
    with pytest.raises(oracle.OracleError):
        oracle.DDSchur(A, 0, 3, 2, 1e-3, 10)


def test_schur_fgmres_converges():
    A = _case(600, 4, seed=4)
    b = np.ones(int(A.rsz.sum()))
    D = oracle.DDSchur(A, 4, 5, 2, 1e-3, 20)
    x, its, rr, st = oracle.fgmres(A, D, b, rtol=1e-8)
    assert st == oracle.OK and rr <= 1e-8
    assert np.linalg.norm(b - oracle.spmv(A, x)) <= 1e-8 * np.linalg.norm(b) * (1 + 1e-6)
    Dj = oracle.DD(A, 4, 0, True, 2, 1e-3, 20)
    _, its_bj, _, _ = oracle.fgmres(A, Dj, b, rtol=1e-8)
    assert its <= its_bj, (its, its_bj)


@pytest.mark.parametrize("t,lfil", [(1e-3, 10), (1e-4, -1)])
def test_union_factorization_with_fixed_rows_is_the_local_ones(t, lfil):
    """Every step stays inside a connected component, so one factorization of
    the subdomains' union (each subdomain's interior rows, then its interface
    rows, interface rows fixed) applies, row for row, what the separate local
    factorizations apply, with and without fixed interface values (the layout
    the library factors)."""
    A = _case(500, 4, seed=8, colscale=True)
    D = oracle.DDSchur(A, 5, 3, 3, t, lfil)
    locs = [D.local(i) for i in range(5)]
    fixed = np.concatenate([(np.arange(len(D.rows(i)[0])) >= D.rows(i)[1]).astype(np.int32) for i in range(5)])
    U = oracle.block_diag(locs)
    Pu = oracle.Prec(U, 3, t, lfil, fixed=fixed)
    xu = np.random.default_rng(5).standard_normal(int(U.rsz.sum()))
    yu = Pu.apply(xu)
    o = 0
    for i, M in enumerate(locs):
        ni = int(M.rsz.sum())
        assert np.array_equal(yu[o:o + ni], D.local_prec(i).apply(xu[o:o + ni])), f"subdomain {i}"
        o += ni
    assert np.array_equal(Pu.last_fixed().astype(bool).sum(), fixed.sum())
