"""Pins of the oracle's solve phase (Alg. 2, VBARMS_Solve) and of FGMRES
against dense linear algebra.  CPU only."""
import numpy as np
import pytest

import oracle
from paper_1508_02219_gb300 import synth
from test_oracle_factor import (_offsets, last_level_dense, level_factor_dense, scalar_perm)


def dense_operator(P: oracle.Prec, lev: int = 0) -> np.ndarray:
    """Dense M_lev assembled from the exported factors:
    M_l = S1^{-1} P_I^T [[P^T L, 0],[G, I]] [[U, W],[0, M_{l+1}]] P_I S2^{-1},
    and the last level M = S1^{-1} (I + L)(D + U) S2^{-1} (Eq. 7, Alg. 2)."""
    if lev == P.levels:
        A, LU, _, _ = last_level_dense(P)
        r, c = P.vec(lev, "r"), P.vec(lev, "c")
        return (LU / r[:, None]) / c[None, :]
    A = P.mat(lev, "A")
    Lo, Up, nf = level_factor_dense(P, lev)
    Up = Up.copy()
    Up[nf:, nf:] = dense_operator(P, lev + 1)
    sp = scalar_perm(A.rsz, P.vec(lev, "pI"))
    n = len(sp)
    Pm = np.eye(n)[sp]  # (P_I x) = x[sp]
    r, c = P.vec(lev, "r"), P.vec(lev, "c")
    M = Pm.T @ (Lo @ Up) @ Pm
    return (M / r[:, None]) / c[None, :]


@pytest.mark.parametrize("nlev,t,lfil", [(1, 1e-3, -1), (2, 1e-3, 5), (3, 1e-2, 3), (0, 1e-3, -1)])
@pytest.mark.parametrize("dominance", [None, 1.5])
def test_apply_is_inverse_of_assembled_operator(nlev, t, lfil, dominance):
    m = synth.geometric(50, 3, seed=2, dominance=dominance)
    c = oracle.compress(m.n, m.rowptr, m.colind, m.val, 0.75)
    P = oracle.Prec(c.A, nlev, t, lfil)
    M = dense_operator(P)
    b = np.random.default_rng(0).standard_normal(m.n)
    x = P.apply(b)
    np.testing.assert_allclose(M @ x, b, rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("nlev", [1, 2, 4])
def test_no_drop_multilevel_is_exact(nlev):
    """t = 0 and no lfil: every level and the last-level block LU are exact,
    so M = A, M^{-1} A x = x and FGMRES converges in one iteration."""
    m = synth.geometric(80, 4, seed=3)
    c = oracle.compress(m.n, m.rowptr, m.colind, m.val, 0.75)
    P = oracle.Prec(c.A, nlev, 0.0, -1)
    Ad = c.A.dense()
    x = np.random.default_rng(1).standard_normal(m.n)
    np.testing.assert_allclose(P.apply(Ad @ x), x, rtol=1e-10, atol=1e-10)
    b = Ad @ np.ones(m.n)
    xs, its, rr, st = oracle.fgmres(c.A, P, b, rtol=1e-8)
    assert st == oracle.OK and its == 1 and rr <= 1e-8


def test_gmres_residual_is_krylov_minimum():
    """Unrestarted GMRES: after k steps the residual is the least-squares
    minimum over x0 + K_k(A, r0)."""
    rng = np.random.default_rng(5)
    m = synth.random_sparse(40, 0.1, seed=5)
    c = oracle.compress(m.n, m.rowptr, m.colind, m.val, 1.0)
    Ad = c.A.dense()
    b = rng.standard_normal(m.n)
    for k in [1, 3, 7, 12]:
        x, its, rr, st = oracle.fgmres(c.A, None, b, rtol=1e-14, restart=60, maxit=k)
        assert its == k and st == oracle.ENOCONV
        K = np.zeros((m.n, k))
        v = b.copy()
        for j in range(k):
            K[:, j] = v
            v = Ad @ v
        Q, _ = np.linalg.qr(K)
        y, *_ = np.linalg.lstsq(Ad @ Q, b, rcond=None)
        best = np.linalg.norm(b - Ad @ Q @ y) / np.linalg.norm(b)
        assert rr == pytest.approx(best, rel=1e-7)


def test_fgmres_matches_dense_solve_and_restarts():
    m = synth.geometric(120, 3, seed=8)
    c = oracle.compress(m.n, m.rowptr, m.colind, m.val, 0.75)
    P = oracle.Prec(c.A, 2, 1e-2, 4)
    Ad = c.A.dense()
    b = Ad @ np.ones(m.n)
    for restart in [5, 50]:
        x, its, rr, st = oracle.fgmres(c.A, P, b, rtol=1e-10, restart=restart)
        assert st == oracle.OK and rr <= 1e-10
        np.testing.assert_allclose(x, np.linalg.solve(Ad, b), rtol=1e-7, atol=1e-7)
        assert rr == pytest.approx(np.linalg.norm(b - Ad @ x) / np.linalg.norm(b), rel=1e-6, abs=1e-15)
    x, its, rr, st = oracle.fgmres(c.A, None, b, rtol=1e-12, restart=5, maxit=3)
    assert st == oracle.ENOCONV and its == 3
    x, its, rr, st = oracle.fgmres(c.A, P, np.zeros(m.n))
    assert its == 0 and rr == 0.0 and not x.any()


def test_spmv_matches_dense():
    m = synth.geometric(70, 5, seed=9)
    c = oracle.compress(m.n, m.rowptr, m.colind, m.val, 0.75)
    x = np.random.default_rng(2).standard_normal(m.n)
    np.testing.assert_allclose(oracle.spmv(c.A, x), c.A.dense() @ x, rtol=1e-13, atol=1e-13)
