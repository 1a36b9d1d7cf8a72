"""Pins of the oracle's graph-based compression (Section 2.2, Alg. 1):
worked cases derived by hand, the T and N formulas against dense counting,
the invariants the method guarantees, and a brute-force replica of the
algorithm that recomputes every density from the dense pattern.  CPU only."""
import numpy as np
import pytest

import oracle
from paper_1508_02219_gb300 import synth


def _csr_from_dense(P):
    n = P.shape[0]
    rowptr = np.concatenate([[0], np.cumsum(P.sum(axis=1))]).astype(np.int64)
    colind = np.concatenate([np.flatnonzero(P[i]) for i in range(n)]).astype(np.int32) if n else np.zeros(0, np.int32)
    return rowptr, colind, np.ones(len(colind))


def _groups(c):
    off = np.concatenate([[0], np.cumsum(c.bsz)])
    return [sorted(c.perm[off[b]:off[b + 1]].tolist()) for b in range(len(c.bsz))]


def _path(n):
    P = np.zeros((n, n), bool)
    for i in range(n):
        for j in (i - 1, i, i + 1):
            if 0 <= j < n:
                P[i, j] = True
    return P


@pytest.mark.parametrize("mu,expected", [
    # Path 0-1-2-3-4 (closed neighbourhoods all distinct, so five singleton
    # supernodes).  mu = 0.6: {0,1} has T = 2*3*2 - 4 = 8, N = 2*(2+3) - (2+2)
    # = 6, 0.75: merged; X = {2} tries {0,1} first: T = 2*4*3 - 9 = 15,
    # N = 2*8 - 7 = 9, 0.6: merged; then {3}: T = 24, N = 12, 0.5: not; X = {3}
    # tries {0,1,2}: 0.5, not, then {4}: T = 8, N = 6, 0.75: merged.
    (0.6, [[0, 1, 2], [3, 4]]),
    # mu = 0.75: {0,1} merges (0.75); {2} with {0,1}: 0.6, with {3}:
    # T = 2*4*2 - 4 = 12, N = 2*6 - 4 = 8, 0.667: neither; {3} with {2}: 0.667,
    # with {4}: 0.75: merged.
    (0.75, [[0, 1], [2], [3, 4]]),
    # above every pair's 0.75: nothing merges
    (0.76, [[0], [1], [2], [3], [4]]),
])
def test_worked_path_cases(mu, expected):
    c = oracle.graph_compress(5, *_csr_from_dense(_path(5)), mu)
    assert _groups(c) == expected
    assert np.array_equal(c.perm, np.arange(5))


def _closed(P):
    return P | P.T | np.eye(P.shape[0], dtype=bool)


def _cross_density(B, S):
    """N and T of vertex set S counted on the dense closed pattern B: the
    rectangles S x adj(S) and adj(S) x S, their area and their nonzeros."""
    S = np.asarray(sorted(S))
    AS = np.flatnonzero(B[S].any(axis=0))
    mask = np.zeros_like(B)
    mask[np.ix_(S, AS)] = True
    mask[np.ix_(AS, S)] = True
    return int((B & mask).sum()), int(mask.sum())


def _classes(B):
    """Vertices with identical closed neighbourhoods, brute force."""
    seen, out = {}, []
    for i in range(B.shape[0]):
        k = B[i].tobytes()
        if k not in seen:
            seen[k] = len(out)
            out.append([])
        out[seen[k]].append(i)
    return out


def _random_pattern(n, deg, seed, sym=True, twins=0):
    rng = np.random.default_rng(seed)
    P = np.zeros((n, n), bool)
    for i in range(n):
        P[i, rng.choice(n, size=min(deg, n), replace=False)] = True
    if sym:
        P |= P.T
    np.fill_diagonal(P, True)
    for _ in range(twins):  # vertices with identical closed neighbourhoods
        i, j = rng.choice(n, 2, replace=False)
        B = _closed(P)
        row = B[i].copy()
        row[j] = True
        P[j] = row
        P[:, j] = row
        P[i, j] = P[j, i] = True
    return P


def _replica(P, mu):
    """Alg. 1 step by step with every density counted on the dense pattern
    (readings G1-G5), for tiny inputs."""
    B = _closed(P)
    n = B.shape[0]
    key = [int(np.flatnonzero(B[i]).sum()) for i in range(n)]
    order = sorted(range(n), key=lambda i: (key[i], i))
    done, V = set(), []
    for x, i in enumerate(order):
        if i in done:
            continue
        Y = [i]
        done.add(i)
        for j in order[x + 1:]:
            if key[j] != key[i]:
                break
            if j not in done and np.array_equal(B[i], B[j]):
                Y.append(j)
                done.add(j)
        V.append(set(Y))
    V.sort(key=min)
    alive = [True] * len(V)
    owner = {v: z for z, Y in enumerate(V) for v in Y}
    for x in range(len(V)):
        if not alive[x]:
            continue
        adjX = set(np.flatnonzero(B[sorted(V[x])].any(axis=0)).tolist())
        cand = sorted({owner[u] for u in adjX if owner[u] != x}, key=lambda z: min(V[z]))
        for z in cand:
            N, T = _cross_density(B, V[x] | V[z])
            if N >= mu * T:
                for v in V[z]:
                    owner[v] = x
                V[x] |= V[z]
                alive[z] = False
    return sorted(sorted(Y) for z, Y in enumerate(V) if alive[z])


@pytest.mark.parametrize("seed,sym,twins", [(0, True, 4), (1, False, 3), (2, True, 0), (3, False, 6)])
@pytest.mark.parametrize("mu", [0.3, 0.55, 0.7, 0.9])
def test_matches_brute_force_replica(seed, sym, twins, mu):
    P = _random_pattern(24, 3, seed, sym, twins)
    c = oracle.graph_compress(24, *_csr_from_dense(P), mu)
    assert _groups(c) == _replica(P, mu)


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("mu", [0.5, 0.7, 0.9])
def test_invariants(seed, mu):
    """Supernodes are unions of the exact classes; every merged supernode's
    block row and column have density N / T >= mu (counted densely); unmerged
    classes have density 1; blocks are ordered by their smallest vertex."""
    m = synth.geometric(60, 3, seed=seed)
    n = m.n
    P = np.zeros((n, n), bool)
    for i in range(n):
        P[i, m.colind[m.rowptr[i]:m.rowptr[i + 1]]] = True
    B = _closed(P)
    c = oracle.graph_compress(n, m.rowptr, m.colind, m.val, mu)
    groups = _groups(c)
    assert sorted(v for g in groups for v in g) == list(range(n))
    assert [g[0] for g in groups] == sorted(g[0] for g in groups)
    cls = {v: k for k, C in enumerate(_classes(B)) for v in C}
    for g in groups:
        ks = {cls[v] for v in g}
        assert all(cls[v] in ks for v in g)
        assert sum(1 for v in range(n) if cls[v] in ks) == len(g), "a class was split"
        N, T = _cross_density(B, g)
        if len(ks) > 1:
            assert N >= mu * T
        else:
            assert N == T
    # the VBCSR is P_B A P_B^T, zero padded
    A = np.zeros((n, n))
    for i in range(n):
        A[i, m.colind[m.rowptr[i]:m.rowptr[i + 1]]] = m.val[m.rowptr[i]:m.rowptr[i + 1]]
    assert np.array_equal(c.A.dense(), A[np.ix_(c.perm, c.perm)])


def test_mu_above_one_keeps_the_exact_classes():
    m = synth.grid_7pt(4, 4, 4, 3, seed=0, scramble=True)
    P = np.zeros((m.n, m.n), bool)
    for i in range(m.n):
        P[i, m.colind[m.rowptr[i]:m.rowptr[i + 1]]] = True
    c = oracle.graph_compress(m.n, m.rowptr, m.colind, m.val, 1.01)
    assert _groups(c) == sorted(sorted(C) for C in _classes(_closed(P)))
    # the planted 3x3 node blocks are exact classes (identical closed
    # neighbourhoods), so the grid's nodes come back whole
    assert sorted(set(c.bsz.tolist())) == [3] and c.av_bd == 1.0


def test_invalid_arguments():
    rp, ci, v = _csr_from_dense(_path(4))
    with pytest.raises(oracle.OracleError):
        oracle.graph_compress(4, rp, ci, v, -0.1)
    bad = ci.copy()
    bad[0] = 7
    with pytest.raises(oracle.OracleError):
        oracle.graph_compress(4, rp, bad, v, 0.5)
