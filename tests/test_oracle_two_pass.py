"""Pins of the oracle's two-pass variant of the angle method (Section 2.1:
identical patterns grouped by a checksum pass, then each unassigned row added
to an existing group by angle): a hand-derived case where it differs from
the one-pass greedy, a brute-force replica, its invariants, and tau = 1
where both methods group exactly the identical patterns.  CPU only."""
import numpy as np
import pytest

import oracle
from paper_1508_02219_gb300 import synth


def _csr(patterns, n):
    rowptr = np.concatenate([[0], np.cumsum([len(p) for p in patterns])]).astype(np.int64)
    colind = np.concatenate([np.asarray(sorted(p), np.int32) for p in patterns]) if patterns else np.zeros(0, np.int32)
    return n, rowptr, colind.astype(np.int32), np.ones(len(colind))


def _groups(c):
    off = np.concatenate([[0], np.cumsum(c.bsz)])
    return [sorted(c.perm[off[b]:off[b + 1]].tolist()) for b in range(len(c.bsz))]


def test_worked_case_differs_from_the_one_pass_greedy():
    """Rows 1 and 2 share the pattern {0,1,2,3}; row 0 is {0..7}, row 3 is
    {4,5,6,7}, rows 4-7 are single columns.  tau = 0.7 (tau^2 = 0.49).
    One pass: leader 0 claims 1 and 2 (|P0 n P1|^2 = 16 >= 0.49 * 8 * 4 =
    15.68) and 3 (also 16 >= 15.68).  Two passes: {1, 2} is a group; row 0
    joins it (16 >= 0.49 * 8 * 4), row 3 shares nothing with {0,1,2,3} and
    stays alone, rows 4-7 too."""
    pats = [set(range(8)), {0, 1, 2, 3}, {0, 1, 2, 3}, {4, 5, 6, 7}, {4}, {5}, {6}, {7}]
    args = _csr(pats, 8)
    assert _groups(oracle.compress(*args, 0.7)) == [[0, 1, 2, 3], [4], [5], [6], [7]]
    assert _groups(oracle.compress_two_pass(*args, 0.7)) == [[0, 1, 2], [3], [4], [5], [6], [7]]


def _replica(rowptr, colind, n, tau):
    P = [frozenset(colind[rowptr[i]:rowptr[i + 1]].tolist()) for i in range(n)]
    cls = {}
    for i in range(n):
        cls.setdefault(P[i], []).append(i)
    groups = sorted([sorted(v) for k, v in cls.items() if len(v) >= 2 and len(k) > 0], key=lambda g: g[0])
    assigned = {i for g in groups for i in g}
    joined = [[] for _ in groups]
    alone = []
    for j in range(n):
        if j in assigned:
            continue
        hit = None
        if P[j]:
            for gi, g in enumerate(groups):
                c = len(P[j] & P[g[0]])
                if c * c >= (tau * tau) * (len(P[j]) * len(P[g[0]])):  # the oracle's one rounded product
                    hit = gi
                    break
        if hit is None:
            alone.append([j])
        else:
            joined[hit].append(j)
    return sorted([sorted(g + jn) for g, jn in zip(groups, joined)] + alone, key=lambda g: g[0])


def _perturbed(seed, nodes=40, ell=3, k=25):
    """Exact node blocks with k rows missing one off-diagonal entry: identical
    classes exist and the perturbed rows sit close to them."""
    m = synth.geometric(nodes, ell, seed=seed, approx=False)
    rng = np.random.default_rng(seed)
    rows = [set(m.colind[m.rowptr[i]:m.rowptr[i + 1]].tolist()) for i in range(m.n)]
    for i in rng.choice(m.n, k, replace=False):
        off = sorted(rows[i] - {i})
        if off:
            rows[i].discard(off[rng.integers(len(off))])
    return rows


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
@pytest.mark.parametrize("tau", [0.5, 0.75, 0.9, 0.97])
def test_matches_brute_force_replica(seed, tau):
    rows = _perturbed(seed)
    n, rowptr, colind, val = _csr(rows, len(rows))
    c = oracle.compress_two_pass(n, rowptr, colind, val, tau)
    ref = _replica(rowptr, colind, n, tau)
    assert _groups(c) == ref
    P = [frozenset(r) for r in rows]
    joined = sum(1 for g in ref if len(g) > 1 for v in g if sum(P[w] == P[v] for w in g) == 1)
    assert joined > 0 or tau > 0.95, "pass 2 joined nothing: the case pins nothing"


@pytest.mark.parametrize("seed", [0, 1])
def test_invariants(seed):
    tau = 0.8
    m = synth.grid_7pt(4, 4, 4, 3, seed=seed, scramble=True)
    # perturb some rows so that pass 2 has work
    rng = np.random.default_rng(seed)
    rows = [set(m.colind[m.rowptr[i]:m.rowptr[i + 1]].tolist()) for i in range(m.n)]
    for i in rng.choice(m.n, 20, replace=False):
        rows[i].discard(next(iter(rows[i] - {i}), i))
    n, rowptr, colind, val = _csr(rows, m.n)
    c = oracle.compress_two_pass(n, rowptr, colind, val, tau)
    P = [frozenset(r) for r in rows]
    groups = _groups(c)
    assert sorted(v for g in groups for v in g) == list(range(n))
    assert [g[0] for g in groups] == sorted(g[0] for g in groups)
    multi = []
    for g in groups:
        pats = {}
        for v in g:
            pats.setdefault(P[v], []).append(v)
        if len(g) == 1:
            continue
        core = [k for k, v in pats.items() if len(v) >= 2]
        assert len(core) == 1, "a group holds one pass-1 class"
        multi.append(core[0])
        for v in g:
            c2 = len(P[v] & core[0]) ** 2
            assert c2 >= tau * tau * len(P[v]) * len(core[0]) * (1 - 1e-12)
    for g in groups:
        if len(g) == 1 and P[g[0]] not in multi:
            v = g[0]
            for k in multi:
                assert len(P[v] & k) ** 2 < tau * tau * len(P[v]) * len(k) * (1 + 1e-12)


@pytest.mark.parametrize("make", [lambda: synth.geometric(150, 4, seed=5),
                                  lambda: synth.grid_7pt(5, 5, 5, 4, seed=1, scramble=True)])
def test_tau_one_is_the_one_pass_method(make):
    m = make()
    a = oracle.compress(m.n, m.rowptr, m.colind, m.val, 1.0)
    b = oracle.compress_two_pass(m.n, m.rowptr, m.colind, m.val, 1.0)
    assert np.array_equal(a.perm, b.perm) and np.array_equal(a.bsz, b.bsz)
    assert np.array_equal(a.A.val, b.A.val)
