"""Pins of the oracle's Step 1 (angle-based compression, Section 2.1; block
permutation, Eq. 3) against brute force and closed forms.  CPU only."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1508_02219_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def brute_groups(m: synth.CSR, tau_num: int, tau_den: int):
    """All-pairs cosine with exact integer arithmetic and the sequential
    leader greedy.  tau = tau_num / tau_den must be a dyadic rational so that
    the oracle's double comparison is exact too."""
    pats = [set(m.colind[m.rowptr[i]:m.rowptr[i + 1]].tolist()) for i in range(m.n)]
    leader = [-1] * m.n
    for i in range(m.n):
        if leader[i] != -1:
            continue
        leader[i] = i
        for j in range(i + 1, m.n):
            if leader[j] != -1 or not pats[i] or not pats[j]:
                continue
            c = len(pats[i] & pats[j])
            # cos >= tau  <=>  c^2 * den^2 >= num^2 * |Pi| |Pj|
            if c * c * tau_den * tau_den >= tau_num * tau_num * len(pats[i]) * len(pats[j]):
                leader[j] = i
    leaders = sorted(set(leader))
    perm = [r for L in leaders for r in range(m.n) if leader[r] == L]
    sizes = [sum(1 for r in range(m.n) if leader[r] == L) for L in leaders]
    return np.array(perm), np.array(sizes)


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("tau", [(1, 1), (3, 4), (1, 2), (7, 8)])
def test_compress_matches_bruteforce_geometric(seed, tau):
    m = synth.geometric(40, 3, seed=seed, scramble=True)
    perm, sizes = brute_groups(m, *tau)
    c = oracle.compress(m.n, m.rowptr, m.colind, m.val, tau[0] / tau[1])
    assert np.array_equal(c.perm, perm)
    assert np.array_equal(c.bsz, sizes)


@pytest.mark.parametrize("seed", [3, 4])
def test_compress_matches_bruteforce_random(seed):
    m = synth.random_sparse(120, 0.05, seed=seed, empty_rows=3)
    for tau in [(1, 1), (1, 2), (1, 4)]:
        perm, sizes = brute_groups(m, *tau)
        c = oracle.compress(m.n, m.rowptr, m.colind, m.val, tau[0] / tau[1])
        assert np.array_equal(c.perm, perm)
        assert np.array_equal(c.bsz, sizes)


@pytest.mark.parametrize("ell", [1, 2, 5, 6])
def test_tau1_recovers_planted_blocks(ell):
    """Closed form: tau = 1 finds exactly the node blocks of a scrambled grid
    (closed 7-point neighbourhoods are distinct), so av_bd = 1, av_bs = ell."""
    m = synth.grid_7pt(6, 5, 4, ell, seed=ell, scramble=True)
    c = oracle.compress(m.n, m.rowptr, m.colind, m.val, 1.0)
    node = m.meta["node_of_row"][m.meta["scramble"]]
    grp = np.repeat(np.arange(len(c.bsz)), c.bsz)
    assert len(c.bsz) == 120
    assert (c.bsz == ell).all()
    for g in range(len(c.bsz)):
        assert len(set(node[c.perm[grp == g]].tolist())) == 1
    assert c.av_bd == 1.0
    assert c.av_bs == float(ell)


def test_grid10_closed_form_golden():
    """10x10x10 grid, ell=5: 1000 supernodes and 1000 + 2*3*10*10*9 = 6400
    stored blocks of the quotient graph (Section 3, E_B), all dense."""
    with open(os.path.join(GOLDEN, "grid10_l5_closed_form.json")) as f:
        g = json.load(f)
    m = synth.grid_7pt(10, 10, 10, 5, seed=0, scramble=True)
    c = oracle.compress(m.n, m.rowptr, m.colind, m.val, 1.0)
    assert len(c.bsz) == g["nblk"]
    assert c.A.nnzb == g["nnzb"]
    assert c.av_bd == g["av_bd"] and c.av_bs == g["av_bs"]
    assert m.nnz == g["nnz"]


def test_vbsr_reproduces_permuted_matrix():
    m = synth.geometric(300, 4, seed=5)
    c = oracle.compress(m.n, m.rowptr, m.colind, m.val, 0.75)
    d = m.dense()[np.ix_(c.perm, c.perm)]
    assert np.array_equal(c.A.dense(), d)
    # a block is stored iff a stored entry falls in it
    pat = np.zeros((m.n, m.n), bool)
    rows = np.repeat(np.arange(m.n), np.diff(m.rowptr))
    pat[rows, m.colind] = True
    pat = pat[np.ix_(c.perm, c.perm)]
    off = np.concatenate([[0], np.cumsum(c.bsz)])
    stored = set()
    for I in range(len(c.bsz)):
        for b in range(c.A.bptr[I], c.A.bptr[I + 1]):
            stored.add((I, int(c.A.bcol[b])))
        cols = c.A.bcol[c.A.bptr[I]:c.A.bptr[I + 1]]
        assert (np.diff(cols) > 0).all()
    expect = set()
    for I in range(len(c.bsz)):
        for J in range(len(c.bsz)):
            if pat[off[I]:off[I + 1], off[J]:off[J + 1]].any():
                expect.add((I, J))
    assert stored == expect
    padded = sum(c.bsz[I] * c.bsz[J] for I, J in stored)
    assert c.av_bd == pytest.approx(m.nnz / padded, rel=0, abs=0)
    assert c.av_bs == m.n / len(c.bsz)


def test_edge_cases():
    # n = 1
    m = synth.from_dense(np.array([[2.0]]))
    c = oracle.compress(1, m.rowptr, m.colind, m.val, 1.0)
    assert list(c.bsz) == [1]
    # all rows identical -> one group; dense matrix at tau = 1 -> one block
    a = np.random.default_rng(0).standard_normal((9, 9))
    m = synth.from_dense(a, keep_zeros=True)
    c = oracle.compress(9, m.rowptr, m.colind, m.val, 1.0)
    assert list(c.bsz) == [9] and c.A.nnzb == 1 and c.av_bd == 1.0
    # empty rows are singletons and join nothing
    a = np.eye(6)
    a[2, :] = 0
    a[4, :] = 0
    a[0, 1] = a[1, 0] = 1.0
    m = synth.from_dense(a)
    c = oracle.compress(6, m.rowptr, m.colind, m.val, 0.5)
    grp = np.repeat(np.arange(len(c.bsz)), c.bsz)
    g_of = dict(zip(c.perm.tolist(), grp.tolist()))
    assert g_of[0] == g_of[1]
    assert list(c.bsz).count(1) == 4
    # n = 0
    c = oracle.compress(0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0), 1.0)
    assert len(c.bsz) == 0


@pytest.mark.parametrize("bad", ["unsorted", "duplicate", "range", "tau0", "tau_gt1"])
def test_invalid_input(bad):
    m = synth.from_dense(np.eye(4) + np.diag(np.ones(3), 1))
    rp, ci, tau = m.rowptr.copy(), m.colind.copy(), 1.0
    if bad == "unsorted":
        ci[0], ci[1] = ci[1], ci[0]
    elif bad == "duplicate":
        ci[1] = ci[0]
    elif bad == "range":
        ci[-1] = 4
    elif bad == "tau0":
        tau = 0.0
    else:
        tau = 1.5
    with pytest.raises(oracle.OracleError) as e:
        oracle.compress(4, rp, ci, m.val, tau)
    assert e.value.status == oracle.EINVAL
