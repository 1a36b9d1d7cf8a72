"""The compression variants on the GPU against the oracle, P_B, the block
sizes and the VBCSR matrix P_B A P_B^T bit for bit.  Graph-based compression
(Section 2.2, Alg. 1): the hand-derived path cases, random patterns with
planted identical neighbourhoods (symmetric and not), geometric matrices of
the input recipe and a scrambled grid (mu > 1 keeps the exact classes).  The
two-pass variant of Section 2.1: the hand-derived case where it differs from
the one-pass method, exact node blocks with perturbed rows, and geometric
matrices with exact and approximate blocks."""
import numpy as np
import pytest

import oracle
from gpu_helpers import as_dict, compare_vb, cuda_ok, torch, vb
from paper_1508_02219_gb300 import synth
from test_oracle_graph import _csr_from_dense, _path, _random_pattern

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]


def _both(n, rowptr, colind, val, mu, on_device=False):
    V = vb()
    if on_device:
        A = V.vbarms_compress_graph(n, torch.from_numpy(rowptr).cuda(), torch.from_numpy(colind).cuda(),
                                    torch.from_numpy(val).cuda(), mu)
    else:
        A = V.vbarms_compress_graph(n, rowptr, colind, val, mu)
    c = oracle.graph_compress(n, rowptr, colind, val, mu)
    g = A.export()
    assert np.array_equal(g["perm"], c.perm), "P_B differs"
    assert np.array_equal(g["bsz"], c.bsz), "block sizes differ"
    compare_vb(dict(rsz=g["bsz"], csz=g["bsz"], bptr=g["bptr"], bcol=g["bcol"], voff=g["voff"], val=g["val"]),
               as_dict(c.A), "VBSR")
    q = A.query()
    assert q["av_bd"] == c.av_bd and q["av_bs"] == c.av_bs
    return g, c


@pytest.mark.parametrize("mu", [0.6, 0.75, 0.76])
def test_path_cases(mu):
    _both(5, *_csr_from_dense(_path(5)), mu)


@pytest.mark.parametrize("seed,sym,twins", [(0, True, 4), (1, False, 3), (2, True, 0), (3, False, 6)])
@pytest.mark.parametrize("mu", [0.3, 0.55, 0.7, 0.9])
def test_random_patterns(seed, sym, twins, mu):
    P = _random_pattern(24, 3, seed, sym, twins)
    _both(24, *_csr_from_dense(P), mu)


@pytest.mark.parametrize("nodes,ell,seed,mu", [(2000, 4, 0, 0.5), (2000, 4, 1, 0.7), (3000, 6, 2, 0.8),
                                               (1500, 3, 3, 0.3)])
def test_geometric(nodes, ell, seed, mu):
    m = synth.geometric(nodes, ell, seed=seed)
    g, c = _both(m.n, m.rowptr, m.colind, m.val, mu, on_device=True)
    assert len(g["bsz"]) < m.n  # something merged


def test_exact_node_blocks_and_mu_above_one():
    m = synth.grid_7pt(6, 6, 6, 4, seed=1, scramble=True)
    g, c = _both(m.n, m.rowptr, m.colind, m.val, 1.01)
    assert sorted(set(g["bsz"].tolist())) == [4]


def test_empty_and_invalid():
    V = vb()
    A = V.vbarms_compress_graph(0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0), 0.5)
    assert A.query()["nblk"] == 0
    rp, ci, v = _csr_from_dense(_path(4))
    with pytest.raises(V.VbarmsError) as e:
        V.vbarms_compress_graph(4, rp, ci, v, -0.1)
    assert e.value.status == V.VB_EINVAL
    bad = ci.copy()
    bad[0] = 7
    with pytest.raises(V.VbarmsError) as e:
        V.vbarms_compress_graph(4, rp, bad, v, 0.5)
    assert e.value.status == V.VB_EINVAL


# ---- the two-pass variant of Section 2.1 ---------------------------------
from test_oracle_two_pass import _csr as _pcsr, _perturbed  # noqa: E402


def _both_two_pass(n, rowptr, colind, val, tau, on_device=False):
    V = vb()
    if on_device:
        A = V.vbarms_compress_two_pass(n, torch.from_numpy(rowptr).cuda(), torch.from_numpy(colind).cuda(),
                                       torch.from_numpy(val).cuda(), tau)
    else:
        A = V.vbarms_compress_two_pass(n, rowptr, colind, val, tau)
    c = oracle.compress_two_pass(n, rowptr, colind, val, tau)
    g = A.export()
    assert np.array_equal(g["perm"], c.perm), "P_B differs"
    assert np.array_equal(g["bsz"], c.bsz), "block sizes differ"
    compare_vb(dict(rsz=g["bsz"], csz=g["bsz"], bptr=g["bptr"], bcol=g["bcol"], voff=g["voff"], val=g["val"]),
               as_dict(c.A), "VBSR")
    return g, c


def test_two_pass_worked_case():
    pats = [set(range(8)), {0, 1, 2, 3}, {0, 1, 2, 3}, {4, 5, 6, 7}, {4}, {5}, {6}, {7}]
    g, c = _both_two_pass(*_pcsr(pats, 8), 0.7)
    assert g["bsz"].tolist() == [3, 1, 1, 1, 1, 1]


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
@pytest.mark.parametrize("tau", [0.5, 0.75, 0.9, 0.97])
def test_two_pass_perturbed_node_blocks(seed, tau):
    rows = _perturbed(seed)
    _both_two_pass(*_pcsr(rows, len(rows)), tau)


@pytest.mark.parametrize("nodes,ell,seed,tau", [(3000, 6, 0, 0.8), (2000, 4, 1, 0.9), (2000, 5, 2, 1.0)])
def test_two_pass_geometric(nodes, ell, seed, tau):
    m = synth.geometric(nodes, ell, seed=seed, approx=False)
    _both_two_pass(m.n, m.rowptr, m.colind, m.val, tau, on_device=True)
    m = synth.geometric(nodes, ell, seed=seed)
    _both_two_pass(m.n, m.rowptr, m.colind, m.val, tau, on_device=True)
