"""The synthetic input recipe (the generator both sides are fed from): the
structure, value distributions, planted conditioning and batch shapes that
the design states.  CPU only."""
import numpy as np
import pytest

from paper_1508_02219_gb300 import synth


def _node_blocks(m, ell):
    """{(a, b): dense ell x ell block} of a node-blocked CSR (dropped entries 0)."""
    out = {}
    for i in range(m.n):
        a = i // ell
        for q in range(m.rowptr[i], m.rowptr[i + 1]):
            j = m.colind[q]
            blk = out.setdefault((a, j // ell), np.zeros((ell, ell)))
            blk[i % ell, j % ell] = m.val[q]
    return out


def test_geometric_structure_and_degree():
    n_nodes, ell = 4000, 3
    m = synth.geometric(n_nodes, ell, seed=1, approx=False)
    assert m.n == n_nodes * ell
    r = (3 * 15 / (4 * np.pi * n_nodes)) ** (1 / 3)
    assert m.meta["radius"] == pytest.approx(r)
    # exact dense node blocks, symmetric node graph
    B = _node_blocks(m, ell)
    assert all(((a, b) in B) == ((b, a) in B) for (a, b) in B)
    deg = np.bincount([a for (a, b) in B if a != b], minlength=n_nodes)
    assert 14.0 < deg.mean() < 16.0  # Poisson-like around 15 neighbours
    assert (np.diff(m.rowptr) == ell * (deg.repeat(ell) + 1)).all()


def test_approximate_blocks_drop_and_noise():
    n_nodes, ell = 3000, 3
    m = synth.geometric(n_nodes, ell, seed=2, approx=True)
    ex = synth.geometric(n_nodes, ell, seed=2, approx=False)
    assert m.meta["approx"] and m.nnz < ex.nnz
    row = np.repeat(np.arange(m.n), np.diff(m.rowptr))
    assert (np.diff(m.rowptr) > 0).all()
    diag_kept = np.zeros(m.n, bool)
    diag_kept[row[m.colind == row]] = True
    assert diag_kept.all(), "scalar diagonal always kept"
    # off-diagonal scalars (those outside the scalar diagonal) dropped with p = 0.1
    ex_row = np.repeat(np.arange(ex.n), np.diff(ex.rowptr))
    off_ex = int((ex.colind != ex_row).sum())
    off_m = int((m.colind != row).sum())
    assert abs(1 - off_m / off_ex - 0.1) < 0.005
    # kept entries of off-diagonal node blocks: N(0, 0.1^2) + N(0, 1e-3)
    offblk = (m.colind // ell) != (row // ell)
    v = m.val[offblk]
    assert abs(v.var() / (0.01 + 1e-3) - 1) < 0.03 and abs(v.mean()) < 2e-3


def test_dominance_and_planted_conditioning():
    n_nodes, ell = 3000, 4
    m = synth.geometric(n_nodes, ell, seed=3, dominance=1.5, ill_frac=0.01)
    ill = set(m.meta["ill_nodes"].tolist())
    assert len(ill) == 30
    B = _node_blocks(m, ell)
    off = np.zeros(n_nodes)
    for (a, b), blk in B.items():
        if a != b:
            off[a] += np.linalg.norm(blk)
    for a in range(n_nodes):
        s = np.linalg.svd(B[(a, a)], compute_uv=False)
        if a in ill:
            assert s[0] / s[-1] == pytest.approx(1e6, rel=1e-6)
            assert s[0] == pytest.approx(1.5 * off[a], rel=1e-10)
        else:
            # sigma_min(D_a) = 1.5 sum_b ||A_ab||_F >= 1.5 sum_b ||A_ab||_2
            assert s[-1] == pytest.approx(1.5 * off[a], rel=1e-10)
            assert s[0] / s[-1] <= 2.0 * (1 + 1e-10)


def test_grid_structure_and_values():
    m = synth.grid_7pt(6, 5, 4, 3, seed=4)
    ell = 3
    B = _node_blocks(m, ell)
    nodes = 6 * 5 * 4
    assert m.n == nodes * ell
    for a in range(nodes):
        x, y, z = a % 6, (a // 6) % 5, a // 30
        nb = {a}
        for d, (c, n) in enumerate([(x, 6), (y, 5), (z, 4)]):
            step = [1, 6, 30][d]
            if c > 0:
                nb.add(a - step)
            if c < n - 1:
                nb.add(a + step)
        assert {b for (aa, b) in B if aa == a} == nb
    diag = np.array([B[(a, a)] for a in range(nodes)])
    assert abs(np.diagonal(diag, axis1=1, axis2=2).mean() - 8.0) < 0.3
    offv = np.concatenate([blk.ravel() for (a, b), blk in B.items() if a != b])
    assert abs(offv.std() - 0.1) < 0.01


def test_batch_shapes_and_workload_scaling():
    shapes = synth.batch_shapes("batch32", seed=0)
    assert len(shapes) == 32
    assert all(20_000 <= n <= 300_000 and e in (4, 5, 6) for n, e in shapes)
    assert shapes == synth.batch_shapes("batch32", seed=0)
    assert sum(n for n, _ in shapes) == pytest.approx(3.67e6, rel=0.01)
    m = synth.make_workload("geo500k_l6", seed=0, scale=0.001)
    assert m.meta["nodes"] == 500 and m.n == 3000
    b = synth.ones_rhs(m)
    assert np.allclose(b, m.matvec(np.ones(m.n)))
