"""Batched factorization (one factorization of the block-diagonal union of
independent matrices, one launch per phase): every matrix's preconditioner
must equal the one its own factorization gives, bit for bit, and the FP64
batch is pinned to the CPU oracle through those single factorizations."""
import numpy as np
import pytest

import oracle
from gpu_helpers import compare_factor, cuda_ok, gpu_compress, torch, vb
from paper_1508_02219_gb300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]


def _mats():
    # uneven sizes and unknowns per node, as in a batch of Jacobians
    return [
        (synth.geometric(1500, 4, seed=21), 0.8),
        (synth.grid_7pt(8, 8, 8, 5, seed=22, scramble=True), 1.0),
        (synth.geometric(2600, 6, seed=23), 0.8),
        (synth.geometric(400, 5, seed=24), 0.75),
    ]


def _apply(V, P, x):
    y = torch.zeros_like(x)
    V.vbarms_apply(P, x, y)
    return y


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batched_equals_single(precision):
    V = vb()
    mats = _mats()
    As = [gpu_compress(m, tau) for m, tau in mats]
    nlev, t, lfil = 3, 1e-4, 20
    singles = [V.vbarms_factor(A, nlev, t, lfil, precision=precision) for A in As]
    batch = V.vbarms_factor_batched(As, nlev, t, lfil, precision=precision)
    rng = np.random.default_rng(5)
    xs = [torch.from_numpy(rng.standard_normal(m.n)).cuda() for m, _ in mats]
    ys = [torch.zeros_like(x) for x in xs]
    V.vbarms_apply_batched(batch, xs, ys)
    for k, ((m, _), P1, Pb, x) in enumerate(zip(mats, singles, batch, xs)):
        y1 = _apply(V, P1, x).cpu().numpy()
        yb = _apply(V, Pb, x).cpu().numpy()
        assert np.array_equal(y1, yb), f"matrix {k}: batched apply differs from the single factorization"
        assert np.array_equal(y1, ys[k].cpu().numpy()), f"matrix {k}: vbarms_apply_batched differs"
    # FGMRES with a batch handle: the same iterations as with the single one
    for (m, _), A, P1, Pb in zip(mats, As, singles, batch):
        b = torch.from_numpy(synth.ones_rhs(m)).cuda()
        x1 = torch.zeros_like(b)
        xb = torch.zeros_like(b)
        it1, rr1, st1 = V.fgmres_solve(A, P1, b, x1, rtol=1e-8)
        itb, rrb, stb = V.fgmres_solve(A, Pb, b, xb, rtol=1e-8)
        assert st1 == stb == V.VB_OK
        assert it1 == itb and rr1 == rrb
        assert torch.equal(x1, xb)


def test_batched_fp64_matches_oracle_per_matrix():
    """Each matrix of an FP64 batch: the oracle's factorization of that matrix
    applied to x equals the batch handle's application (to rounding of the
    solve, which the single-matrix parity tests pin bit for bit)."""
    V = vb()
    mats = _mats()[:2]
    As = [gpu_compress(m, tau) for m, tau in mats]
    batch = V.vbarms_factor_batched(As, 2, 1e-3, 10, precision="fp64")
    for (m, tau), A, Pb in zip(mats, As, batch):
        c = oracle.compress(m.n, m.rowptr, m.colind, m.val, tau)
        Po = oracle.Prec(c.A, 2, 1e-3, 10)
        P1 = V.vbarms_factor(A, 2, 1e-3, 10, precision="fp64")
        compare_factor(P1, Po)
        x = np.random.default_rng(9).standard_normal(m.n)
        yo = np.empty(m.n)
        yo[c.perm] = Po.apply(x[c.perm])
        yb = _apply(V, Pb, torch.from_numpy(x).cuda()).cpu().numpy()
        assert np.linalg.norm(yb - yo) <= 1e-12 * np.linalg.norm(yo)


def test_batched_parameter_groups_and_edges():
    V = vb()
    mats = _mats()[:3]
    As = [gpu_compress(m, tau) for m, tau in mats]
    # two groups: lfil differs for the middle matrix
    batch = V.vbarms_factor_batched(As, [2, 2, 2], [1e-3, 1e-3, 1e-3], [10, 5, 10])
    for (m, _), A, Pb, lf in zip(mats, As, batch, [10, 5, 10]):
        P1 = V.vbarms_factor(A, 2, 1e-3, lf)
        x = torch.from_numpy(np.random.default_rng(3).standard_normal(m.n)).cuda()
        assert torch.equal(_apply(V, P1, x), _apply(V, Pb, x))
    assert V.vbarms_factor_batched([], 2, 1e-3, 10) == []
    with pytest.raises(V.VbarmsError) as e:
        V.vbarms_factor_batched(As[:1], -1, 1e-3, 10)
    assert e.value.status == V.VB_EINVAL
    # the fixed-scratch apply serves whole factorizations only
    x = torch.zeros(mats[0][0].n, dtype=torch.float64, device="cuda")
    with pytest.raises(V.VbarmsError) as e:
        V.vbarms_apply_static(batch[0], x, torch.zeros_like(x))
    assert e.value.status == V.VB_EINVAL
