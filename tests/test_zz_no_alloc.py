"""vbarms_apply_static: the preconditioner solve for callers that cannot
allocate device memory when they apply it -- solver loops with a fixed
memory budget that forbid allocator calls once set-up is over, and
applications whose device memory belongs to another runtime's pool.  Its
scratch is a fixed device array inside the library; this file checks it
against vbarms_apply and checks that it allocates nothing.  It is collected
last so that a run stopping at the first failure has run every other test."""
import numpy as np
import pytest

from gpu_helpers import cuda_ok, gpu_compress, rel_fro, torch, vb
from paper_1508_02219_gb300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_static_apply_matches_apply_on_two_calls(precision):
    V = vb()
    m = synth.geometric(3000, 6, seed=21, dominance=1.5, ill_frac=0.003)
    A = gpu_compress(m, 0.8)
    P = V.vbarms_factor(A, 3, 1e-4, 30, precision=precision)
    need = V.vbarms_apply_static_need(P)
    assert 0 < need <= V.apply_static_max_bytes()
    rng = np.random.default_rng(3)
    for call in range(2):  # the array keeps the previous call's contents
        x = torch.from_numpy(rng.standard_normal(m.n)).cuda()
        y_ref = torch.zeros(m.n, dtype=torch.float64, device="cuda")
        y = torch.full((m.n,), np.nan, dtype=torch.float64, device="cuda")
        V.vbarms_apply(P, x, y_ref)
        torch.cuda.synchronize()
        a0 = V.alloc_count()
        V.vbarms_apply_static(P, x, y)
        torch.cuda.synchronize()
        assert V.alloc_count() == a0, f"call {call}: the library allocated device memory"
        assert rel_fro(y.cpu().numpy(), y_ref.cpu().numpy()) <= 1e-12, f"call {call}"


def test_static_apply_rejects_oversized_factorizations():
    V = vb()
    n = 3_000_000  # diagonal matrix: its last-level solve needs > 64 MiB of scratch
    rowptr = np.arange(n + 1, dtype=np.int64)
    colind = np.arange(n, dtype=np.int32)
    val = np.full(n, 2.0)
    A = V.vbarms_compress(n, rowptr, colind, val, 1.0)
    P = V.vbarms_factor(A, 0, 0.0, -1)
    assert V.vbarms_apply_static_need(P) > V.apply_static_max_bytes()
    x = torch.ones(n, dtype=torch.float64, device="cuda")
    y = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(V.VbarmsError) as e:
        V.vbarms_apply_static(P, x, y)
    assert e.value.status == V.VB_EINVAL and "maximum" in str(e.value)
    V.vbarms_apply(P, x, y)
    assert torch.allclose(y, torch.full_like(y, 0.5))
