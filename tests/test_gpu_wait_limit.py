"""Bounded device waits: the last-level block ILUT is a sync-free kernel whose
rows wait for the rows they depend on (Alg. 3 in block form: row i needs the
finished U rows of its L columns).  Every wait carries a time limit
(vbarms_opts.wait_limit); when it runs out the kernel records VB_ETIMEOUT,
raises its abort flag and returns, and the host reports the status.  This
test drives that path with a limit shorter than any dependency takes -- the
kernel returns on its own, nothing faults -- and checks that the device is
still usable: a following factorization with the default limit matches the
oracle bit for bit."""
import pytest

import oracle
from gpu_helpers import compare_factor, cuda_ok, gpu_compress, vb
from paper_1508_02219_gb300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]


def test_wait_limit_runs_out_and_the_device_stays_usable():
    V = vb()
    m = synth.geometric(2000, 4, seed=31)
    A = gpu_compress(m, 0.8)
    with pytest.raises(V.VbarmsError) as e:
        V.vbarms_factor(A, 2, 1e-3, -1, wait_limit=1)  # 1 ns per wait
    assert e.value.status == V.VB_ETIMEOUT, str(e.value)
    P = V.vbarms_factor(A, 2, 1e-3, -1)
    c = oracle.compress(m.n, m.rowptr, m.colind, m.val, 0.8)
    Po = oracle.Prec(c.A, 2, 1e-3, -1)
    compare_factor(P, Po)
