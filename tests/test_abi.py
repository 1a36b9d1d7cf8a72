"""The C-ABI library loads and exports every symbol include/vbarms.h declares
(no compute call: runs without a GPU)."""
import ctypes
import subprocess

import pytest


def test_library_builds_and_exports_header_symbols():
    from paper_1508_02219_gb300 import build, vbarms
    path = build.build()
    lib = ctypes.CDLL(path)
    syms = vbarms.exported_symbols()
    assert {"vbarms_compress", "vbarms_factor", "vbarms_apply", "fgmres_solve"} <= set(syms)
    for s in syms:
        assert hasattr(lib, s), f"{s} declared in vbarms.h but not exported"
    nm = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    for s in syms:
        assert f" {s}" in nm


def test_opts_default_and_last_error_without_gpu():
    from paper_1508_02219_gb300 import vbarms
    o = vbarms.make_opts()
    assert o.precision == vbarms.VB_FP64 and o.fp64_pivot_cond == 1e4 and o.ddtol == 0.0
    assert isinstance(vbarms.lib().vbarms_last_error(), bytes)


def test_invalid_arguments_rejected_on_host():
    """Argument checks that return before any device work."""
    import numpy as np
    from paper_1508_02219_gb300 import vbarms
    with pytest.raises(vbarms.VbarmsError) as e:
        vbarms.vbarms_compress(3, np.zeros(4, np.int64), np.zeros(0, np.int32), np.zeros(0), 1.5)
    assert e.value.status == vbarms.VB_EINVAL
    with pytest.raises(vbarms.VbarmsError) as e:
        vbarms.vbarms_compress(-1, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0), 1.0)
    assert e.value.status == vbarms.VB_EINVAL
    # NULL handles of the other entry points, rejected before any device work
    import ctypes as C
    L = vbarms.lib()
    h = C.c_void_p()
    o = vbarms.make_opts()
    assert L.vbarms_factor(None, 2, 1e-3, -1, C.byref(o), C.byref(h)) == vbarms.VB_EINVAL
    assert L.vbarms_dd_factor(None, 4, 1, 1, 2, 1e-3, -1, C.byref(o), C.byref(h)) == vbarms.VB_EINVAL
    assert L.vbarms_dd_layout(None, None, None, None, None, None, None, None) == vbarms.VB_EINVAL
    assert L.vbarms_dd_schur_factor(None, 4, 5, 2, 1e-3, -1, C.byref(o), C.byref(h)) == vbarms.VB_EINVAL
    assert L.vbarms_dd_schur_layout(None, None, None, None, None, None, None, None, None) == vbarms.VB_EINVAL
    assert L.vbarms_apply(None, None, None) == vbarms.VB_EINVAL
    assert L.vbarms_factor_batched(-1, None, None, None, None, C.byref(o), None) == vbarms.VB_EINVAL
    assert L.fgmres_solve(None, None, None, None, 1e-8, 50, 1000, None, None) == vbarms.VB_EINVAL
    assert h.value is None
