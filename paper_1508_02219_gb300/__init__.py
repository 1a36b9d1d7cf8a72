"""GB300 (sm_103a) VBARMS: angle-based graph compression and the multilevel
block partial factorization of arXiv 1508.02219, behind a C ABI.

``synth`` builds seeded synthetic inputs; ``vbarms`` is the ctypes binding of
``libvbarms.so`` (loaded on first use, no CPU fallback).
"""

__all__ = ["synth", "vbarms", "build"]


def __getattr__(name):
    if name in ("vbarms", "synth", "build"):
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
