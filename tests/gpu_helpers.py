"""Shared helpers of the GPU parity tests: run the CUDA library through its C
ABI and the CPU oracle on the same seeded inputs and compare."""
import numpy as np
import pytest

import oracle
from paper_1508_02219_gb300 import synth

torch = pytest.importorskip("torch")

# FP64 factors: the tolerance the method's statement fixes for no-drop and
# forced-mask factors (relative Frobenius error per component).
FP64_REL = 1e-11


def cuda_ok() -> bool:
    return torch.cuda.is_available()


def vb():
    from paper_1508_02219_gb300 import build, vbarms
    build.build()
    return vbarms


def gpu_compress(m: synth.CSR, tau: float, on_device=False):
    V = vb()
    if on_device:
        rp = torch.from_numpy(m.rowptr).cuda()
        ci = torch.from_numpy(m.colind).cuda()
        vv = torch.from_numpy(m.val).cuda()
        A = V.vbarms_compress(m.n, rp, ci, vv, tau)
        torch.cuda.synchronize()
        return A
    return V.vbarms_compress(m.n, m.rowptr, m.colind, m.val, tau)


def as_dict(M: oracle.VBMat) -> dict:
    return dict(rsz=M.rsz, csz=M.csz, bptr=M.bptr, bcol=M.bcol, voff=M.voff, val=M.val)


def rel_fro(a: np.ndarray, b: np.ndarray) -> float:
    nb = np.linalg.norm(b)
    d = np.linalg.norm(a - b)
    return d / nb if nb > 0 else d


def compare_vb(g: dict, o: dict, what: str, rel: float = 0.0):
    """Structure identical; values bit-identical (rel = 0) or within rel."""
    for k in ("rsz", "csz", "bptr", "bcol", "voff"):
        assert np.array_equal(np.asarray(g[k]), np.asarray(o[k])), f"{what}: {k} differs"
    if rel == 0.0:
        if not np.array_equal(g["val"], o["val"]):
            bad = np.nonzero(g["val"] != o["val"])[0]
            raise AssertionError(f"{what}: {len(bad)} values differ, first at {bad[:5]}, "
                                 f"max abs diff {np.abs(g['val'] - o['val']).max():.3e}, "
                                 f"rel fro {rel_fro(g['val'], o['val']):.3e}")
    else:
        r = rel_fro(g["val"], o["val"])
        assert r <= rel, f"{what}: relative Frobenius error {r:.3e} > {rel:.1e}"


def compare_factor(P, Po: oracle.Prec, rel: float = 0.0, mats=("A", "D", "F", "E", "C", "W", "G", "S")):
    assert P.levels == Po.levels, f"levels {P.levels} vs {Po.levels}"
    for lev in range(Po.levels):
        assert np.array_equal(P.vector(lev, "pI"), Po.vec(lev, "pI")), f"level {lev}: ordering P_I differs"
        for v in ("r", "c", "w"):
            assert np.array_equal(P.vector(lev, v), Po.vec(lev, v)), f"level {lev}: {v} differs"
        assert np.array_equal(P.vector(lev, "piv"), Po.vec(lev, "piv")), f"level {lev}: pivots differ"
        for w in mats:
            compare_vb(P.export(lev, w), as_dict(Po.mat(lev, w)), f"level {lev} {w}", rel)
    last = Po.levels
    for v in ("r", "c"):
        assert np.array_equal(P.vector(last, v), Po.vec(last, v)), f"last level: {v} differs"
    assert np.array_equal(P.vector(last, "piv"), Po.vec(last, "piv")), "last level: pivots differ"
    for w in ("A", "D", "L", "U"):
        compare_vb(P.export(last, w), as_dict(Po.mat(last, w)), f"last level {w}", rel)
