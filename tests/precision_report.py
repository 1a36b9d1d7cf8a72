"""Per-result error of a GPU factorization against the FP64 oracle's.

The two factorizations may order the levels below the first differently (the
mixed factor's level inputs carry FP32 rounding), so blocks are matched by
the supernodes of the compressed matrix they belong to: every level's block
rows are traced back through the orderings P_I to their compressed block row.
For each result the relative Frobenius error is taken over the blocks both
factorizations store; the blocks only one of them stores are counted.
Plain numpy: no kernel, no oracle arithmetic."""
from __future__ import annotations

import numpy as np


def _level_maps(levels: int, nblk0: int, pI_of, nD_of):
    """orig[l][k] = compressed block row of block row k of level l
    (l = levels: the last level)."""
    orig = [np.arange(nblk0, dtype=np.int64)]
    for lev in range(levels):
        pI = np.asarray(pI_of(lev), np.int64)
        orig.append(orig[-1][pI[nD_of(lev):]])
    return orig


def _value_index(voff, sel):
    """Indices into val of the blocks sel (in order), and their sizes."""
    starts = voff[sel]
    sizes = voff[sel + 1] - starts
    total = int(sizes.sum())
    if total == 0:
        return np.zeros(0, np.int64), sizes
    cs = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    return np.repeat(starts - cs, sizes) + np.arange(total, dtype=np.int64), sizes


def compare_blocks(g: dict, o: dict, rows_g, cols_g, rows_o, cols_o) -> dict:
    """g, o: VBCSR dicts (bptr, bcol, voff, val); rows_*/cols_*: compressed
    block row of each block row / block column."""
    big = np.int64(max(int(np.max(cols_g, initial=0)), int(np.max(cols_o, initial=0))) + 1)

    def keys(m, rows, cols):
        br = np.repeat(np.arange(len(m["bptr"]) - 1, dtype=np.int64), np.diff(m["bptr"]))
        return np.asarray(rows, np.int64)[br] * big + np.asarray(cols, np.int64)[np.asarray(m["bcol"], np.int64)]

    kg, ko = keys(g, rows_g, cols_g), keys(o, rows_o, cols_o)
    _, ig, io = np.intersect1d(kg, ko, assume_unique=True, return_indices=True)
    xg, sg = _value_index(np.asarray(g["voff"], np.int64), ig)
    xo, so = _value_index(np.asarray(o["voff"], np.int64), io)
    assert np.array_equal(sg, so), "matched blocks of different sizes"
    vg, vo = np.asarray(g["val"])[xg], np.asarray(o["val"])[xo]
    ref = float(np.linalg.norm(vo))
    err = float(np.linalg.norm(vg - vo))
    # per matched block ||g - o||_F / ||o||_F: its median is the typical
    # error, which a few large blocks (multipliers of ill-conditioned pivot
    # blocks) cannot dominate as they dominate the overall Frobenius ratio
    med = 0.0
    if len(sg):
        starts = np.concatenate([[0], np.cumsum(sg)[:-1]])
        nz = sg > 0
        d2 = np.add.reduceat((vg - vo) ** 2, starts[nz]) if nz.any() else np.zeros(0)
        o2 = np.add.reduceat(vo ** 2, starts[nz]) if nz.any() else np.zeros(0)
        ok = o2 > 0
        if ok.any():
            med = float(np.median(np.sqrt(d2[ok] / o2[ok])))
    return {"rel_fro": err / ref if ref > 0 else err, "block_rel_median": med, "blocks_common": int(len(ig)),
            "blocks_only_gpu": int(len(kg) - len(ig)), "blocks_only_oracle": int(len(ko) - len(ig))}


def factor_errors(P, Po) -> dict:
    """Every level's W, G, S and the last level's L, U of the GPU handle P
    against the oracle Prec Po (both of the same compressed matrix)."""
    nblk0 = P.shape(0, "A")["nbr"]
    og = _level_maps(P.levels, nblk0, lambda l: P.vector(l, "pI"), lambda l: P.shape(l, "D")["nbr"])
    oo = _level_maps(Po.levels, nblk0, lambda l: Po.vec(l, "pI"), Po.nD)
    out = {}
    for lev in range(min(P.levels, Po.levels)):
        pg, po = np.asarray(P.vector(lev, "pI"), np.int64), np.asarray(Po.vec(lev, "pI"), np.int64)
        ndg, ndo = P.shape(lev, "D")["nbr"], Po.nD(lev)
        dg, cg = og[lev][pg[:ndg]], og[lev][pg[ndg:]]
        do, co = oo[lev][po[:ndo]], oo[lev][po[ndo:]]
        same_order = bool(np.array_equal(pg, po))
        out[f"level{lev}"] = {"ordering_identical": same_order}
        for name, (rg, cg_, ro, co_) in {"W": (dg, cg, do, co), "G": (cg, dg, co, do), "S": (cg, cg, co, co)}.items():
            gm = P.export(lev, name)
            om = Po.mat(lev, name)
            od = dict(bptr=om.bptr, bcol=om.bcol, voff=om.voff, val=om.val)
            out[f"level{lev}"][name] = compare_blocks(gm, od, rg, cg_, ro, co_)
    lg, lo = og[P.levels], oo[Po.levels]
    out["last"] = {}
    for name in ("L", "U"):
        gm = P.export(P.levels, name)
        om = Po.mat(Po.levels, name)
        od = dict(bptr=om.bptr, bcol=om.bcol, voff=om.voff, val=om.val)
        out["last"][name] = compare_blocks(gm, od, lg, lg, lo, lo)
    return out


def rel(a, b) -> float:
    nb = float(np.linalg.norm(b))
    d = float(np.linalg.norm(np.asarray(a) - np.asarray(b)))
    return d / nb if nb > 0 else d


def summary(errs: dict, key: str = "rel_fro") -> dict:
    """Flat {result: error} of factor_errors' output (key = rel_fro or
    block_rel_median)."""
    flat = {}
    for k, v in errs.items():
        if isinstance(v, dict):
            for name, r in v.items():
                if isinstance(r, dict) and key in r:
                    flat[f"{k}.{name}"] = r[key]
    return flat
