"""FP64 CPU oracle of VBARMS (arXiv 1508.02219) -- TEST INFRASTRUCTURE ONLY.

A plain single-threaded C++ restatement of the paper's method
(``vbarms_oracle.cpp``), loaded through ctypes.  Only the test suite,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import
this package; the CUDA library never does and shares no code with it.

Matrices come back as :class:`VBMat` (variable block CSR, blocks row-major).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vbarms_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ESINGULAR, ENOCONV = 0, 1, 4, 6


def build(force: bool = False) -> str:
    """Compile the oracle with strict IEEE evaluation (no contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            vp, i64, i32, d = C.c_void_p, C.c_int64, C.c_int, C.c_double
            P = C.POINTER
            sig = {
                "or_last_status": (i32, []),
                "or_compress": (vp, [i64, vp, vp, vp, d]),
                "or_graph_compress": (vp, [i64, vp, vp, vp, d]),
                "or_compress_two_pass": (vp, [i64, vp, vp, vp, d]),
                "or_cmp_free": (None, [vp]),
                "or_cmp_nblk": (i64, [vp]),
                "or_cmp_perm": (None, [vp, vp, vp]),
                "or_cmp_quality": (None, [vp, P(d), P(d)]),
                "or_cmp_matrix": (vp, [vp]),
                "or_vb_create": (vp, [i64, i64, vp, vp, vp, vp, vp, vp]),
                "or_vb_free": (None, [vp]),
                "or_vb_dims": (None, [vp, P(i64), P(i64), P(i64), P(i64)]),
                "or_vb_export": (None, [vp, vp, vp, vp, vp, vp, vp]),
                "or_vb_spmv": (None, [vp, vp, vp]),
                "or_scale": (None, [vp, vp, vp]),
                "or_is_order": (i64, [vp, d, vp, vp]),
                "or_gepp": (i32, [vp, i32, vp]),
                "or_dropped": (i32, [vp, i32, i32, d]),
                "or_factor": (vp, [vp, i32, d, i32, d, i32]),
                "or_factor_fixed": (vp, [vp, i32, d, i32, d, i32, vp]),
                "or_factor_groups": (vp, [vp, i32, d, i32, d, i32, i32, i32]),
                "or_prec_gptr": (i64, [vp, i32, vp]),
                "or_prec_free": (None, [vp]),
                "or_prec_levels": (i32, [vp]),
                "or_prec_fill": (d, [vp]),
                "or_prec_nd": (i64, [vp, i32]),
                "or_prec_mat": (vp, [vp, i32, i32]),
                "or_prec_vec": (i64, [vp, i32, i32, vp, vp]),
                "or_apply": (None, [vp, vp, vp]),
                "or_fgmres": (i32, [vp, vp, vp, vp, d, i32, i32, P(i32), P(d)]),
                "or_dd_build": (vp, [vp, i32, i32, i32, i32, d, i32, d, i32]),
                "or_dd_free": (None, [vp]),
                "or_dd_part": (i64, [vp, vp]),
                "or_dd_rows": (i64, [vp, i32, vp]),
                "or_dd_local": (vp, [vp, i32]),
                "or_dd_local_prec": (vp, [vp, i32]),
                "or_dd_apply": (None, [vp, vp, vp]),
                "or_dd_fgmres": (i32, [vp, vp, vp, vp, d, i32, i32, P(i32), P(d)]),
                "or_dds_build": (vp, [vp, i32, i32, i32, d, i32, d, i32]),
                "or_dds_free": (None, [vp]),
                "or_dds_iface": (i64, [vp, vp, vp]),
                "or_dds_rows": (i64, [vp, i32, vp, P(i64)]),
                "or_dds_local": (vp, [vp, i32]),
                "or_dds_local_prec": (vp, [vp, i32]),
                "or_dds_coupling": (vp, [vp]),
                "or_dds_ng": (i64, [vp]),
                "or_dds_sinv": (None, [vp, vp, vp]),
                "or_dds_apply": (None, [vp, vp, vp]),
                "or_dds_fgmres": (i32, [vp, vp, vp, vp, d, i32, i32, P(i32), P(d)]),
                "or_prec_last_fixed": (i64, [vp, vp]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class OracleError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"oracle {what} failed with status {status}")
        self.status = status


@dataclass
class VBMat:
    """Variable block CSR: block (I, bcol[b]) is val[voff[b]:voff[b+1]]
    reshaped to (rsz[I], csz[bcol[b]]), row-major."""
    rsz: np.ndarray
    csz: np.ndarray
    bptr: np.ndarray
    bcol: np.ndarray
    voff: np.ndarray
    val: np.ndarray

    @property
    def nbr(self):
        return len(self.rsz)

    @property
    def nbc(self):
        return len(self.csz)

    @property
    def nnzb(self):
        return len(self.bcol)

    def block(self, b: int) -> np.ndarray:
        r = np.searchsorted(self.bptr, b, side="right") - 1
        return self.val[self.voff[b]:self.voff[b + 1]].reshape(self.rsz[r], self.csz[self.bcol[b]])

    def dense(self) -> np.ndarray:
        ro = np.concatenate([[0], np.cumsum(self.rsz)]).astype(np.int64)
        co = np.concatenate([[0], np.cumsum(self.csz)]).astype(np.int64)
        a = np.zeros((ro[-1], co[-1]))
        for I in range(self.nbr):
            for b in range(self.bptr[I], self.bptr[I + 1]):
                J = self.bcol[b]
                a[ro[I]:ro[I + 1], co[J]:co[J + 1]] = \
                    self.val[self.voff[b]:self.voff[b + 1]].reshape(self.rsz[I], self.csz[J])
        return a


def _export(h) -> VBMat:
    L = lib()
    nbr, nbc, nnzb, nval = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
    L.or_vb_dims(h, C.byref(nbr), C.byref(nbc), C.byref(nnzb), C.byref(nval))
    m = VBMat(np.zeros(nbr.value, np.int32), np.zeros(nbc.value, np.int32),
              np.zeros(nbr.value + 1, np.int64), np.zeros(nnzb.value, np.int32),
              np.zeros(nnzb.value + 1, np.int64), np.zeros(nval.value, np.float64))
    L.or_vb_export(h, _p(m.rsz), _p(m.csz), _p(m.bptr), _p(m.bcol), _p(m.voff), _p(m.val))
    return m


class _VBHandle:
    """An oracle-owned copy of a VBMat (for feeding identical input)."""

    def __init__(self, m: VBMat):
        self._keep = [np.ascontiguousarray(m.rsz, np.int32), np.ascontiguousarray(m.csz, np.int32),
                      np.ascontiguousarray(m.bptr, np.int64), np.ascontiguousarray(m.bcol, np.int32),
                      np.ascontiguousarray(m.voff, np.int64), np.ascontiguousarray(m.val, np.float64)]
        k = self._keep
        self.h = lib().or_vb_create(len(k[0]), len(k[1]), *[_p(a) for a in k])

    def __del__(self):
        if getattr(self, "h", None):
            lib().or_vb_free(self.h)
            self.h = None


@dataclass
class Compressed:
    perm: np.ndarray
    bsz: np.ndarray
    A: VBMat
    av_bd: float
    av_bs: float
    handle: object = None


def compress(n, rowptr, colind, val, tau) -> Compressed:
    """Step 1: angle-based compression (Section 2.1) and P_B A P_B^T (Eq. 3)."""
    return _compressed(lib().or_compress, "compress", n, rowptr, colind, val, tau)


def compress_two_pass(n, rowptr, colind, val, tau) -> Compressed:
    """The two-pass variant of the angle method (Section 2.1): identical
    patterns grouped first, then unassigned rows added to a group by angle."""
    return _compressed(lib().or_compress_two_pass, "compress_two_pass", n, rowptr, colind, val, tau)


def graph_compress(n, rowptr, colind, val, mu) -> Compressed:
    """Graph-based compression with minimum block density mu (Section 2.2,
    Alg. 1) and P_B A P_B^T."""
    return _compressed(lib().or_graph_compress, "graph_compress", n, rowptr, colind, val, mu)


def _compressed(fn, what, n, rowptr, colind, val, param) -> Compressed:
    L = lib()
    rowptr = np.ascontiguousarray(rowptr, np.int64)
    colind = np.ascontiguousarray(colind, np.int32)
    val = np.ascontiguousarray(val, np.float64)
    h = fn(int(n), _p(rowptr), _p(colind), _p(val), float(param))
    if not h:
        raise OracleError(L.or_last_status(), what)
    p = L.or_cmp_nblk(h)
    perm = np.zeros(int(n), np.int32)
    bsz = np.zeros(p, np.int32)
    L.or_cmp_perm(h, _p(perm), _p(bsz))
    bd, bs = C.c_double(), C.c_double()
    L.or_cmp_quality(h, C.byref(bd), C.byref(bs))
    A = _export(L.or_cmp_matrix(h))
    out = Compressed(perm, bsz, A, bd.value, bs.value, _CmpHandle(h))
    return out


class _CmpHandle:
    def __init__(self, h):
        self.h = h

    def __del__(self):
        if self.h:
            lib().or_cmp_free(self.h)
            self.h = None


def scale(m: VBMat):
    """Step 2 (two-sided max-abs scaling) on a copy; returns (scaled, r, c)."""
    h = _VBHandle(m)
    r = np.zeros(int(m.rsz.sum()))
    c = np.zeros(int(m.csz.sum()))
    lib().or_scale(h.h, _p(r), _p(c))
    return _export(h.h), r, c


def is_order(m: VBMat, ddtol: float = 0.0):
    """Step 3: weighted greedy block independent set; returns (pI, nD, w)."""
    h = _VBHandle(m)
    pI = np.zeros(m.nbr, np.int32)
    w = np.zeros(m.nbr)
    nD = lib().or_is_order(h.h, float(ddtol), _p(pI), _p(w))
    return pI, int(nD), w


def gepp(a: np.ndarray):
    """GEPP of one dense block; returns (lu, piv) or raises on a zero pivot."""
    a = np.ascontiguousarray(a, np.float64).copy()
    piv = np.zeros(a.shape[0], np.int32)
    st = lib().or_gepp(_p(a), a.shape[0], _p(piv))
    if st:
        raise OracleError(st, "gepp")
    return a, piv


def dropped(b: np.ndarray, t: float) -> bool:
    b = np.ascontiguousarray(b, np.float64)
    return bool(lib().or_dropped(_p(b), b.shape[0], b.shape[1], float(t)))


def spmv(m: VBMat, x: np.ndarray) -> np.ndarray:
    h = _VBHandle(m)
    x = np.ascontiguousarray(x, np.float64)
    y = np.zeros(int(m.rsz.sum()))
    lib().or_vb_spmv(h.h, _p(x), _p(y))
    return y


MAT = dict(A=0, D=1, F=2, E=3, C=4, W=5, G=6, S=7, L=8, U=9, Lg=10, Ug=11)
DVEC = dict(r=0, c=1, w=2)
IVEC = dict(pI=3, piv=4)


class Prec:
    """Multilevel factorization (Steps 2-4 repeated, Eq. 7-8, last-level ILUT)."""

    def __init__(self, A: VBMat, nlev: int, droptol: float, lfil: int, ddtol: float = 0.0,
                 schur_drop_all: bool = False, fixed=None, gs: int = 1, grouped: bool = False):
        """fixed: optional flags per block row; flagged rows never enter an
        independent set (Section 5, Schur-complement preconditioner).  gs:
        supernodes per independent group (grouped: the grouped code even for
        gs = 1)."""
        self._A = _VBHandle(A)
        self.n = int(A.rsz.sum())
        L = lib()
        if gs > 1 or grouped:
            assert fixed is None
            self.h = L.or_factor_groups(self._A.h, int(nlev), float(droptol), int(lfil), float(ddtol),
                                        int(bool(schur_drop_all)), int(gs), int(bool(grouped)))
        elif fixed is None:
            self.h = L.or_factor(self._A.h, int(nlev), float(droptol), int(lfil), float(ddtol),
                                 int(bool(schur_drop_all)))
        else:
            self._fixed = np.ascontiguousarray(fixed, np.int32)
            assert len(self._fixed) == A.nbr
            self.h = L.or_factor_fixed(self._A.h, int(nlev), float(droptol), int(lfil), float(ddtol),
                                       int(bool(schur_drop_all)), _p(self._fixed))
        if not self.h:
            raise OracleError(L.or_last_status(), "factor")
        self.levels = L.or_prec_levels(self.h)

    def __del__(self):
        if getattr(self, "h", None):
            lib().or_prec_free(self.h)
            self.h = None

    def nD(self, lev: int) -> int:
        return int(lib().or_prec_nd(self.h, lev))

    def mat(self, lev: int, which: str) -> VBMat:
        h = lib().or_prec_mat(self.h, lev, MAT[which])
        if not h:
            raise KeyError(which)
        return _export(h)

    def vec(self, lev: int, which: str) -> np.ndarray:
        L = lib()
        if which in DVEC:
            n = L.or_prec_vec(self.h, lev, DVEC[which], None, None)
            out = np.zeros(max(n, 0))
            L.or_prec_vec(self.h, lev, DVEC[which], _p(out), None)
        else:
            n = L.or_prec_vec(self.h, lev, IVEC[which], None, None)
            out = np.zeros(max(n, 0), np.int32)
            L.or_prec_vec(self.h, lev, IVEC[which], None, _p(out))
        if n < 0:
            raise KeyError(which)
        return out

    def gptr(self, lev: int) -> np.ndarray:
        """Group boundaries over the D rows of a grouped level."""
        L = lib()
        out = np.zeros(L.or_prec_gptr(self.h, lev, None), np.int64)
        L.or_prec_gptr(self.h, lev, _p(out))
        return out

    def last_fixed(self) -> np.ndarray:
        """Rows of the last level kept out of every independent set (empty:
        the factorization has none)."""
        L = lib()
        out = np.zeros(L.or_prec_last_fixed(self.h, None), np.int32)
        L.or_prec_last_fixed(self.h, _p(out))
        return out

    @property
    def fill(self) -> float:
        return float(lib().or_prec_fill(self.h))

    def apply(self, b: np.ndarray) -> np.ndarray:
        """x = M^{-1} b (Alg. 2) in the block-permuted numbering."""
        b = np.ascontiguousarray(b, np.float64)
        x = np.zeros(self.n)
        lib().or_apply(self.h, _p(b), _p(x))
        return x


def block_diag(mats) -> VBMat:
    """The block-diagonal concatenation of square-partitioned VBMats."""
    rsz, bcol, val = [], [], []
    bptr, voff = [0], [0]
    r0 = 0
    for M in mats:
        rsz.append(M.rsz)
        bptr.extend((M.bptr[1:] + bptr[-1]).tolist())
        bcol.append(M.bcol + r0)
        voff.extend((M.voff[1:] + voff[-1]).tolist())
        val.append(M.val)
        r0 += M.nbr
    cat = lambda xs, t: np.concatenate(xs).astype(t) if xs else np.zeros(0, t)
    rs = cat(rsz, np.int32)
    return VBMat(rs, rs.copy(), np.asarray(bptr, np.int64), cat(bcol, np.int32), np.asarray(voff, np.int64),
                 cat(val, np.float64))


class _LocalPrec(Prec):
    """A local factorization owned by a DD (not freed on its own)."""

    def __init__(self, h, n, owner):
        self.h, self.n, self._owner = h, n, owner
        self.levels = lib().or_prec_levels(h)

    def __del__(self):
        pass


class DD:
    """Section 5 global preconditioners with VBARMS local solvers: block
    Jacobi (overlap 0), additive Schwarz, restricted additive Schwarz."""

    def __init__(self, A: VBMat, nparts: int, overlap: int, restricted: bool, nlev: int, droptol: float,
                 lfil: int, ddtol: float = 0.0, schur_drop_all: bool = False):
        self._A = _VBHandle(A)
        self.n = int(A.rsz.sum())
        self.nparts = int(nparts)
        L = lib()
        self.h = L.or_dd_build(self._A.h, int(nparts), int(overlap), int(bool(restricted)), int(nlev),
                               float(droptol), int(lfil), float(ddtol), int(bool(schur_drop_all)))
        if not self.h:
            raise OracleError(L.or_last_status(), "dd_build")

    def __del__(self):
        if getattr(self, "h", None):
            lib().or_dd_free(self.h)
            self.h = None

    def part(self) -> np.ndarray:
        L = lib()
        out = np.zeros(L.or_dd_part(self.h, None), np.int32)
        L.or_dd_part(self.h, _p(out))
        return out

    def rows(self, i: int) -> np.ndarray:
        """W_i^delta: the block rows of subdomain i with its overlap."""
        L = lib()
        out = np.zeros(L.or_dd_rows(self.h, i, None), np.int32)
        L.or_dd_rows(self.h, i, _p(out))
        return out

    def local(self, i: int) -> VBMat:
        return _export(lib().or_dd_local(self.h, i))

    def local_prec(self, i: int) -> Prec:
        m = self.local(i)
        return _LocalPrec(lib().or_dd_local_prec(self.h, i), int(m.rsz.sum()), self)

    def apply(self, b: np.ndarray) -> np.ndarray:
        b = np.ascontiguousarray(b, np.float64)
        x = np.zeros(self.n)
        lib().or_dd_apply(self.h, _p(b), _p(x))
        return x


class DDSchur:
    """Section 5 Schur-complement global preconditioner (eq. gschur and
    eq. loc_var_schur) with VBARMS local factorizations whose interface rows
    are kept to the last level."""

    def __init__(self, A: VBMat, nparts: int, msteps: int, nlev: int, droptol: float, lfil: int,
                 ddtol: float = 0.0, schur_drop_all: bool = False):
        self._A = _VBHandle(A)
        self.n = int(A.rsz.sum())
        self.nparts = int(nparts)
        L = lib()
        self.h = L.or_dds_build(self._A.h, int(nparts), int(msteps), int(nlev), float(droptol), int(lfil),
                                float(ddtol), int(bool(schur_drop_all)))
        if not self.h:
            raise OracleError(L.or_last_status(), "dds_build")
        self.ng = int(L.or_dds_ng(self.h))

    def __del__(self):
        if getattr(self, "h", None):
            lib().or_dds_free(self.h)
            self.h = None

    def part(self):
        """(subdomain, interface flag) of every block row of A."""
        L = lib()
        p = L.or_dds_iface(self.h, None, None)
        part, iface = np.zeros(p, np.int32), np.zeros(p, np.int32)
        L.or_dds_iface(self.h, _p(part), _p(iface))
        return part, iface

    def rows(self, i: int):
        """Subdomain i's block rows of A (interior, then interface) and the
        interior count."""
        L = lib()
        ni = C.c_int64()
        out = np.zeros(L.or_dds_rows(self.h, i, None, C.byref(ni)), np.int32)
        L.or_dds_rows(self.h, i, _p(out), C.byref(ni))
        return out, int(ni.value)

    def local(self, i: int) -> VBMat:
        return _export(lib().or_dds_local(self.h, i))

    def local_prec(self, i: int) -> Prec:
        m = self.local(i)
        return _LocalPrec(lib().or_dds_local_prec(self.h, i), int(m.rsz.sum()), self)

    def coupling(self) -> VBMat:
        """The E_ij blocks on the global interface numbering."""
        return _export(lib().or_dds_coupling(self.h))

    def sinv(self, v: np.ndarray) -> np.ndarray:
        v = np.ascontiguousarray(v, np.float64)
        out = np.zeros(self.ng)
        lib().or_dds_sinv(self.h, _p(v), _p(out))
        return out

    def apply(self, b: np.ndarray) -> np.ndarray:
        b = np.ascontiguousarray(b, np.float64)
        x = np.zeros(self.n)
        lib().or_dds_apply(self.h, _p(b), _p(x))
        return x


def fgmres(A: VBMat, prec, b, x0=None, rtol=1e-8, restart=50, maxit=1000):
    """Right-preconditioned FGMRES(m) on the block-permuted system; prec is a
    Prec, a DD, a DDSchur or None."""
    h = _VBHandle(A)
    b = np.ascontiguousarray(b, np.float64)
    x = np.zeros_like(b) if x0 is None else np.ascontiguousarray(x0, np.float64).copy()
    it, rr = C.c_int(), C.c_double()
    f = (lib().or_dd_fgmres if isinstance(prec, DD) else
         lib().or_dds_fgmres if isinstance(prec, DDSchur) else lib().or_fgmres)
    st = f(h.h, prec.h if prec is not None else None, _p(b), _p(x), float(rtol),
           int(restart), int(maxit), C.byref(it), C.byref(rr))
    return x, it.value, rr.value, st
