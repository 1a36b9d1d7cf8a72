"""Python binding of the C ABI in ``include/vbarms.h`` (ctypes).

Argument marshalling only: every step of the method runs in the CUDA library
``libvbarms.so``.  Device vectors are passed as torch CUDA tensors (or raw
device addresses); host arrays as numpy arrays.  The names follow the C entry
points: :func:`vbarms_compress`, :func:`vbarms_factor`, :func:`vbarms_apply`,
:func:`fgmres_solve`.

There is no CPU fallback: if the library is missing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

VB_OK, VB_EINVAL, VB_ENOMEM, VB_ECUDA, VB_ESINGULAR, VB_ETIMEOUT, VB_ENOCONV, VB_EINTERNAL = range(8)
VB_FP64, VB_FP32_MIXED = 0, 1
STATUS_NAMES = {0: "VB_OK", 1: "VB_EINVAL", 2: "VB_ENOMEM", 3: "VB_ECUDA", 4: "VB_ESINGULAR",
                5: "VB_ETIMEOUT", 6: "VB_ENOCONV", 7: "VB_EINTERNAL"}
MAT = dict(A=0, D=1, F=2, E=3, C=4, W=5, G=6, S=7, L=8, U=9, Lg=10, Ug=11)
VEC_D = dict(r=0, c=1, w=2)
VEC_I = dict(pI=3, piv=4, ptag=5, gptr=6)
PHASES = ["scale", "ordering", "gather", "pivot_lu", "W", "G", "schur", "last_ilut"]


class VbarmsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("fp64_pivot_cond", C.c_double), ("ddtol", C.c_double),
                ("wait_limit", C.c_uint64), ("schur_drop_all", C.c_int), ("keep_factors", C.c_int),
                ("group_size", C.c_int)]


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libvbarms.so (built in-tree by ``build()``)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_build.LIB):
                raise ImportError(f"{_build.LIB} is missing: run __graft_entry__.build() "
                                  "(the CUDA library has no CPU fallback)")
            L = C.CDLL(_build.LIB)
            vp, i64, i32, d = C.c_void_p, C.c_int64, C.c_int, C.c_double
            P = C.POINTER
            sig = {
                "vbarms_opts_default": (None, [P(Opts)]),
                "vbarms_last_error": (C.c_char_p, []),
                "vbarms_compress": (i32, [i64, vp, vp, vp, i32, d, vp, P(vp)]),
                "vbarms_compress_graph": (i32, [i64, vp, vp, vp, i32, d, vp, P(vp)]),
                "vbarms_compress_two_pass": (i32, [i64, vp, vp, vp, i32, d, vp, P(vp)]),
                "vbarms_vbsr_from_blocks": (i32, [i64, vp, vp, vp, vp, vp, vp, P(vp)]),
                "vbarms_vbsr_query": (i32, [vp, P(i64), P(i64), P(i64), P(i64), P(d), P(d)]),
                "vbarms_vbsr_export": (i32, [vp, vp, vp, vp, vp, vp, vp]),
                "vbarms_factor": (i32, [vp, i32, d, i32, P(Opts), P(vp)]),
                "vbarms_apply": (i32, [vp, vp, vp]),
                "vbarms_factor_batched": (i32, [i32, vp, vp, vp, vp, P(Opts), vp]),
                "vbarms_apply_batched": (i32, [i32, vp, vp, vp]),
                "vbarms_dd_factor": (i32, [vp, i32, i32, i32, i32, d, i32, P(Opts), P(vp)]),
                "vbarms_dd_layout": (i32, [vp, P(i32), P(i32), P(i32), P(i64), vp, vp, vp]),
                "vbarms_dd_schur_factor": (i32, [vp, i32, i32, i32, d, i32, P(Opts), P(vp)]),
                "vbarms_dd_schur_layout": (i32, [vp, P(i32), P(i32), P(i64), P(i64), vp, vp, vp, vp]),
                "fgmres_solve": (i32, [vp, vp, vp, vp, d, i32, i32, P(i32), P(d)]),
                "vbarms_prec_stats": (i32, [vp, P(i32), P(d), vp]),
                "vbarms_prec_export": (i32, [vp, i32, i32, P(i64), P(i64), P(i64), P(i64), vp, vp, vp, vp, vp,
                                             vp]),
                "vbarms_prec_vector": (i32, [vp, i32, i32, vp, vp, P(i64)]),
                "vbarms_prec_kernel_stats": (i32, [vp, i32, P(i32), P(d), P(d), P(d)]),
                "vbarms_launch_count": (C.c_uint64, []),
                "vbarms_apply_static": (i32, [vp, vp, vp]),
                "vbarms_apply_static_max_bytes": (C.c_uint64, []),
                "vbarms_apply_static_need": (i32, [vp, P(C.c_uint64)]),
                "vbarms_alloc_count": (C.c_uint64, []),
                "vbarms_prec_ilut_geometry": (i32, [vp, P(i32), P(i32), P(i32), P(i32), P(d)]),
                "vbarms_prec_pivot_tiles": (i32, [vp, i32, vp, vp, P(i32)]),
                "vbarms_prec_ilut_chain": (i32, [vp, P(i64)]),
                "vbarms_vbsr_destroy": (None, [vp]),
                "vbarms_prec_destroy": (None, [vp]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(st: int):
    if st != VB_OK:
        raise VbarmsError(st, lib().vbarms_last_error().decode())


def _hp(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _dp(x) -> int:
    """Device address of a torch tensor or an int."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class VBSR:
    """Handle of a VBCSR matrix P_B A P_B^T (with P_B)."""

    def __init__(self, h):
        self.h = h

    def __del__(self):
        if getattr(self, "h", None):
            lib().vbarms_vbsr_destroy(self.h)
            self.h = None

    def query(self) -> dict:
        n, nblk, nnzb, nval = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
        bd, bs = C.c_double(), C.c_double()
        _check(lib().vbarms_vbsr_query(self.h, C.byref(n), C.byref(nblk), C.byref(nnzb), C.byref(nval),
                                       C.byref(bd), C.byref(bs)))
        return dict(n=n.value, nblk=nblk.value, nnzb=nnzb.value, nval=nval.value, av_bd=bd.value, av_bs=bs.value)

    def export(self) -> dict:
        q = self.query()
        perm = np.zeros(q["n"], np.int32)
        bsz = np.zeros(q["nblk"], np.int32)
        bptr = np.zeros(q["nblk"] + 1, np.int64)
        bcol = np.zeros(q["nnzb"], np.int32)
        voff = np.zeros(q["nnzb"] + 1, np.int64)
        val = np.zeros(q["nval"], np.float64)
        _check(lib().vbarms_vbsr_export(self.h, _hp(perm), _hp(bsz), _hp(bptr), _hp(bcol), _hp(voff), _hp(val)))
        return dict(perm=perm, bsz=bsz, bptr=bptr, bcol=bcol, voff=voff, val=val)


def vbarms_compress(n, rowptr, colind, val, tau, stream=None) -> VBSR:
    """Step 1 (angle compression).  Host numpy arrays or device torch tensors."""
    h = C.c_void_p()
    if isinstance(rowptr, np.ndarray):
        rp = np.ascontiguousarray(rowptr, np.int64)
        ci = np.ascontiguousarray(colind, np.int32)
        vv = np.ascontiguousarray(val, np.float64)
        st = lib().vbarms_compress(int(n), _hp(rp), _hp(ci), _hp(vv), 0, float(tau), _stream(stream), C.byref(h))
    else:
        st = lib().vbarms_compress(int(n), _dp(rowptr), _dp(colind), _dp(val), 1, float(tau), _stream(stream),
                                   C.byref(h))
    _check(st)
    return VBSR(h.value)


def vbarms_compress_graph(n, rowptr, colind, val, mu, stream=None) -> VBSR:
    """Graph-based compression (Section 2.2, Alg. 1) with minimum block
    density mu.  Host numpy arrays or device torch tensors."""
    h = C.c_void_p()
    if isinstance(rowptr, np.ndarray):
        rp = np.ascontiguousarray(rowptr, np.int64)
        ci = np.ascontiguousarray(colind, np.int32)
        vv = np.ascontiguousarray(val, np.float64)
        st = lib().vbarms_compress_graph(int(n), _hp(rp), _hp(ci), _hp(vv), 0, float(mu), _stream(stream),
                                         C.byref(h))
    else:
        st = lib().vbarms_compress_graph(int(n), _dp(rowptr), _dp(colind), _dp(val), 1, float(mu),
                                         _stream(stream), C.byref(h))
    _check(st)
    return VBSR(h.value)


def vbarms_compress_two_pass(n, rowptr, colind, val, tau, stream=None) -> VBSR:
    """The two-pass checksum and angle variant of Section 2.1.  Host numpy
    arrays or device torch tensors."""
    h = C.c_void_p()
    if isinstance(rowptr, np.ndarray):
        rp = np.ascontiguousarray(rowptr, np.int64)
        ci = np.ascontiguousarray(colind, np.int32)
        vv = np.ascontiguousarray(val, np.float64)
        st = lib().vbarms_compress_two_pass(int(n), _hp(rp), _hp(ci), _hp(vv), 0, float(tau), _stream(stream),
                                            C.byref(h))
    else:
        st = lib().vbarms_compress_two_pass(int(n), _dp(rowptr), _dp(colind), _dp(val), 1, float(tau),
                                            _stream(stream), C.byref(h))
    _check(st)
    return VBSR(h.value)


def vbarms_vbsr_from_blocks(bsz, bptr, bcol, voff, val, stream=None) -> VBSR:
    bsz = np.ascontiguousarray(bsz, np.int32)
    bptr = np.ascontiguousarray(bptr, np.int64)
    bcol = np.ascontiguousarray(bcol, np.int32)
    voff = np.ascontiguousarray(voff, np.int64)
    val = np.ascontiguousarray(val, np.float64)
    h = C.c_void_p()
    _check(lib().vbarms_vbsr_from_blocks(len(bsz), _hp(bsz), _hp(bptr), _hp(bcol), _hp(voff), _hp(val),
                                         _stream(stream), C.byref(h)))
    return VBSR(h.value)


class Prec:
    """Handle of a multilevel VBARMS factorization."""

    def __init__(self, h, A: VBSR):
        self.h = h
        self.A = A  # keeps the matrix alive (same stream)

    def __del__(self):
        if getattr(self, "h", None):
            lib().vbarms_prec_destroy(self.h)
            self.h = None

    def stats(self) -> dict:
        lv, mr = C.c_int(), C.c_double()
        ph = (C.c_double * 8)()
        _check(lib().vbarms_prec_stats(self.h, C.byref(lv), C.byref(mr), C.cast(ph, C.c_void_p)))
        return dict(levels=lv.value, mem_ratio=mr.value, phase_s=dict(zip(PHASES, list(ph))))

    def kernel_stats(self, kernel: int = 0) -> dict:
        n = C.c_int()
        ms, by, fl = C.c_double(), C.c_double(), C.c_double()
        _check(lib().vbarms_prec_kernel_stats(self.h, kernel, C.byref(n), C.byref(ms), C.byref(by), C.byref(fl)))
        return dict(launches=n.value, ms=ms.value, bytes=by.value, flops=fl.value)

    @property
    def levels(self) -> int:
        return self.stats()["levels"]

    def ilut_chain(self) -> int:
        """Rows on the longest chain of waits of the last-level ILUT."""
        n = C.c_int64()
        _check(lib().vbarms_prec_ilut_chain(self.h, C.byref(n)))
        return n.value

    def pivot_tiles(self, lev: int) -> dict:
        """Blocks per size class of level lev's pivot phase and the mode each
        class ran in (thread or warp per block), and how the modes were chosen."""
        cnt = np.zeros(5, np.int32)
        md = np.zeros(5, np.int32)
        src = C.c_int()
        _check(lib().vbarms_prec_pivot_tiles(self.h, int(lev), _hp(cnt), _hp(md), C.byref(src)))
        return dict(counts=cnt.tolist(), modes=[["thread", "warp"][m] for m in md],
                    source=["default", "timed", "cached"][src.value])

    def ilut_geometry(self) -> dict:
        """The per-warp workspace of the last-level ILUT and how it was chosen."""
        sl, vb_, wps, src = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        ts = C.c_double()
        _check(lib().vbarms_prec_ilut_geometry(self.h, C.byref(sl), C.byref(vb_), C.byref(wps), C.byref(src),
                                               C.byref(ts)))
        return dict(slots=sl.value, value_bytes=vb_.value, warps_per_sm=wps.value,
                    source=["default", "timed", "cached"][src.value], tune_s=ts.value)

    def shape(self, lev: int, which: str) -> dict:
        """Sizes of one exported factor (nbr, nbc, nnzb, nval) without its arrays."""
        nbr, nbc, nnzb, nval = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
        _check(lib().vbarms_prec_export(self.h, lev, MAT[which], C.byref(nbr), C.byref(nbc), C.byref(nnzb),
                                        C.byref(nval), None, None, None, None, None, None))
        return dict(nbr=nbr.value, nbc=nbc.value, nnzb=nnzb.value, nval=nval.value)

    def export(self, lev: int, which: str) -> dict:
        w = MAT[which]
        nbr, nbc, nnzb, nval = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
        _check(lib().vbarms_prec_export(self.h, lev, w, C.byref(nbr), C.byref(nbc), C.byref(nnzb), C.byref(nval),
                                        None, None, None, None, None, None))
        rsz = np.zeros(nbr.value, np.int32)
        csz = np.zeros(nbc.value, np.int32)
        bptr = np.zeros(nbr.value + 1, np.int64)
        bcol = np.zeros(nnzb.value, np.int32)
        voff = np.zeros(nnzb.value + 1, np.int64)
        val = np.zeros(nval.value, np.float64)
        _check(lib().vbarms_prec_export(self.h, lev, w, None, None, None, None, _hp(rsz), _hp(csz), _hp(bptr),
                                        _hp(bcol), _hp(voff), _hp(val)))
        return dict(rsz=rsz, csz=csz, bptr=bptr, bcol=bcol, voff=voff, val=val)

    def vector(self, lev: int, which: str) -> np.ndarray:
        n = C.c_int64()
        w = VEC_D.get(which, VEC_I.get(which))
        _check(lib().vbarms_prec_vector(self.h, lev, w, None, None, C.byref(n)))
        if which in VEC_D:
            out = np.zeros(n.value, np.float64)
            _check(lib().vbarms_prec_vector(self.h, lev, w, _hp(out), None, C.byref(n)))
        else:
            out = np.zeros(n.value, np.int32)
            _check(lib().vbarms_prec_vector(self.h, lev, w, None, _hp(out), C.byref(n)))
        return out


def make_opts(precision="fp64", fp64_pivot_cond=1e4, ddtol=0.0, wait_limit=0, schur_drop_all=False,
              keep_factors=True, group_size=1) -> Opts:
    o = Opts()
    lib().vbarms_opts_default(C.byref(o))
    o.precision = VB_FP64 if precision in ("fp64", VB_FP64) else VB_FP32_MIXED
    o.fp64_pivot_cond = float(fp64_pivot_cond)
    o.ddtol = float(ddtol)
    o.wait_limit = int(wait_limit)
    o.schur_drop_all = int(bool(schur_drop_all))
    o.keep_factors = int(bool(keep_factors))
    o.group_size = int(group_size)
    return o


def vbarms_factor(A: VBSR, nlev: int, droptol: float, lfil: int, precision="fp64", **kw) -> Prec:
    """Steps 2-4 repeated nlev times, then the last-level block ILUT."""
    o = make_opts(precision, **kw)
    h = C.c_void_p()
    _check(lib().vbarms_factor(A.h, int(nlev), float(droptol), int(lfil), C.byref(o), C.byref(h)))
    return Prec(h.value, A)


def vbarms_factor_batched(As, nlev, droptol, lfil, precision="fp64", **kw) -> list:
    """Factor several matrices at once (their block-diagonal union, one
    launch per phase); nlev, droptol, lfil are scalars or per-matrix lists."""
    nm = len(As)
    def per(v, t):
        return [t(x) for x in v] if isinstance(v, (list, tuple, np.ndarray)) else [t(v)] * nm
    nl = np.asarray(per(nlev, int), np.int32)
    dt = np.asarray(per(droptol, float), np.float64)
    lf = np.asarray(per(lfil, int), np.int32)
    hs = (C.c_void_p * max(nm, 1))(*[A.h for A in As])
    out = (C.c_void_p * max(nm, 1))()
    o = make_opts(precision, **kw)
    _check(lib().vbarms_factor_batched(nm, C.cast(hs, C.c_void_p), _hp(nl), _hp(dt), _hp(lf), C.byref(o),
                                       C.cast(out, C.c_void_p)))
    return [Prec(out[m], As[m]) for m in range(nm)]


def vbarms_dd_factor(A: VBSR, nparts: int, overlap: int, restricted: bool, nlev: int, droptol: float, lfil: int,
                     precision="fp64", **kw) -> Prec:
    """Section 5 global preconditioner (block Jacobi / additive Schwarz /
    restricted additive Schwarz) with VBARMS local solvers on every subdomain."""
    o = make_opts(precision, **kw)
    h = C.c_void_p()
    _check(lib().vbarms_dd_factor(A.h, int(nparts), int(overlap), int(bool(restricted)), int(nlev), float(droptol),
                                  int(lfil), C.byref(o), C.byref(h)))
    return Prec(h.value, A)


def dd_layout(M: Prec):
    """(part per block row of A, dstart[nparts + 1], union rows -> block rows of A)."""
    L = lib()
    npart, ov, rs, nu = C.c_int(), C.c_int(), C.c_int(), C.c_int64()
    _check(L.vbarms_dd_layout(M.h, C.byref(npart), C.byref(ov), C.byref(rs), C.byref(nu), None, None, None))
    part = np.zeros(max(M.A.query()["nblk"], 1), np.int32)
    dstart = np.zeros(npart.value + 1, np.int64)
    rows = np.zeros(max(nu.value, 1), np.int32)
    _check(L.vbarms_dd_layout(M.h, None, None, None, None, _hp(part), _hp(dstart), _hp(rows)))
    return part[:M.A.query()["nblk"]], dstart, rows[:nu.value]


def vbarms_dd_schur_factor(A: VBSR, nparts: int, msteps: int, nlev: int, droptol: float, lfil: int,
                           precision="fp64", **kw) -> Prec:
    """Section 5 Schur-complement global preconditioner: VBARMS local
    factorizations with the interface rows kept to the last level, msteps of
    GMRES on the global interface system per application."""
    o = make_opts(precision, **kw)
    h = C.c_void_p()
    _check(lib().vbarms_dd_schur_factor(A.h, int(nparts), int(msteps), int(nlev), float(droptol), int(lfil),
                                        C.byref(o), C.byref(h)))
    return Prec(h.value, A)


def dd_schur_layout(M: Prec) -> dict:
    """Subdomain and interface flag per block row of A, the union's rows (each
    subdomain's interior rows, then its interface rows), interior counts."""
    L = lib()
    npart, ms, ng, ngb = C.c_int(), C.c_int(), C.c_int64(), C.c_int64()
    _check(L.vbarms_dd_schur_layout(M.h, C.byref(npart), C.byref(ms), C.byref(ng), C.byref(ngb), None, None, None,
                                    None))
    p = M.A.query()["nblk"]
    part, iface, rows = (np.zeros(max(p, 1), np.int32) for _ in range(3))
    nint = np.zeros(max(npart.value, 1), np.int64)
    _check(L.vbarms_dd_schur_layout(M.h, None, None, None, None, _hp(part), _hp(iface), _hp(rows), _hp(nint)))
    return dict(nparts=npart.value, msteps=ms.value, ng=ng.value, ngb=ngb.value, part=part[:p], iface=iface[:p],
                rows=rows[:p], nint=nint[:npart.value])


def vbarms_apply_batched(Ms, xs, ys):
    """ys[m] = Ms[m]^{-1} xs[m]; handles of one batched factorization share one
    application."""
    nm = len(Ms)
    hs = (C.c_void_p * max(nm, 1))(*[M.h for M in Ms])
    xp = (C.c_void_p * max(nm, 1))(*[_dp(x) for x in xs])
    yp = (C.c_void_p * max(nm, 1))(*[_dp(y) for y in ys])
    _check(lib().vbarms_apply_batched(nm, C.cast(hs, C.c_void_p), C.cast(xp, C.c_void_p), C.cast(yp, C.c_void_p)))


def vbarms_apply(M: Prec, x, y):
    """y = M^{-1} x (Alg. 2); x, y CUDA float64 tensors in original numbering."""
    _check(lib().vbarms_apply(M.h, _dp(x), _dp(y)))


def vbarms_apply_static(M: Prec, x, y):
    """y = M^{-1} x without any device allocation (fixed library scratch);
    for callers that cannot allocate device memory when they apply."""
    _check(lib().vbarms_apply_static(M.h, _dp(x), _dp(y)))


def apply_static_max_bytes() -> int:
    return int(lib().vbarms_apply_static_max_bytes())


def vbarms_apply_static_need(M: Prec) -> int:
    """Bytes of scratch vbarms_apply_static needs for M (no device work)."""
    b = C.c_uint64()
    _check(lib().vbarms_apply_static_need(M.h, C.byref(b)))
    return int(b.value)


def fgmres_solve(A: VBSR, M: Prec | None, b, x, rtol=1e-8, restart=50, maxit=1000, raise_noconv=False):
    """FGMRES(restart); returns (iters, relres, status).  x is updated in place."""
    it, rr = C.c_int(), C.c_double()
    st = lib().fgmres_solve(A.h, M.h if M is not None else None, _dp(b), _dp(x), float(rtol), int(restart),
                            int(maxit), C.byref(it), C.byref(rr))
    if st not in (VB_OK, VB_ENOCONV) or (raise_noconv and st == VB_ENOCONV):
        _check(st)
    return it.value, rr.value, st


def exported_symbols() -> list[str]:
    """Names of the C ABI functions declared in include/vbarms.h."""
    import re
    hdr = os.path.join(_build.INCLUDE, "vbarms.h")
    txt = open(hdr).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(vbarms_\w+|fgmres_solve)\s*\(", txt)))


def launch_count() -> int:
    """Kernels launched by the library since it was loaded."""
    return int(lib().vbarms_launch_count())


def alloc_count() -> int:
    """Device allocations made by the library since it was loaded."""
    return int(lib().vbarms_alloc_count())
