"""CPU oracle for restarted mixed-precision CG (Prolubnikov, arXiv 2412.08059).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import this package.  It shares no code with
the CUDA library of ``paper_2412_08059_gb300``; neither imports the other.

The arithmetic lives in ``oracle.c`` (plain C, one thread, built with
``-ffp-contract=off``); this module compiles it with gcc and marshals numpy
arrays through ctypes.  ``metrics.py`` holds the paper's cost model.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK = 0
WARN_EPS1_NOT_REACHED = 1
WARN_TRUE_RESID_RESTARTED = 2
ERR_INVALID_ARG = -1
ERR_BREAKDOWN = -3
ERR_NAN = -4
ERR_NOT_CONVERGED = -5


def build(force: bool = False) -> str:
    """Compile liboracle.so next to oracle.c (gcc, -O2 -ffp-contract=off)."""
    src = os.path.join(_HERE, "oracle.c")
    hdr = os.path.join(_HERE, "oracle.h")
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class Csr(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int32),
                ("row_ptr", C.c_void_p), ("col", C.c_void_p), ("val", C.c_void_p)]


class Sample(C.Structure):
    _fields_ = [("feat", C.c_void_p), ("cls", C.c_void_p), ("count", C.c_int32),
                ("fmin", C.c_double * 4), ("fmax", C.c_double * 4)]


class Opts(C.Structure):
    _fields_ = [("eps1", C.c_double), ("eps2", C.c_double), ("k0", C.c_int32),
                ("knn_k", C.c_int32), ("weighted", C.c_int32), ("tol_relative", C.c_int32),
                ("max_it_fp32", C.c_int32), ("max_it_fp64", C.c_int32),
                ("max_true_restarts", C.c_int32), ("feat_mask", C.c_uint32),
                ("bfs_starts", C.c_int32), ("precond", C.c_int32),
                ("stop_true_residual", C.c_int32), ("acc32", C.c_int32)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("n1", C.c_int32), ("n2", C.c_int32),
                ("cls", C.c_int32), ("k0_done", C.c_int32), ("eps1", C.c_double),
                ("true_rel_resid", C.c_double), ("pdiam", C.c_double), ("v", C.c_double),
                ("feat", C.c_double * 4), ("restarts", C.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "feat"} | {
            "feat": list(self.feat)}


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_SO)
            P = C.c_void_p
            L.orc_spmv64.argtypes = [C.POINTER(Csr), P, P]
            L.orc_spmv32.argtypes = [C.c_int32, P, P, P, P, P]
            L.orc_dot64.argtypes = [C.c_int32, P, P]
            L.orc_dot64.restype = C.c_double
            L.orc_dot32.argtypes = [C.c_int32, P, P]
            L.orc_dot32.restype = C.c_double
            L.orc_dot32_f.argtypes = [C.c_int32, P, P]
            L.orc_dot32_f.restype = C.c_double
            L.orc_cg64.argtypes = [C.POINTER(Csr), P, P, C.c_double, C.c_int32, C.c_int32,
                                   C.c_int32, C.c_int32, C.POINTER(C.c_int32), P]
            L.orc_cg64.restype = C.c_int32
            L.orc_cg32.argtypes = [C.POINTER(Csr), P, P, C.c_double, C.c_int32, C.c_int32,
                                   C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_int32), P]
            L.orc_cg32.restype = C.c_int32
            L.orc_bfs.argtypes = [C.POINTER(Csr), C.c_int32, P]
            L.orc_bfs.restype = C.c_int32
            L.orc_pseudo_diameter.argtypes = [C.POINTER(Csr), C.POINTER(C.c_int32)]
            L.orc_pseudo_diameter.restype = C.c_int32
            L.orc_pseudo_diameter_rep.argtypes = [C.POINTER(Csr), C.c_int32, C.POINTER(C.c_int32)]
            L.orc_pseudo_diameter_rep.restype = C.c_int32
            L.orc_components.argtypes = [C.POINTER(Csr), P]
            L.orc_components.restype = C.c_int32
            L.orc_knn.argtypes = [P, C.POINTER(Sample), C.c_int32, C.c_int32, C.c_uint32, P, P]
            L.orc_knn.restype = C.c_int32
            L.orc_opts_default.argtypes = []
            L.orc_opts_default.restype = Opts
            L.orc_solve.argtypes = [C.POINTER(Csr), P, P, C.POINTER(Sample), C.POINTER(Opts),
                                    C.POINTER(Result)]
            L.orc_solve.restype = C.c_int32
            L.orc_features.argtypes = [C.POINTER(Csr), P, C.POINTER(Opts), P,
                                       C.POINTER(C.c_int32)]
            L.orc_features.restype = C.c_int32
            L.orc_true_rel_resid.argtypes = [C.POINTER(Csr), P, P]
            L.orc_true_rel_resid.restype = C.c_double
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class _CsrHolder:
    """Keeps contiguous numpy copies alive while the C struct points at them."""

    def __init__(self, row_ptr, col, val):
        self.row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.val = np.ascontiguousarray(val, dtype=np.float64)
        n = self.row_ptr.size - 1
        self.s = Csr(n, self.col.size, _ptr(self.row_ptr).value, _ptr(self.col).value,
                     _ptr(self.val).value)

    @property
    def n(self):
        return self.s.n


def csr(A) -> _CsrHolder:
    """Accepts an object with row_ptr/col/val attributes or a (row_ptr, col, val) tuple."""
    if isinstance(A, _CsrHolder):
        return A
    if isinstance(A, tuple):
        return _CsrHolder(*A)
    return _CsrHolder(A.row_ptr, A.col, A.val)


class _SampleHolder:
    def __init__(self, feat, cls, fmin=None, fmax=None):
        self.feat = np.ascontiguousarray(feat, dtype=np.float64).reshape(-1, 4)
        self.cls = np.ascontiguousarray(cls, dtype=np.int8)
        fmin = self.feat.min(axis=0) if fmin is None else np.asarray(fmin, dtype=np.float64)
        fmax = self.feat.max(axis=0) if fmax is None else np.asarray(fmax, dtype=np.float64)
        self.s = Sample(_ptr(self.feat).value, _ptr(self.cls).value, self.feat.shape[0],
                        (C.c_double * 4)(*fmin), (C.c_double * 4)(*fmax))


def sample(feat, cls, fmin=None, fmax=None) -> _SampleHolder:
    """Labelled kNN sample; min/max default to the sample's own (Sec. 11.1)."""
    return _SampleHolder(feat, cls, fmin, fmax)


def opts(**kw) -> Opts:
    o = lib().orc_opts_default()
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def spmv64(A, x):
    h = csr(A)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(h.n, dtype=np.float64)
    lib().orc_spmv64(C.byref(h.s), _ptr(x), _ptr(y))
    return y


def spmv32(A, x):
    h = csr(A)
    v32 = h.val.astype(np.float32)
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.empty(h.n, dtype=np.float32)
    lib().orc_spmv32(h.n, _ptr(h.row_ptr), _ptr(h.col), _ptr(v32), _ptr(x), _ptr(y))
    return y


def dot32(a, b, acc32=0):
    """Inner product of two float vectors: summed in double, or with acc32=1
    summed in float in index order."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    b = np.ascontiguousarray(b, dtype=np.float32)
    f = lib().orc_dot32_f if acc32 else lib().orc_dot32
    return f(a.size, _ptr(a), _ptr(b))


def dot64(a, b):
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    return lib().orc_dot64(a.size, _ptr(a), _ptr(b))


def cg64(A, b, eps, x0=None, tol_relative=1, max_it=None, history=False, precond=0,
         true_res=0):
    """Plain FP64 CG (Sec. 3), or with precond=1 the Jacobi PCG of Sec. 5;
    true_res=1 stops on ||b - A x|| (the loop test as printed) instead of
    the recursive r.  Returns (x, iters, status[, res_hist])."""
    h = csr(A)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(h.n) if x0 is None else np.array(x0, dtype=np.float64)
    max_it = 10 * h.n if max_it is None else int(max_it)
    it = C.c_int32(0)
    hist = np.full(max_it + 1, np.nan) if history else None
    st = lib().orc_cg64(C.byref(h.s), _ptr(b), _ptr(x), eps, tol_relative, max_it,
                        int(precond), int(true_res), C.byref(it),
                        _ptr(hist) if history else None)
    out = (x, it.value, st)
    return out + (hist[: it.value + 1],) if history else out


def cg32(A, b, eps, tol_relative=1, max_it=None, history=False, precond=0, true_res=0,
         acc32=0):
    """Plain FP32 CG on float32(A), float32(b) from 0 (precond=1: Jacobi PCG;
    true_res=1: stop on ||b~ - A~ x~||; acc32=1: inner products summed in
    float).  Returns (x32, iters, status[, hist])."""
    h = csr(A)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(h.n, dtype=np.float32)
    max_it = 10 * h.n if max_it is None else int(max_it)
    it = C.c_int32(0)
    hist = np.full(max_it + 1, np.nan) if history else None
    st = lib().orc_cg32(C.byref(h.s), _ptr(b), _ptr(x), eps, tol_relative, max_it,
                        int(precond), int(true_res), int(acc32), C.byref(it),
                        _ptr(hist) if history else None)
    out = (x, it.value, st)
    return out + (hist[: it.value + 1],) if history else out


def bfs(A, src):
    h = csr(A)
    dist = np.empty(h.n, dtype=np.int32)
    reached = lib().orc_bfs(C.byref(h.s), int(src), _ptr(dist))
    return dist, reached


def pseudo_diameter(A, return_t=False, starts=1):
    """2BFS pseudo-diameter (Sec. 6); starts > 1: the repeated 2BFS of the
    remark there (the largest value over `starts` runs)."""
    h = csr(A)
    t = C.c_int32(-1)
    ell = lib().orc_pseudo_diameter_rep(C.byref(h.s), int(starts), C.byref(t))
    return (ell, t.value) if return_t else ell


def components(A):
    h = csr(A)
    lab = np.empty(h.n, dtype=np.int32)
    cnt = lib().orc_components(C.byref(h.s), _ptr(lab))
    return lab, cnt


def knn(chi, S, k=5, weighted=1, feat_mask=0xF, details=False):
    S = S if isinstance(S, _SampleHolder) else sample(*S)
    chi = np.ascontiguousarray(chi, dtype=np.float64)
    kk = min(k, S.feat.shape[0])
    nbr = np.full(max(kk, 1), -1, dtype=np.int32)
    score = np.zeros(16)
    t = lib().orc_knn(_ptr(chi), C.byref(S.s), k, weighted, feat_mask, _ptr(nbr), _ptr(score))
    return (t, nbr[:kk], score) if details else t


def features(A, b, **kw):
    h = csr(A)
    b = np.ascontiguousarray(b, dtype=np.float64)
    o = opts(**kw)
    feat = np.zeros(4)
    k0d = C.c_int32(0)
    st = lib().orc_features(C.byref(h.s), _ptr(b), C.byref(o), _ptr(feat), C.byref(k0d))
    return feat, k0d.value, st


def solve(A, b, S=None, **kw):
    """Algorithm I (eps1 > 0) or II (eps1 <= 0).  Returns (x, result dict)."""
    h = csr(A)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(h.n)
    o = opts(**kw)
    res = Result()
    Sh = None if S is None else (S if isinstance(S, _SampleHolder) else sample(*S))
    lib().orc_solve(C.byref(h.s), _ptr(b), _ptr(x), C.byref(Sh.s) if Sh else None,
                    C.byref(o), C.byref(res))
    return x, res.as_dict()


def true_rel_resid(A, b, x):
    h = csr(A)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    return lib().orc_true_rel_resid(C.byref(h.s), _ptr(b), _ptr(x))
