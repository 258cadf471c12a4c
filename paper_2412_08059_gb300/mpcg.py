"""Python binding of libmpcg (include/mpcg.h): ctypes argument marshalling only.

Device arrays are torch CUDA tensors; their raw pointers and the current CUDA
stream are handed to the C ABI.  Every step of the solver runs in the CUDA
kernels of libmpcg.so; this module holds no numerical code and no fallback:
if the library is missing it raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmpcg.so")
_lock = threading.Lock()
_lib = None

OK = 0
WARN_EPS1_NOT_REACHED = 1
WARN_TRUE_RESID_RESTARTED = 2
ERR_INVALID_ARG = -1
ERR_WORKSPACE = -2
ERR_BREAKDOWN = -3
ERR_NAN = -4
ERR_NOT_CONVERGED = -5
ERR_TIMEOUT = -6
ERR_CUDA = -7
ERR_CANCELLED = -8
PHASE_NEW, PHASE_STAGE1, PHASE_STAGE2, PHASE_STAGE2_RUN, PHASE_DONE = 0, 1, 2, 3, 4
KNN_MAX_SAMPLE = 65536
KNN_MAX_K = 64


class CsrDesc(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int32), ("row_ptr", C.c_void_p),
                ("col", C.c_void_p), ("val", C.c_void_p)]


class Features(C.Structure):
    _fields_ = [("n", C.c_double), ("m", C.c_double), ("pdiam", C.c_double), ("v", C.c_double),
                ("k0_done", C.c_int32), ("status", C.c_int32)]


class SampleDesc(C.Structure):
    _fields_ = [("feat", C.c_void_p), ("cls", C.c_void_p), ("count", C.c_int32),
                ("fmin", C.c_double * 4), ("fmax", C.c_double * 4)]


class Options(C.Structure):
    _fields_ = [("eps1", C.c_double), ("eps2", C.c_double), ("k0", C.c_int32),
                ("knn_k", C.c_int32), ("weighted", C.c_int32), ("tol_relative", C.c_int32),
                ("max_it_fp32", C.c_int32), ("max_it_fp64", C.c_int32),
                ("max_true_restarts", C.c_int32), ("feat_mask", C.c_uint32),
                ("fp64_only", C.c_int32), ("grid_blocks", C.c_int32), ("timeout_ms", C.c_int32),
                ("stage1_only", C.c_int32), ("team_rows", C.c_int32),
                ("serve_split", C.c_int32), ("bfs_starts", C.c_int32),
                ("precond", C.c_int32), ("stop_true_residual", C.c_int32),
                ("cancel", C.c_void_p), ("acc32", C.c_int32),
                ("spmv_variant", C.c_int32), ("team_rows_sys", C.c_void_p)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("n1", C.c_int32), ("n2", C.c_int32), ("cls", C.c_int32),
                ("k0_done", C.c_int32), ("restarts", C.c_int32), ("eps1", C.c_double),
                ("true_rel_resid", C.c_double), ("pdiam", C.c_double), ("v", C.c_double),
                ("res_fp32", C.c_double), ("res_fp64", C.c_double),
                ("t_start_ns", C.c_uint64), ("t_features_ns", C.c_uint64),
                ("t_fp32_ns", C.c_uint64), ("t_fp64_ns", C.c_uint64), ("t_end_ns", C.c_uint64),
                ("t_prep_ns", C.c_uint64), ("t_stage2_ns", C.c_uint64), ("spmv_cols", C.c_int32),
                ("team_blocks", C.c_int32)]

    def as_dict(self) -> dict:
        """Fields plus phase durations from the device clock marks: ms_prep (set-up),
        ms_features (set-up end to eps1 known; overlapped with stage 1 in
        Algorithm II), ms_fp32 (set-up end to end of stage 1, features included),
        ms_fp64 (stage 2), ms_total."""
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["ms_prep"] = (self.t_prep_ns - self.t_start_ns) / 1e6
        d["ms_features"] = (self.t_features_ns - self.t_prep_ns) / 1e6
        d["ms_fp32"] = (self.t_fp32_ns - self.t_prep_ns) / 1e6
        d["ms_fp64"] = (self.t_fp64_ns - self.t_fp32_ns) / 1e6
        d["ms_total"] = (self.t_end_ns - self.t_start_ns) / 1e6
        return d


SYMBOLS = ("mpcg_options_default", "mpcg_status_string", "mpcg_workspace_bytes", "mpcg_features",
           "mpcg_choose_eps1", "mpcg_solve", "mpcg_batch_workspace_bytes", "mpcg_solve_batch",
           "mpcg_spmv", "mpcg_bfs", "mpcg_pseudo_diameter", "mpcg_solve_static",
           "mpcg_server_workspace_bytes", "mpcg_server_create", "mpcg_server_destroy",
           "mpcg_server_admit", "mpcg_batch_step", "mpcg_batch_step_launches", "mpcg_server_retire", "mpcg_batch_tune", "mpcg_batch_plan",
           "mpcg_knn_batch")


def load(path: str = LIB_PATH):
    """Load libmpcg.so and declare the C signatures.  Raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"libmpcg.so is not built ({path}); run "
                               "paper_2412_08059_gb300.build.build() first")
        L = C.CDLL(path)
        P, I32, SZ = C.c_void_p, C.c_int32, C.c_size_t
        L.mpcg_options_default.restype = Options
        L.mpcg_options_default.argtypes = []
        L.mpcg_status_string.restype = C.c_char_p
        L.mpcg_status_string.argtypes = [I32]
        L.mpcg_workspace_bytes.restype = SZ
        L.mpcg_workspace_bytes.argtypes = [I32, I32, C.POINTER(Options)]
        L.mpcg_features.restype = I32
        L.mpcg_features.argtypes = [C.POINTER(CsrDesc), P, C.POINTER(Options), P, SZ, P, P]
        L.mpcg_choose_eps1.restype = I32
        L.mpcg_choose_eps1.argtypes = [P, C.POINTER(SampleDesc), C.POINTER(Options), P, P, P]
        L.mpcg_knn_batch.restype = I32
        L.mpcg_knn_batch.argtypes = [C.POINTER(SampleDesc), P, I32, C.POINTER(Options), P, P, P]
        L.mpcg_solve.restype = I32
        L.mpcg_solve.argtypes = [C.POINTER(CsrDesc), P, P, C.POINTER(SampleDesc),
                                 C.POINTER(Options), P, SZ, P, P]
        L.mpcg_batch_workspace_bytes.restype = SZ
        L.mpcg_batch_workspace_bytes.argtypes = [I32, P, P, C.POINTER(Options)]
        L.mpcg_solve_batch.restype = I32
        L.mpcg_solve_batch.argtypes = [I32, P, P, P, C.POINTER(SampleDesc), C.POINTER(Options),
                                       P, SZ, P, P]
        L.mpcg_spmv.restype = I32
        L.mpcg_spmv.argtypes = [C.POINTER(CsrDesc), I32, P, P, P, SZ, P]
        L.mpcg_bfs.restype = I32
        L.mpcg_bfs.argtypes = [C.POINTER(CsrDesc), I32, P, P, SZ, P]
        L.mpcg_pseudo_diameter.restype = I32
        L.mpcg_pseudo_diameter.argtypes = [C.POINTER(CsrDesc), P, P, SZ, P]
        L.mpcg_batch_plan.restype = I32
        L.mpcg_batch_plan.argtypes = [I32, P, P, C.POINTER(Options), I32, P]
        L.mpcg_batch_tune.restype = I32
        L.mpcg_batch_tune.argtypes = [I32, P, P, P, C.POINTER(SampleDesc), C.POINTER(Options),
                                      P, SZ, P, P, C.POINTER(I32), P, P]
        L.mpcg_server_workspace_bytes.restype = SZ
        L.mpcg_server_workspace_bytes.argtypes = [I32, SZ]
        L.mpcg_server_create.restype = I32
        L.mpcg_server_create.argtypes = [P, SZ, I32, C.POINTER(SampleDesc), C.POINTER(Options),
                                         C.POINTER(C.c_void_p)]
        L.mpcg_server_destroy.restype = None
        L.mpcg_server_destroy.argtypes = [P]
        L.mpcg_server_admit.restype = I32
        L.mpcg_server_admit.argtypes = [P, C.POINTER(CsrDesc), P, P, C.c_double, P,
                                        C.POINTER(I32)]
        L.mpcg_batch_step.restype = I32
        L.mpcg_batch_step.argtypes = [P, I32, P, P]
        L.mpcg_batch_step_launches.restype = I32
        L.mpcg_batch_step_launches.argtypes = [P]
        L.mpcg_server_retire.restype = I32
        L.mpcg_server_retire.argtypes = [P, I32]
        L.mpcg_solve_static.restype = I32
        L.mpcg_solve_static.argtypes = [C.POINTER(CsrDesc), P, P, C.POINTER(SampleDesc),
                                        C.POINTER(Options), P, P]
        _lib = L
        return L


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def status_string(st: int) -> str:
    return load().mpcg_status_string(st).decode()


def options(**kw) -> Options:
    """Default options with the given fields set.  team_rows_sys takes a
    sequence of per-system rows per block (kept alive by the returned object)."""
    o = load().mpcg_options_default()
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        if k == "team_rows_sys" and v is not None and not isinstance(v, int):
            arr = np.ascontiguousarray(v, dtype=np.int32)
            o._team_rows_sys = arr
            v = arr.ctypes.data
        setattr(o, k, v)
    return o


def _check(st: int, what: str):
    if st != OK:
        raise RuntimeError(f"{what}: {status_string(st)} ({st})")


class DeviceCSR:
    """A CSR matrix held in torch CUDA tensors (int32 row_ptr/col, float64 val)."""

    def __init__(self, row_ptr, col, val, device="cuda"):
        self.row_ptr = torch.as_tensor(row_ptr, dtype=torch.int32, device=device).contiguous()
        self.col = torch.as_tensor(col, dtype=torch.int32, device=device).contiguous()
        self.val = torch.as_tensor(val, dtype=torch.float64, device=device).contiguous()
        self.n = self.row_ptr.numel() - 1
        self.nnz = self.col.numel()
        self.desc = CsrDesc(self.n, self.nnz, self.row_ptr.data_ptr(), self.col.data_ptr(),
                            self.val.data_ptr())

    @classmethod
    def from_host(cls, A, device="cuda"):
        return cls(torch.from_numpy(A.row_ptr), torch.from_numpy(A.col), torch.from_numpy(A.val),
                   device)


class DeviceSample:
    """A labelled kNN sample in device memory (raw features [count, 4], int8 classes)."""

    def __init__(self, feat, cls, fmin=None, fmax=None, device="cuda"):
        f = torch.as_tensor(feat, dtype=torch.float64).reshape(-1, 4)
        self.feat = f.to(device).contiguous()
        self.cls = torch.as_tensor(cls, dtype=torch.int8).to(device).contiguous()
        fmin = f.min(dim=0).values.tolist() if fmin is None else list(map(float, fmin))
        fmax = f.max(dim=0).values.tolist() if fmax is None else list(map(float, fmax))
        self.desc = SampleDesc(self.feat.data_ptr(), self.cls.data_ptr(), f.shape[0],
                               (C.c_double * 4)(*fmin), (C.c_double * 4)(*fmax))


def workspace_bytes(n: int, nnz: int, opts: Options | None = None) -> int:
    """mpcg_workspace_bytes; the options matter only with precond (16 n more bytes)."""
    return int(load().mpcg_workspace_bytes(n, nnz, C.byref(opts) if opts is not None else None))


def workspace(n: int, nnz: int, device="cuda", opts: Options | None = None) -> torch.Tensor:
    """A device byte buffer large enough for (n, nnz) and the options, base
    256-byte aligned."""
    nb = workspace_bytes(n, nnz, opts)
    if nb == 0:
        raise ValueError("invalid sizes")
    return torch.empty(nb, dtype=torch.uint8, device=device)


def _ws_for(A: DeviceCSR, ws, opts: Options | None = None):
    return workspace(A.n, A.nnz, A.val.device, opts) if ws is None else ws


def result_buffer(count: int = 1, device="cuda") -> torch.Tensor:
    return torch.zeros(count * C.sizeof(Result), dtype=torch.uint8, device=device)


def read_results(buf: torch.Tensor, count: int = 1) -> list[dict]:
    raw = bytes(buf.cpu().numpy())
    sz = C.sizeof(Result)
    return [Result.from_buffer_copy(raw[i * sz:(i + 1) * sz]).as_dict() for i in range(count)]


def solve_async(A: DeviceCSR, b: torch.Tensor, x: torch.Tensor, opts: Options, ws: torch.Tensor,
                res: torch.Tensor, sample: DeviceSample | None = None, stream=None) -> None:
    """Enqueue mpcg_solve on the stream; no host synchronisation."""
    st = load().mpcg_solve(C.byref(A.desc), _ptr(b), _ptr(x),
                           C.byref(sample.desc) if sample is not None else None, C.byref(opts),
                           _ptr(ws), ws.numel(), _ptr(res), _stream(stream))
    _check(st, "mpcg_solve")


STATIC_WS_BYTES = 64 << 20  # MPCG_STATIC_WS_BYTES


def solve_static_async(A: DeviceCSR, b: torch.Tensor, x: torch.Tensor, opts: Options,
                       res: torch.Tensor, sample: DeviceSample | None = None, stream=None) -> int:
    """Enqueue mpcg_solve_static (the library's fixed scratch array, no
    workspace, no allocation); returns the call's status without raising."""
    return int(load().mpcg_solve_static(C.byref(A.desc), _ptr(b), _ptr(x),
                                        C.byref(sample.desc) if sample is not None else None,
                                        C.byref(opts), _ptr(res), _stream(stream)))


def solve(A: DeviceCSR, b: torch.Tensor, sample: DeviceSample | None = None, ws=None, **kw):
    """mpcg_solve; returns (x, result dict) after synchronising."""
    x = torch.empty(A.n, dtype=torch.float64, device=b.device)
    res = result_buffer(1, b.device)
    o = options(**kw)
    solve_async(A, b, x, o, _ws_for(A, ws, o), res, sample)
    torch.cuda.synchronize(b.device)
    return x, read_results(res)[0]


def features(A: DeviceCSR, b: torch.Tensor, ws=None, **kw) -> dict:
    out = torch.zeros(C.sizeof(Features), dtype=torch.uint8, device=b.device)
    o = options(**kw)
    w = _ws_for(A, ws, o)
    st = load().mpcg_features(C.byref(A.desc), _ptr(b), C.byref(o), _ptr(w),
                              w.numel(), _ptr(out), _stream())
    _check(st, "mpcg_features")
    f = Features.from_buffer_copy(bytes(out.cpu().numpy()))
    return {k: getattr(f, k) for k, _ in f._fields_}


def choose_eps1(feat4, sample: DeviceSample, **kw):
    """kNN on a feature vector (n, m, l~, v) given as 4 numbers; returns (eps1, t)."""
    f = Features(*[float(v) for v in feat4], 0, 0)
    fdev = torch.frombuffer(bytearray(bytes(f)), dtype=torch.uint8).to("cuda")
    eps = torch.zeros(1, dtype=torch.float64, device="cuda")
    cls = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = load().mpcg_choose_eps1(_ptr(fdev), C.byref(sample.desc), C.byref(options(**kw)),
                                 _ptr(eps), _ptr(cls), _stream())
    _check(st, "mpcg_choose_eps1")
    return float(eps.item()), int(cls.item())


def knn_batch(chi, sample: DeviceSample, neighbours: bool = False, stream=None, **kw):
    """mpcg_knn_batch: the kNN vote for every row of chi ([count, 4] raw
    features).  Returns the classes (int32 tensor, -1 for an invalid query)
    and, with neighbours, the [count, knn_k] neighbour indices (-1 padded)."""
    o = options(**kw)
    q = torch.as_tensor(chi, dtype=torch.float64).reshape(-1, 4).to(sample.feat.device).contiguous()
    count = q.shape[0]
    cls = torch.empty(count, dtype=torch.int32, device=q.device)
    nbr = (torch.empty((count, o.knn_k), dtype=torch.int32, device=q.device)
           if neighbours else None)
    st = load().mpcg_knn_batch(C.byref(sample.desc), _ptr(q), count, C.byref(o), _ptr(cls),
                               _ptr(nbr), _stream(stream))
    _check(st, "mpcg_knn_batch")
    return (cls, nbr) if neighbours else cls


def spmv(A: DeviceCSR, x: torch.Tensor, ws=None) -> torch.Tensor:
    fp32 = x.dtype == torch.float32
    y = torch.empty_like(x)
    w = _ws_for(A, ws)
    st = load().mpcg_spmv(C.byref(A.desc), int(fp32), _ptr(x), _ptr(y), _ptr(w), w.numel(),
                          _stream())
    _check(st, "mpcg_spmv")
    return y


def bfs(A: DeviceCSR, src: int, ws=None) -> torch.Tensor:
    dist = torch.empty(A.n, dtype=torch.int32, device=A.val.device)
    w = _ws_for(A, ws)
    st = load().mpcg_bfs(C.byref(A.desc), int(src), _ptr(dist), _ptr(w), w.numel(), _stream())
    _check(st, "mpcg_bfs")
    return dist


def pseudo_diameter(A: DeviceCSR, ws=None) -> tuple[int, int]:
    out = torch.zeros(2, dtype=torch.int32, device=A.val.device)
    w = _ws_for(A, ws)
    st = load().mpcg_pseudo_diameter(C.byref(A.desc), _ptr(out), _ptr(w), w.numel(), _stream())
    _check(st, "mpcg_pseudo_diameter")
    o = out.cpu().tolist()
    return o[0], o[1]


def solve_batch_async(mats: list[DeviceCSR], bs: list, xs: list, opts: Options,
                      ws: torch.Tensor, res: torch.Tensor, sample: DeviceSample | None = None,
                      stream=None) -> None:
    n = len(mats)
    descs = (CsrDesc * n)(*[m.desc for m in mats])
    bp = (C.c_void_p * n)(*[b.data_ptr() for b in bs])
    xp = (C.c_void_p * n)(*[x.data_ptr() for x in xs])
    st = load().mpcg_solve_batch(n, descs, bp, xp,
                                 C.byref(sample.desc) if sample is not None else None,
                                 C.byref(opts), _ptr(ws), ws.numel(), _ptr(res), _stream(stream))
    _check(st, "mpcg_solve_batch")


TUNE_CANDIDATES = 4
TUNE_RUNS = TUNE_CANDIDATES + 1


def batch_tune(mats: list[DeviceCSR], bs: list, xs: list, opts: Options, ws: torch.Tensor,
               res: torch.Tensor, sample: DeviceSample | None = None, stream=None,
               per_system: bool = False):
    """mpcg_batch_tune: (fastest uniform team_rows, milliseconds per timed call
    [4 candidates, then the per-system call or -1]), plus with per_system the
    per-system rows per block (numpy int32).  Synchronises."""
    n = len(mats)
    descs = (CsrDesc * n)(*[m.desc for m in mats])
    bp = (C.c_void_p * n)(*[b.data_ptr() for b in bs])
    xp = (C.c_void_p * n)(*[x.data_ptr() for x in xs])
    best = C.c_int32(0)
    ms = (C.c_float * TUNE_RUNS)()
    rows = np.zeros(n, dtype=np.int32)
    st = load().mpcg_batch_tune(n, descs, bp, xp,
                                C.byref(sample.desc) if sample is not None else None,
                                C.byref(opts), _ptr(ws), ws.numel(), _ptr(res), _stream(stream),
                                C.byref(best), rows.ctypes.data if per_system else None, ms)
    _check(st, "mpcg_batch_tune")
    if per_system:
        return best.value, list(ms), rows
    return best.value, list(ms)


def batch_plan(ns, nnzs, opts: Options | None = None, grid_blocks: int = 0) -> list[int]:
    """mpcg_batch_plan: the team size (blocks) the batch planner gives each
    system (host only when grid_blocks > 0)."""
    k = len(ns)
    nv = (C.c_int32 * k)(*[int(v) for v in ns])
    mv = (C.c_int32 * k)(*[int(v) for v in nnzs])
    out = (C.c_int32 * k)()
    o = opts if opts is not None else options()
    _check(load().mpcg_batch_plan(k, nv, mv, C.byref(o), int(grid_blocks), out),
           "mpcg_batch_plan")
    return list(out)


def batch_workspace_bytes(mats: list[DeviceCSR]) -> int:
    n = len(mats)
    ns = (C.c_int32 * n)(*[m.n for m in mats])
    nz = (C.c_int32 * n)(*[m.nnz for m in mats])
    return int(load().mpcg_batch_workspace_bytes(n, ns, nz, None))


class Server:
    """Continuous batching over a slot table (mpcg_server_* and mpcg_batch_step).
    The caller keeps each admitted system's CSR, b, x and result record alive
    until it retires the slot."""

    def __init__(self, max_slots: int, pool_bytes: int, opts: Options,
                 sample: DeviceSample | None = None, device="cuda"):
        L = load()
        nb = int(L.mpcg_server_workspace_bytes(max_slots, pool_bytes))
        if nb == 0:
            raise ValueError("invalid server size")
        self.ws = torch.empty(nb, dtype=torch.uint8, device=device)
        self.max_slots = max_slots
        self.sample = sample
        h = C.c_void_p()
        st = L.mpcg_server_create(_ptr(self.ws), nb, max_slots,
                                  C.byref(sample.desc) if sample is not None else None,
                                  C.byref(opts), C.byref(h))
        _check(st, "mpcg_server_create")
        self.h = h
        self.phase = torch.full((max_slots,), -1, dtype=torch.int32).pin_memory()

    def admit(self, A: DeviceCSR, b: torch.Tensor, x: torch.Tensor, eps2: float,
              res: torch.Tensor):
        """Slot number, or None when no slot or pool block is free."""
        slot = C.c_int32(-1)
        st = load().mpcg_server_admit(self.h, C.byref(A.desc), _ptr(b), _ptr(x), float(eps2),
                                      _ptr(res), C.byref(slot))
        if st == ERR_WORKSPACE:
            return None
        _check(st, "mpcg_server_admit")
        return slot.value

    def step(self, max_iters: int, stream=None) -> None:
        """Enqueue one step; self.phase holds the slot phases after a synchronise."""
        st = load().mpcg_batch_step(self.h, int(max_iters), C.c_void_p(self.phase.data_ptr()),
                                    _stream(stream))
        _check(st, "mpcg_batch_step")

    def launches_per_step(self) -> int:
        """Kernel launches of one step while a system is admitted."""
        return int(load().mpcg_batch_step_launches(self.h))

    def retire(self, slot: int) -> None:
        _check(load().mpcg_server_retire(self.h, int(slot)), "mpcg_server_retire")

    def close(self) -> None:
        if self.h is not None:
            load().mpcg_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
