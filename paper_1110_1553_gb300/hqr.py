"""Thin Python binding of the C ABI in include/hqr.h (argument marshalling only).

Every computation runs in ``libhqr.so`` (host C++ for the elimination lists,
sm_103a CUDA kernels for everything numeric). PyTorch supplies device memory
and streams. There is no fallback: if the library is missing, loading fails
with an error that says how to build it.

Matrices cross the boundary column-major. A torch tensor of shape (M, N) is
passed as is when its storage is already column-major (``A.stride(0) == 1``);
otherwise a column-major copy is made.
"""
import ctypes
import os

import numpy as np

from . import _build

FLAT, BINARY, GREEDY, FIBONACCI = 0, 1, 2, 3
TREES = {"flat": FLAT, "binary": BINARY, "greedy": GREEDY, "fibonacci": FIBONACCI}
TS, TT = 0, 1
FP64, FP32, FP32_BF16X3 = 0, 1, 2

(SUCCESS, ERR_CUDA, ERR_TIMEOUT, ERR_NOMEM, ERR_CAPACITY, ERR_INVALID_LIST, ERR_SINGULAR, ERR_INTERNAL,
 ERR_TOO_LARGE, ERR_BUSY, ERR_BUDGET, ERR_NOCONV) = range(12)

ELIM_DTYPE = np.dtype([("k", np.int32), ("i", np.int32), ("killer", np.int32), ("kind", np.int32),
                       ("level", np.int32), ("step", np.int32)])

EXPORTS = ["hqr_elim_list", "hqr_elim_list_domino", "hqr_validate_list", "hqr_task_graph", "hqr_geqrf", "hqr_refactor", "hqr_refactor_async",
           "hqr_status", "hqr_get_r", "hqr_get_tiles", "hqr_get_t", "hqr_factors_info", "hqr_kernel_ms", "hqr_kernel_times", "hqr_trace", "hqr_apply_q",
           "hqr_gels", "hqr_gels_qr", "hqr_geqrf_r_noalloc", "hqr_ls_plan_create", "hqr_ls_plan_create_tol",
           "hqr_ls_plan_refine_info", "hqr_critical_path", "hqr_set_split_launch", "hqr_fp64_pipe_rates",
           "hqr_widen_f32", "hqr_ls_plan_run",
           "hqr_ls_plan_capture", "hqr_ls_plan_status", "hqr_ls_plan_correction", "hqr_ls_plan_info", "hqr_ls_plan_config",
           "hqr_ls_plan_free", "hqr_ls_plan_trace", "hqr_set_tuning", "hqr_autotune", "hqr_server_create", "hqr_server_start",
           "hqr_server_submit", "hqr_server_poll", "hqr_server_stats", "hqr_server_progress", "hqr_server_counters", "hqr_server_stop", "hqr_server_free", "hqr_debug_block_task", "hqr_factors_free", "hqr_set_timeout_ms", "hqr_strerror", "hqr_last_error", "hqr_set_slab_widths",
           "hqr_set_priority_policy", "hqr_set_panel_split",
           "hqr_last_launches"]


class HQRError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        text = _lib.hqr_strerror(status).decode() if _lib is not None else str(status)
        if status == ERR_CUDA and _lib is not None:
            text += ": " + _lib.hqr_last_error().decode()
        super().__init__("%s failed with status %d (%s)" % (where, status, text))


_lib = None


def library_path():
    return _build.OUT


def load(build_if_missing=False):
    """Load libhqr.so (building it first when asked). Raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if build_if_missing:
            _build.build()
        else:
            raise ImportError("libhqr.so is not built; run __graft_entry__.build() or "
                              "python -m paper_1110_1553_gb300._build")
    lib = ctypes.CDLL(path)
    vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
    pf = ctypes.POINTER(vp)
    lib.hqr_elim_list.argtypes = [i32, i32, i32, i32, i32, i32, vp, sz, ctypes.POINTER(sz)]
    lib.hqr_elim_list_domino.argtypes = [i32, i32, i32, i32, i32, i32, vp, sz, ctypes.POINTER(sz)]
    lib.hqr_validate_list.argtypes = [i32, i32, vp, sz]
    lib.hqr_task_graph.argtypes = [i32, i32, i32, i32, i32, vp, sz, i32, i32, vp, i64, vp, vp, i64,
                                   ctypes.POINTER(i64), ctypes.POINTER(i64)]
    lib.hqr_geqrf.argtypes = [vp, i32, i32, i32, i32, i32, i32, vp, sz, pf, vp]
    lib.hqr_refactor.argtypes = [vp, vp, i32, vp]
    lib.hqr_refactor_async.argtypes = [vp, vp, i32, vp]
    lib.hqr_status.argtypes = [vp, vp]
    lib.hqr_get_r.argtypes = [vp, vp, i32, vp]
    lib.hqr_get_tiles.argtypes = [vp, vp, i32, vp]
    lib.hqr_get_t.argtypes = [vp, vp, vp]
    ip = ctypes.POINTER(i32)
    lib.hqr_factors_info.argtypes = [vp, ip, ip, ip, ip, ip, ip, ctypes.POINTER(i64)]
    lib.hqr_kernel_ms.argtypes = [vp, ctypes.POINTER(ctypes.c_float)]
    lib.hqr_kernel_times.argtypes = [vp, ctypes.POINTER(ctypes.c_float), i32, ctypes.POINTER(i32)]
    lib.hqr_trace.argtypes = [vp, i32, vp, sz, ctypes.POINTER(sz)]
    lib.hqr_apply_q.argtypes = [vp, i32, vp, i32, i32, vp]
    lib.hqr_gels_qr.argtypes = [vp, i32, i32, i32, vp, i32, i32, vp, i32, i32, i32, i32, vp, sz, vp]
    lib.hqr_gels.argtypes = [vp, i32, i32, i32, vp, vp, i32, ctypes.c_double, i32, vp, vp]
    lib.hqr_ls_plan_create.argtypes = [i32, vp, vp, i32, i32, pf]
    lib.hqr_ls_plan_create_tol.argtypes = [i32, vp, vp, i32, i32, ctypes.c_double, pf]
    lib.hqr_ls_plan_refine_info.argtypes = [vp, i32, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_double),
                                            ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i64), vp]
    lib.hqr_ls_plan_run.argtypes = [vp, vp]
    lib.hqr_ls_plan_capture.argtypes = [vp, vp]
    lib.hqr_ls_plan_status.argtypes = [vp, vp]
    lib.hqr_ls_plan_info.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_float)]
    lib.hqr_ls_plan_config.argtypes = [vp, i32, vp]
    lib.hqr_ls_plan_correction.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_double), vp]
    lib.hqr_ls_plan_trace.argtypes = [vp, i32, vp, sz, ctypes.POINTER(sz)]
    lib.hqr_ls_plan_free.argtypes = [vp]
    lib.hqr_ls_plan_free.restype = None
    lib.hqr_set_tuning.argtypes = [i32, vp, vp]
    lib.hqr_server_create.argtypes = [vp, pf]
    lib.hqr_server_start.argtypes = [vp]
    lib.hqr_server_submit.argtypes = [vp, vp, ctypes.POINTER(i64)]
    lib.hqr_server_poll.argtypes = [vp, vp, i32, ctypes.POINTER(i32)]
    lib.hqr_server_stats.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i32),
                                     ctypes.POINTER(sz)]
    lib.hqr_server_counters.argtypes = [vp, vp, i32]
    lib.hqr_server_progress.argtypes = [vp, i64, ctypes.POINTER(i32), ctypes.POINTER(i32)]
    lib.hqr_server_stop.argtypes = [vp]
    lib.hqr_server_free.argtypes = [vp]
    lib.hqr_server_free.restype = None
    lib.hqr_critical_path.argtypes = [i32, i32, i32, i32, i32, vp, sz, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double)]
    lib.hqr_autotune.argtypes = [i32, vp, vp, i32, i32, i32, vp, vp, i32, ctypes.POINTER(i32), vp]
    lib.hqr_geqrf_r_noalloc.argtypes = [vp, i32, i32, i32, i32, i32, vp, sz, vp, i32, vp]
    lib.hqr_debug_block_task.argtypes = [vp, i64, i32]
    lib.hqr_factors_free.argtypes = [vp]
    lib.hqr_factors_free.restype = None
    lib.hqr_set_slab_widths.argtypes = [i32, i32, i32]
    lib.hqr_set_priority_policy.argtypes = [i32]
    lib.hqr_set_panel_split.argtypes = [i32]
    lib.hqr_set_split_launch.argtypes = [i32]
    lib.hqr_fp64_pipe_rates.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    lib.hqr_widen_f32.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong, ctypes.c_void_p]
    lib.hqr_set_timeout_ms.argtypes = [i64]
    lib.hqr_set_timeout_ms.restype = None
    lib.hqr_strerror.argtypes = [i32]
    lib.hqr_strerror.restype = ctypes.c_char_p
    lib.hqr_last_error.restype = ctypes.c_char_p
    lib.hqr_last_launches.restype = i64
    _lib = lib
    return lib


def _check(status, where):
    if status != 0:
        raise HQRError(status, where)


# ----------------------------------------------------------- host only --

def elim_list(m, n, a, p, low, high, domino=False):
    """HQR elimination list as a structured numpy array (fields k, i,
    killer, kind, level, step), sorted by (k, step, i); with domino=True the
    coupling level of Sec. 4.2 is included (hqr_elim_list_domino)."""
    lib = load()
    fn = lib.hqr_elim_list_domino if domino else lib.hqr_elim_list
    low = TREES.get(low, low)
    high = TREES.get(high, high)
    cnt = ctypes.c_size_t(0)
    st = fn(m, n, a, p, low, high, None, 0, ctypes.byref(cnt))
    if st not in (0, ERR_CAPACITY):
        _check(st, "hqr_elim_list")
    out = np.zeros(cnt.value, dtype=ELIM_DTYPE)
    st = fn(m, n, a, p, low, high, out.ctypes.data if cnt.value else None, cnt.value, ctypes.byref(cnt))
    _check(st, "hqr_elim_list")
    return out


def as_records(lst):
    """Structured elimination array -> list of (k, i, killer, kind, level, step)."""
    return [tuple(int(x) for x in r) for r in lst]


def to_array(records):
    return np.array([tuple(r) for r in records], dtype=ELIM_DTYPE)


def validate_list(m, n, records):
    """Status of hqr_validate_list (0 = valid)."""
    lib = load()
    arr = records if isinstance(records, np.ndarray) else to_array(records)
    arr = np.ascontiguousarray(arr, dtype=ELIM_DTYPE)
    return lib.hqr_validate_list(m, n, arr.ctypes.data if len(arr) else None, len(arr))


GRAPH_KINDS = {"factor": 0, "qt": 1, "q": 2, "ls": 3, "request": 4, "ls_tol": 5, "noalloc": 6}


def task_graph(m, n, nb, ib, records, prec=FP64, kind="factor", param=0):
    """A task graph of the library for an m x n tile matrix (host only): kind
    "factor" (hqr_geqrf), "qt" / "q" (Q^T / Q applied to `param` column
    slabs), "ls" (a plan's least-squares problem with `param` refinement
    rounds), "request" (the same as a server request, packing first). Returns an int32 array of (op, blk, i, r, k, j, c0, cw, trans,
    tgt) per task in a topological order, and the successors as CSR
    (offsets, ids)."""
    lib = load()
    arr = records if isinstance(records, np.ndarray) else to_array(records)
    arr = np.ascontiguousarray(arr, dtype=ELIM_DTYPE)
    lp = arr.ctypes.data if len(arr) else None
    kd = GRAPH_KINDS[kind]
    nt, ne = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(lib.hqr_task_graph(m, n, nb, ib, prec, lp, len(arr), kd, int(param), None, 0, None, None, 0,
                              ctypes.byref(nt), ctypes.byref(ne)), "hqr_task_graph")
    tasks = np.zeros((nt.value, 10), dtype=np.int32)
    ptr = np.zeros(nt.value + 1, dtype=np.int64)
    succ = np.zeros(max(ne.value, 1), dtype=np.int32)
    _check(lib.hqr_task_graph(m, n, nb, ib, prec, lp, len(arr), kd, int(param), tasks.ctypes.data, nt.value,
                              ptr.ctypes.data, succ.ctypes.data, len(succ), ctypes.byref(nt), ctypes.byref(ne)),
           "hqr_task_graph")
    return tasks, ptr, succ[:ne.value]


def critical_path(m, n, nb, ib, records, prec=FP64):
    """(critical path, total work) of the factorization graph in units of
    b^3 / 3 (hqr_critical_path)."""
    lib = load()
    arr = records if isinstance(records, np.ndarray) else to_array(records)
    arr = np.ascontiguousarray(arr, dtype=ELIM_DTYPE)
    cp, w = ctypes.c_double(0), ctypes.c_double(0)
    _check(lib.hqr_critical_path(m, n, nb, ib, prec, arr.ctypes.data if len(arr) else None, len(arr),
                                 ctypes.byref(cp), ctypes.byref(w)), "hqr_critical_path")
    return cp.value, w.value


def set_slab_widths(w=0, wt=0, vc=0):
    _check(load().hqr_set_slab_widths(int(w), int(wt), int(vc)), "hqr_set_slab_widths")


def set_panel_split(min_nb):
    """Split CUDA-core panels of tiles with nb >= min_nb into block tasks (0: never)."""
    _check(load().hqr_set_panel_split(int(min_nb)), "hqr_set_panel_split")


def fp64_pipe_rates():
    """(DFMA, DMMA) FP64 TFLOP/s of the current GPU (hqr_fp64_pipe_rates)."""
    a, b = ctypes.c_double(0), ctypes.c_double(0)
    _check(load().hqr_fp64_pipe_rates(ctypes.byref(a), ctypes.byref(b)), "hqr_fp64_pipe_rates")
    return a.value, b.value


def widen_f32(x, y, stream=None):
    """y <- x widened exactly from FP32 to FP64 (contiguous CUDA tensors of
    the same length), the refinement kernels' integer-pipe widening
    (hqr_widen_f32); asynchronous on `stream`."""
    if x.numel() != y.numel() or not (x.is_contiguous() and y.is_contiguous()):
        raise ValueError("x and y: contiguous, same length")
    _check(load().hqr_widen_f32(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), x.numel(),
                                _stream_ptr(stream)), "hqr_widen_f32")


def set_split_launch(on):
    """Mixed tensor-core / CUDA-core plans as two launches side by side (hqr_set_split_launch)."""
    _check(load().hqr_set_split_launch(1 if on else 0), "hqr_set_split_launch")


def set_priority_policy(policy):
    _check(load().hqr_set_priority_policy(int(policy)), "hqr_set_priority_policy")


def set_timeout_ms(ms):
    load().hqr_set_timeout_ms(int(ms))


def last_launches():
    return int(load().hqr_last_launches())


# -------------------------------------------------------------- device --

def _torch():
    import torch
    return torch


def _stream_ptr(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def prec_of(A, tensor=False):
    """Library precision of a matrix: FP64 for float64; for float32, FP32
    (CUDA-core arithmetic) or, with tensor=True, FP32_BF16X3 (tensor-core
    updates on tiles of 128)."""
    torch = _torch()
    if A.dtype == torch.float64:
        return FP64
    if A.dtype == torch.float32:
        return FP32_BF16X3 if tensor else FP32
    raise TypeError("expected a float64 or float32 CUDA tensor")


def _prec_dtype(dtype, tensor):
    torch = _torch()
    if dtype == torch.float64:
        return FP64
    return FP32_BF16X3 if tensor else FP32


def colmajor(A):
    """A column-major view or copy of a 2-D (or 1-D) float64/float32 CUDA
    tensor. Returns (tensor, ld)."""
    if A.dim() == 1:
        A = A.reshape(-1, 1)
    prec_of(A)
    if not A.is_cuda:
        raise TypeError("expected a CUDA tensor")
    M = A.shape[0]
    if A.stride(0) == 1 and (A.shape[1] == 1 or A.stride(1) >= max(M, 1)):
        return A, max(A.stride(1) if A.shape[1] > 1 else M, 1)
    C = A.t().contiguous().t()
    return C, M


def empty_colmajor(M, N, device="cuda", dtype=None):
    torch = _torch()
    return torch.empty((N, M), dtype=dtype or torch.float64, device=device).t()


class Factors:
    """A factorization A = Q R made by ``geqrf`` (owns the library object)."""

    def __init__(self, handle, M, N, dtype):
        self._h = handle
        self.M, self.N = M, N
        self.dtype = dtype
        lib = load()
        vals = [ctypes.c_int(0) for _ in range(6)]
        nt = ctypes.c_int64(0)
        _check(lib.hqr_factors_info(self._h, *[ctypes.byref(v) for v in vals], ctypes.byref(nt)),
               "hqr_factors_info")
        self.Mp, self.Np, self.m, self.n, self.nb, self.ib = [v.value for v in vals]
        self.ntasks = nt.value

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.hqr_factors_free(self._h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def refactor(self, A, stream=None):
        A, lda = colmajor(A)
        _check(load().hqr_refactor(self._h, ctypes.c_void_p(A.data_ptr()), lda, _stream_ptr(stream)),
               "hqr_refactor")

    def refactor_async(self, A, stream=None):
        A, lda = colmajor(A)
        _check(load().hqr_refactor_async(self._h, ctypes.c_void_p(A.data_ptr()), lda, _stream_ptr(stream)),
               "hqr_refactor_async")

    def debug_block_task(self, task, extra):
        _check(load().hqr_debug_block_task(self._h, int(task), int(extra)), "hqr_debug_block_task")

    def kernel_ms(self):
        """Device time of the last persistent task-kernel run (CUDA events)."""
        ms = ctypes.c_float(0)
        _check(load().hqr_kernel_ms(self._h, ctypes.byref(ms)), "hqr_kernel_ms")
        return ms.value

    def kernel_times(self):
        """Device times (ms) of the task-kernel runs since the previous call
        (at most the last 64), oldest first."""
        lib = load()
        buf = (ctypes.c_float * 64)()
        cnt = ctypes.c_int32(0)
        _check(lib.hqr_kernel_times(self._h, buf, 64, ctypes.byref(cnt)), "hqr_kernel_times")
        return [buf[q] for q in range(cnt.value)]

    def trace(self, enable=None):
        """enable=True/False switches per-task tracing; with no argument,
        returns the last run's records as an (ntasks, 3) uint64 array
        (start ns, end ns, CTA << 32 | SM)."""
        lib = load()
        cnt = ctypes.c_size_t(0)
        if enable is not None:
            _check(lib.hqr_trace(self._h, 1 if enable else 0, None, 0, ctypes.byref(cnt)), "hqr_trace")
            return None
        st = lib.hqr_trace(self._h, -1, None, 0, ctypes.byref(cnt))
        if st not in (0, ERR_CAPACITY):
            _check(st, "hqr_trace")
        out = np.zeros((cnt.value, 3), dtype=np.uint64)
        if cnt.value:
            _check(lib.hqr_trace(self._h, -1, out.ctypes.data, out.size, ctypes.byref(cnt)), "hqr_trace")
        return out

    def status(self, stream=None):
        return load().hqr_status(self._h, _stream_ptr(stream))

    def R(self, stream=None):
        R = empty_colmajor(self.N, self.N, dtype=self.dtype)
        _check(load().hqr_get_r(self._h, ctypes.c_void_p(R.data_ptr()), self.N, _stream_ptr(stream)),
               "hqr_get_r")
        return R

    def tiles(self, stream=None):
        X = empty_colmajor(self.Mp, self.Np, dtype=self.dtype)
        _check(load().hqr_get_tiles(self._h, ctypes.c_void_p(X.data_ptr()), self.Mp, _stream_ptr(stream)),
               "hqr_get_tiles")
        return X

    def T(self, stream=None):
        """All T factors, shape (n, m, 2, nb, ib): [k, i, which] is the
        ib x nb column-major array of tile (i, k) (which 0: GEQRT, 1: kill)."""
        torch = _torch()
        T = torch.empty((self.n, self.m, 2, self.nb, self.ib), dtype=self.dtype, device="cuda")
        _check(load().hqr_get_t(self._h, ctypes.c_void_p(T.data_ptr()), _stream_ptr(stream)), "hqr_get_t")
        return T

    def apply_q(self, B, trans, stream=None):
        """B <- Q^T B (trans=True) or Q B, in place when B is column-major;
        returns the result."""
        Bc, ldb = colmajor(B)
        nrhs = Bc.shape[1] if Bc.dim() == 2 else 1
        _check(load().hqr_apply_q(self._h, 1 if trans else 0, ctypes.c_void_p(Bc.data_ptr()), ldb, nrhs,
                                  _stream_ptr(stream)), "hqr_apply_q")
        if Bc.data_ptr() != B.data_ptr():
            B.copy_(Bc.reshape(B.shape))
        return B


def _list_arg(records):
    if records is None:
        return None, 0, None
    arr = records if isinstance(records, np.ndarray) else to_array(records)
    arr = np.ascontiguousarray(arr, dtype=ELIM_DTYPE)
    return ctypes.c_void_p(arr.ctypes.data), len(arr), arr


def geqrf(A, nb, ib, records=None, stream=None, tensor=False):
    """Tile QR of a float64 / float32 CUDA matrix with the given elimination
    list (None = library default). tensor=True (float32, nb = 128) runs the
    updates on the tensor cores. Returns a Factors object."""
    A, lda = colmajor(A)
    M, N = A.shape
    ptr, cnt, keep = _list_arg(records)
    h = ctypes.c_void_p(0)
    st = load().hqr_geqrf(ctypes.c_void_p(A.data_ptr()), M, N, lda, prec_of(A, tensor), nb, ib, ptr, cnt,
                          ctypes.byref(h), _stream_ptr(stream))
    del keep
    _check(st, "hqr_geqrf")
    return Factors(h, M, N, A.dtype)


class GelsInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("converged", ctypes.c_int), ("rel_correction", ctypes.c_double),
                ("backward_error", ctypes.c_double), ("normal_residual", ctypes.c_double),
                ("singular_index", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def gels(A, b, tol=1e-14, max_iter=30, tensor=False, stream=None, raise_on_error=True):
    """hqr_gels: least-squares solution x (float64, N) of min ||b - A x|| for
    a float32 (mixed precision) or float64 A and a float64 b of M entries,
    with tolerance-stopped refinement. Returns (x, status, info dict)."""
    torch = _torch()
    A, lda = colmajor(A)
    M, N = A.shape
    if b.dtype != torch.float64 or not b.is_contiguous() or b.numel() != M:
        raise TypeError("b must be a contiguous float64 CUDA vector of M entries")
    x = torch.zeros(N, dtype=torch.float64, device=A.device)
    info = GelsInfo()
    st = load().hqr_gels(ctypes.c_void_p(A.data_ptr()), M, N, lda, ctypes.c_void_p(b.data_ptr()),
                         ctypes.c_void_p(x.data_ptr()), prec_of(A, tensor), float(tol), int(max_iter),
                         ctypes.byref(info), _stream_ptr(stream))
    if raise_on_error and st not in (SUCCESS, ERR_NOCONV, ERR_SINGULAR):
        _check(st, "hqr_gels")
    return x, st, info.as_dict()


def gels_qr(A, b, nb, ib, records=None, stream=None, tensor=False):
    """hqr_gels_qr: least-squares solution x of min ||b - A x|| in the storage
    precision (b: M or M x nrhs)."""
    A, lda = colmajor(A)
    M, N = A.shape
    vec = b.dim() == 1
    bc, ldb = colmajor(b)
    nrhs = bc.shape[1]
    x = empty_colmajor(N, nrhs, dtype=A.dtype)
    ptr, cnt, keep = _list_arg(records)
    st = load().hqr_gels_qr(ctypes.c_void_p(A.data_ptr()), M, N, lda, ctypes.c_void_p(bc.data_ptr()), ldb,
                            nrhs, ctypes.c_void_p(x.data_ptr()), N, prec_of(A, tensor), nb, ib, ptr, cnt,
                            _stream_ptr(stream))
    del keep
    _check(st, "hqr_gels_qr")
    return x[:, 0] if vec else x


def geqrf_r_noalloc(A, nb, ib, records, R, stream=None):
    """R factor of A into the caller's column-major N x N tensor R through
    hqr_geqrf_r_noalloc, which allocates no memory (limits in include/hqr.h).
    Returns the library status (0 on success)."""
    A, lda = colmajor(A)
    M, N = A.shape
    if R.stride(0) != 1 or R.shape != (N, N):
        raise ValueError("R must be a column-major N x N float64 CUDA tensor")
    ptr, cnt, keep = _list_arg(records)
    st = load().hqr_geqrf_r_noalloc(ctypes.c_void_p(A.data_ptr()), M, N, lda, nb, ib, ptr, cnt,
                                    ctypes.c_void_p(R.data_ptr()), R.stride(1), _stream_ptr(stream))
    del keep
    return st


# ------------------------------------------------------- least squares --

class LSProblem(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int), ("N", ctypes.c_int), ("dA", ctypes.c_void_p), ("lda", ctypes.c_int),
                ("db", ctypes.c_void_p), ("dx", ctypes.c_void_p)]


class TileConfig(ctypes.Structure):
    _fields_ = [("nb", ctypes.c_int), ("ib", ctypes.c_int), ("a", ctypes.c_int), ("p", ctypes.c_int),
                ("low_tree", ctypes.c_int), ("high_tree", ctypes.c_int)]

    def as_tuple(self):
        return (self.nb, self.ib, self.a, self.p, self.low_tree, self.high_tree)


def tile_config(nb=0, ib=0, a=1, p=1, low="greedy", high="greedy"):
    return TileConfig(nb, ib, a, p, TREES.get(low, low), TREES.get(high, high))


class LSPlan:
    """Many least-squares problems solved by one persistent launch (see
    hqr_ls_plan_create). `problems` is a list of (A, b, x) CUDA tensors: A
    column-major M x N (float32 or float64, all the same), b float64 (M),
    x float64 (N, written by run()). tensor=True (float32) runs tiles of
    128 on the tensor cores."""

    def __init__(self, problems, refine_iters, configs=None, tensor=False, tol=None):
        """tol=None: `refine_iters` fixed rounds (hqr_ls_plan_create); a
        number: at most `refine_iters` rounds that stop at that tolerance
        (hqr_ls_plan_create_tol)."""
        torch = _torch()
        self._keep = []
        arr = (LSProblem * len(problems))()
        dtype = None
        for q, (A, b, x) in enumerate(problems):
            Ac, lda = colmajor(A)
            if dtype is None:
                dtype = Ac.dtype
            elif Ac.dtype != dtype:
                raise TypeError("all matrices of a plan share one precision")
            if b.dtype != torch.float64 or x.dtype != torch.float64 or not b.is_contiguous() \
                    or not x.is_contiguous():
                raise TypeError("b and x must be contiguous float64 CUDA vectors")
            self._keep += [Ac, b, x]
            arr[q] = LSProblem(Ac.shape[0], Ac.shape[1], Ac.data_ptr(), lda, b.data_ptr(), x.data_ptr())
        cfg = None
        if configs is not None:
            cfg = (TileConfig * len(problems))(*configs)
        h = ctypes.c_void_p(0)
        if tol is None:
            st = load().hqr_ls_plan_create(len(problems), ctypes.byref(arr), ctypes.byref(cfg) if cfg else None,
                                           prec_of(self._keep[0], tensor), int(refine_iters), ctypes.byref(h))
            _check(st, "hqr_ls_plan_create")
        else:
            st = load().hqr_ls_plan_create_tol(len(problems), ctypes.byref(arr),
                                               ctypes.byref(cfg) if cfg else None, prec_of(self._keep[0], tensor),
                                               int(refine_iters), float(tol), ctypes.byref(h))
            _check(st, "hqr_ls_plan_create_tol")
        self._h = h
        self.count = len(problems)

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.hqr_ls_plan_free(self._h)
            self._h = None

    def run(self, stream=None):
        _check(load().hqr_ls_plan_run(self._h, _stream_ptr(stream)), "hqr_ls_plan_run")

    def capture(self, stream):
        _check(load().hqr_ls_plan_capture(self._h, ctypes.c_void_p(stream.cuda_stream)), "hqr_ls_plan_capture")

    def status(self, stream=None):
        return load().hqr_ls_plan_status(self._h, _stream_ptr(stream))

    def refine_info(self, idx=0, stream=None):
        """(rounds applied, last applied correction, tolerance met, first zero
        diagonal column or -1, compensated rounds) of problem idx
        (hqr_ls_plan_refine_info)."""
        it, met, nc = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0)
        rel, sing = ctypes.c_double(0), ctypes.c_int64(0)
        _check(load().hqr_ls_plan_refine_info(self._h, idx, ctypes.byref(it), ctypes.byref(rel), ctypes.byref(met),
                                              ctypes.byref(nc), ctypes.byref(sing), _stream_ptr(stream)),
               "hqr_ls_plan_refine_info")
        return it.value, rel.value, bool(met.value), sing.value, nc.value

    def correction(self, idx=0, stream=None):
        """max |d| / max |x| of the last refinement correction of problem idx (-1: no rounds)."""
        rel = ctypes.c_double(0)
        _check(load().hqr_ls_plan_correction(self._h, int(idx), ctypes.byref(rel), _stream_ptr(stream)),
               "hqr_ls_plan_correction")
        return rel.value

    def info(self):
        nt, fl, ms = ctypes.c_int64(0), ctypes.c_double(0), ctypes.c_float(0)
        _check(load().hqr_ls_plan_info(self._h, ctypes.byref(nt), ctypes.byref(fl), ctypes.byref(ms)),
               "hqr_ls_plan_info")
        return {"tasks": nt.value, "qr_flops": fl.value, "kernel_ms": ms.value}

    def trace(self, enable=None):
        """enable=True/False switches tracing; no argument: the last run's
        records, (ntasks, 4) uint64 (start, end, CTA << 32 | SM, op << 24 | pid)."""
        lib = load()
        cnt = ctypes.c_size_t(0)
        if enable is not None:
            _check(lib.hqr_ls_plan_trace(self._h, 1 if enable else 0, None, 0, ctypes.byref(cnt)),
                   "hqr_ls_plan_trace")
            return None
        st = lib.hqr_ls_plan_trace(self._h, -1, None, 0, ctypes.byref(cnt))
        if st not in (0, ERR_CAPACITY):
            _check(st, "hqr_ls_plan_trace")
        out = np.zeros((cnt.value, 4), dtype=np.uint64)
        if cnt.value:
            _check(lib.hqr_ls_plan_trace(self._h, -1, out.ctypes.data, out.size, ctypes.byref(cnt)),
                   "hqr_ls_plan_trace")
        return out

    def config(self, idx):
        c = TileConfig()
        _check(load().hqr_ls_plan_config(self._h, idx, ctypes.byref(c)), "hqr_ls_plan_config")
        return c.as_tuple()


def set_tuning(table):
    """Install an autotuner table {(floor(log2 M), floor(log2 N)): TileConfig}."""
    keys = (ctypes.c_int * (2 * max(1, len(table))))()
    cfgs = (TileConfig * max(1, len(table)))()
    for e, ((lm, ln), c) in enumerate(sorted(table.items())):
        keys[2 * e], keys[2 * e + 1] = lm, ln
        cfgs[e] = c
    _check(load().hqr_set_tuning(len(table), keys, cfgs), "hqr_set_tuning")


def autotune(shapes, dtype, refine_iters, reps=32, stream=None, tensor=False):
    """Run the library's measured autotuner over the shape classes of
    `shapes` [(M, N), ...]; installs and returns the table
    {(log2 M, log2 N): (nb, ib, a, p, low, high)}."""
    n = len(shapes)
    Ms = (ctypes.c_int * n)(*[m for m, _ in shapes])
    Ns = (ctypes.c_int * n)(*[k for _, k in shapes])
    cap = 256
    keys = (ctypes.c_int * (2 * cap))()
    cfgs = (TileConfig * cap)()
    nout = ctypes.c_int(0)
    prec = _prec_dtype(dtype, tensor)
    _check(load().hqr_autotune(n, Ms, Ns, prec, int(refine_iters), int(reps), keys, cfgs, cap, ctypes.byref(nout),
                               _stream_ptr(stream)), "hqr_autotune")
    return {(keys[2 * e], keys[2 * e + 1]): cfgs[e].as_tuple() for e in range(nout.value)}


# --------------------------------------------------------------- server --

class ServerOpts(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("refine_iters", ctypes.c_int), ("max_live", ctypes.c_int),
                ("hbm_budget", ctypes.c_size_t), ("task_pool", ctypes.c_int64), ("edge_pool", ctypes.c_int64)]


class Server:
    """Continuous-batching least-squares server (hqr_server_*). submit()
    returns a ticket, or None when the request does not fit right now."""

    def __init__(self, dtype, refine_iters, max_live=1024, hbm_budget=8 << 30, task_pool=8 << 20,
                 edge_pool=32 << 20, tensor=False):
        prec = _prec_dtype(dtype, tensor)
        o = ServerOpts(prec, int(refine_iters), int(max_live), int(hbm_budget), int(task_pool), int(edge_pool))
        h = ctypes.c_void_p(0)
        _check(load().hqr_server_create(ctypes.byref(o), ctypes.byref(h)), "hqr_server_create")
        self._h = h
        self._keep = {}
        self._done = (ctypes.c_int64 * 4096)()

    def start(self):
        _check(load().hqr_server_start(self._h), "hqr_server_start")

    def submit(self, A, b, x):
        Ac, lda = colmajor(A)
        pr = LSProblem(Ac.shape[0], Ac.shape[1], Ac.data_ptr(), lda, b.data_ptr(), x.data_ptr())
        t = ctypes.c_int64(0)
        st = load().hqr_server_submit(self._h, ctypes.byref(pr), ctypes.byref(t))
        if st == ERR_BUSY:
            return None
        _check(st, "hqr_server_submit")
        self._keep[t.value] = (Ac, b, x)
        return t.value

    def poll(self):
        """Tickets completed since the last poll."""
        cnt = ctypes.c_int(0)
        st = load().hqr_server_poll(self._h, self._done, len(self._done), ctypes.byref(cnt))
        _check(st, "hqr_server_poll")
        out = [self._done[q] for q in range(min(cnt.value, len(self._done)))]
        for t in out:
            self._keep.pop(t, None)
        return out

    def stats(self):
        s, c, lv, by = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int(0), ctypes.c_size_t(0)
        _check(load().hqr_server_stats(self._h, ctypes.byref(s), ctypes.byref(c), ctypes.byref(lv), ctypes.byref(by)),
               "hqr_server_stats")
        return {"submitted": s.value, "completed": c.value, "live": lv.value, "bytes_in_use": by.value}

    def progress(self, ticket):
        """(tasks completed, tasks in total) of a live request."""
        d, t = ctypes.c_int(0), ctypes.c_int(0)
        _check(load().hqr_server_progress(self._h, ctypes.c_int64(ticket), ctypes.byref(d), ctypes.byref(t)),
               "hqr_server_progress")
        return d.value, t.value

    def counters(self):
        out = (ctypes.c_uint32 * 5)()
        _check(load().hqr_server_counters(self._h, out, 5), "hqr_server_counters")
        return {"inbox_claimed": out[0], "inbox_posted": out[1], "stop": out[2], "outstanding": out[3],
                "running": bool(out[4])}

    def stop(self):
        _check(load().hqr_server_stop(self._h), "hqr_server_stop")

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.hqr_server_free(self._h)
            self._h = None
