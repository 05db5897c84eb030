"""ctypes binding of ``libspand.so`` (include/spand.h).

Argument marshalling only: host arrays are passed as numpy buffers, device
arrays as ``torch.Tensor.data_ptr()`` and streams as the raw ``cudaStream_t``
of a ``torch.cuda.Stream``.  Every computation happens in the library.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libspand.so")

SPAND_OK = 0
SPAND_EINVAL = -1
SPAND_ENOTSPD = -2
SPAND_ENOMEM = -3
SPAND_ECUDA = -4
SPAND_ENOCONV = -5
SPAND_ESTATE = -6
SPAND_ETIMEOUT = -7

# Every entry point declared in include/spand.h.
EXPORTS = [
    "spand_analyze", "spand_factor", "spand_tune", "spand_test_set_qr_wait", "spand_apply",
    "spand_pcg",
    "spand_pcg_host",
    "spand_matvec", "spand_info", "spand_ranks", "spand_cluster_map", "spand_num_clusters",
    "spand_pcg_noalloc", "spand_set_profiling", "spand_kernel_stats",
    "spand_apply_many", "spand_pcg_many",
    "spand_batch_create", "spand_batch_factor", "spand_batch_pcg", "spand_batch_info",
    "spand_batch_set_profiling", "spand_batch_kernel_stats", "spand_batch_destroy",
    "spand_server_create", "spand_server_add", "spand_server_submit", "spand_server_wait",
    "spand_server_get_stats", "spand_server_destroy",
    "spand_measure_fma_peak", "spand_destroy", "spand_strerror", "spand_last_error",
]
_VOID = ("spand_destroy", "spand_batch_destroy", "spand_server_destroy", "spand_strerror",
         "spand_last_error")


class SpandError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"spand error {code}: {msg}")
        self.code = code


class _CSR(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("rowptr", ctypes.c_void_p), ("colind", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class _Opts(ctypes.Structure):
    _fields_ = [("skip", ctypes.c_int32), ("maxit", ctypes.c_int32),
                ("true_res_every", ctypes.c_int32), ("max_restarts", ctypes.c_int32),
                ("rrqr_kernel", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("plain_launches", ctypes.c_int32), ("rrqr_threads", ctypes.c_int32),
                ("partition", ctypes.c_int32), ("prescale", ctypes.c_int32),
                ("schur_simt", ctypes.c_int32), ("apply_kernels", ctypes.c_int32)]


class _Stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz_a", ctypes.c_int64), ("nnz_factor", ctypes.c_int64),
                ("mu", ctypes.c_double), ("nlevels", ctypes.c_int32), ("skip", ctypes.c_int32),
                ("scheme", ctypes.c_int32), ("eps", ctypes.c_double), ("nstages", ctypes.c_int32),
                ("nclusters_total", ctypes.c_int32), ("ninterfaces_sparsified", ctypes.c_int32),
                ("factor_ms", ctypes.c_double), ("pcg_ms", ctypes.c_double),
                ("pcg_iters", ctypes.c_int32), ("pcg_relres", ctypes.c_double),
                ("kernel_launches", ctypes.c_int64), ("device_bytes", ctypes.c_int64)]


class _ServerOpts(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_size_t), ("max_entries", ctypes.c_int64),
                ("max_segments", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("tol", ctypes.c_double)]


class _ServerStats(ctypes.Structure):
    _fields_ = [("requests", ctypes.c_int64), ("solves", ctypes.c_int64),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("max_ms", ctypes.c_double),
                ("elapsed_s", ctypes.c_double), ("solves_per_s", ctypes.c_double),
                ("ticks", ctypes.c_int64), ("max_inflight", ctypes.c_int32),
                ("resident_problems", ctypes.c_int32), ("resident_bytes", ctypes.c_int64),
                ("factor_wait_p50_ms", ctypes.c_double), ("factor_wait_p99_ms", ctypes.c_double),
                ("queue_p50_ms", ctypes.c_double), ("queue_p99_ms", ctypes.c_double),
                ("solve_p50_ms", ctypes.c_double), ("solve_p99_ms", ctypes.c_double),
                ("max_split_ms", ctypes.c_double * 3)]


class _KStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64),
                ("total_ms", ctypes.c_double), ("flops", ctypes.c_double), ("bytes", ctypes.c_double)]


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libspand.so; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                           "or python -m paper_2007_00789_gb300.build")
    L = ctypes.CDLL(path)
    vp, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    L.spand_analyze.argtypes = [ctypes.POINTER(_CSR), vp, ctypes.c_int, ctypes.c_int, f64,
                                ctypes.c_int, ctypes.POINTER(_Opts), ctypes.POINTER(vp)]
    L.spand_factor.argtypes = [vp, vp]
    L.spand_test_set_qr_wait.argtypes = [vp, i64, i32]
    L.spand_tune.argtypes = [vp, vp, vp]
    L.spand_apply.argtypes = [vp, vp, vp, vp]
    L.spand_pcg.argtypes = [vp, vp, vp, f64, ctypes.POINTER(i32), ctypes.POINTER(f64), vp]
    L.spand_pcg_host.argtypes = [vp, vp, vp, f64, ctypes.POINTER(i32), ctypes.POINTER(f64), vp]
    L.spand_pcg_noalloc.argtypes = [vp, vp, vp, f64, ctypes.POINTER(i32), ctypes.POINTER(f64), vp]
    L.spand_matvec.argtypes = [vp, vp, vp, vp]
    L.spand_apply_many.argtypes = [vp, vp, vp, i32, i64, vp]
    L.spand_pcg_many.argtypes = [vp, vp, vp, i32, i64, f64, vp, vp, vp]
    L.spand_info.argtypes = [vp, ctypes.POINTER(_Stats)]
    L.spand_ranks.argtypes = [vp, vp, i64, ctypes.POINTER(i64)]
    L.spand_cluster_map.argtypes = [vp, ctypes.c_int, vp]
    L.spand_num_clusters.argtypes = [vp, ctypes.c_int, ctypes.POINTER(i32)]
    L.spand_set_profiling.argtypes = [vp, ctypes.c_int]
    L.spand_kernel_stats.argtypes = [vp, ctypes.POINTER(_KStat), ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    L.spand_batch_create.argtypes = [vp, i32, ctypes.POINTER(vp)]
    L.spand_batch_factor.argtypes = [vp, vp]
    L.spand_batch_pcg.argtypes = [vp, vp, vp, f64, vp, vp, vp]
    L.spand_batch_info.argtypes = [vp, ctypes.POINTER(f64), ctypes.POINTER(f64),
                                   ctypes.POINTER(i64), ctypes.POINTER(i64)]
    L.spand_batch_set_profiling.argtypes = [vp, ctypes.c_int]
    L.spand_batch_kernel_stats.argtypes = [vp, ctypes.POINTER(_KStat), ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_int)]
    L.spand_batch_destroy.argtypes = [vp]
    L.spand_batch_destroy.restype = None
    L.spand_server_create.argtypes = [ctypes.POINTER(_ServerOpts), ctypes.POINTER(vp)]
    L.spand_server_add.argtypes = [vp, vp, i32, ctypes.POINTER(i32)]
    L.spand_server_submit.argtypes = [vp, i32, i32, vp, vp, ctypes.POINTER(i64)]
    L.spand_server_wait.argtypes = [vp, i64, vp, vp, ctypes.POINTER(f64)]
    L.spand_server_get_stats.argtypes = [vp, ctypes.POINTER(_ServerStats)]
    L.spand_server_destroy.argtypes = [vp]
    L.spand_server_destroy.restype = None
    L.spand_measure_fma_peak.argtypes = [ctypes.c_int, ctypes.POINTER(f64), ctypes.POINTER(f64)]
    L.spand_destroy.argtypes = [vp]
    L.spand_destroy.restype = None
    L.spand_strerror.argtypes = [ctypes.c_int]
    L.spand_strerror.restype = ctypes.c_char_p
    L.spand_last_error.argtypes = []
    L.spand_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in _VOID:
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(rc: int, allow=()):
    if rc != SPAND_OK and rc not in allow:
        L = load_library()
        raise SpandError(rc, f"{L.spand_strerror(rc).decode()}: {L.spand_last_error().decode()}")
    return rc


def _stream_ptr(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dptr(t) -> int:
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    return t.data_ptr()


class Spand:
    """One analysed (and possibly factored) SPD system A with grid coordinates."""

    def __init__(self, rowptr, colind, val, coords, nlevels: int, eps: float, scheme: int = 1,
                 skip: int | None = None, maxit: int | None = None, true_res_every: int | None = None,
                 max_restarts: int | None = None, rrqr_kernel: int = 0, precision: int = 0,
                 plain_launches: bool = False, rrqr_threads: int = 0, partition: int = 0,
                 prescale: bool = False, schur_simt: bool = False, apply_kernels: int = 0):
        """coords None (or partition=1): algebraic nested dissection of A's graph;
        prescale: factor D^{-1/2} A D^{-1/2} and precondition with D^{-1/2} M~ D^{-1/2}."""
        L = load_library()
        self._lib = L
        self._rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
        self._colind = np.ascontiguousarray(colind, dtype=np.int32)
        self._val = np.ascontiguousarray(val, dtype=np.float64)
        if coords is not None:
            coords = np.ascontiguousarray(coords, dtype=np.float64)
            if coords.ndim == 1:
                coords = coords[:, None]
        self.n = int(self._rowptr.size - 1)
        self.nnz = int(self._rowptr[-1])
        csr = _CSR(self.n, self.nnz, self._rowptr.ctypes.data, self._colind.ctypes.data,
                   self._val.ctypes.data)
        opts = _Opts(-1 if skip is None else int(skip), 0 if maxit is None else int(maxit),
                     0 if true_res_every is None else int(true_res_every),
                     -1 if max_restarts is None else int(max_restarts), int(rrqr_kernel),
                     int(precision), 1 if plain_launches else 0, int(rrqr_threads),
                     int(partition), 1 if prescale else 0, 1 if schur_simt else 0,
                     int(apply_kernels))
        h = ctypes.c_void_p()
        cptr = None if coords is None else coords.ctypes.data
        cdim = 0 if coords is None else coords.shape[1]
        _check(L.spand_analyze(ctypes.byref(csr), cptr, cdim, int(nlevels), float(eps), int(scheme),
                               ctypes.byref(opts), ctypes.byref(h)))
        self._h = h
        self.nlevels = int(nlevels)

    @classmethod
    def from_problem(cls, prob, nlevels, eps, scheme=1, **kw):
        return cls(prob.rowptr, prob.colind, prob.val, prob.coords, nlevels, eps, scheme, **kw)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.spand_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def factor(self, stream=None):
        _check(self._lib.spand_factor(self._h, _stream_ptr(stream)))

    def tune(self, stream=None) -> dict:
        """spand_tune: the fastest RRQR launch shape per size bucket and the faster apply form;
        leaves the handle factored.  Returns {bucket: (threads per CTA, cluster growth)} for the
        buckets that occurred and {"apply": "persistent" | "per_phase"}."""
        ch = np.zeros(12, dtype=np.int32)
        _check(self._lib.spand_tune(self._h, _stream_ptr(stream), ch.ctypes.data))
        out = {b + 1: (int(ch[2 * b]), int(ch[2 * b + 1])) for b in range(5) if ch[2 * b]}
        out["apply"] = "persistent" if ch[10] == 0 else "per_phase"
        return out

    def test_set_qr_wait(self, limit: int = 0, unreachable: bool = False):
        """Testing hook of the multi-CTA RRQR's bounded barrier wait (spand_test_set_qr_wait)."""
        _check(self._lib.spand_test_set_qr_wait(self._h, int(limit), 1 if unreachable else 0))

    def apply(self, r, z, stream=None):
        _check(self._lib.spand_apply(self._h, _dptr(r), _dptr(z), _stream_ptr(stream)))

    def matvec(self, x, y, stream=None):
        _check(self._lib.spand_matvec(self._h, _dptr(x), _dptr(y), _stream_ptr(stream)))

    def pcg(self, b, x, tol: float, stream=None, allow_noconv: bool = False):
        it = ctypes.c_int32()
        rel = ctypes.c_double()
        _check(self._lib.spand_pcg(self._h, _dptr(b), _dptr(x), float(tol), ctypes.byref(it),
                                   ctypes.byref(rel), _stream_ptr(stream)),
               allow=(SPAND_ENOCONV,) if allow_noconv else ())
        return int(it.value), float(rel.value)

    def apply_many(self, r, z, stream=None):
        """z[j] = M r[j] for the rows of 2-D float64 CUDA tensors (nrhs, ld >= n)."""
        nrhs, ld = r.shape
        if z.shape != r.shape or r.stride(1) != 1 or z.stride(1) != 1:
            raise ValueError("r and z: same shape, contiguous rows")
        _check(self._lib.spand_apply_many(self._h, _dptr(r), _dptr(z), nrhs, r.stride(0),
                                          _stream_ptr(stream)))

    def pcg_many(self, b, x, tol: float, stream=None, allow_noconv: bool = False):
        """PCG for every row of b (nrhs, ld >= n) into x; returns (iterations, relres) arrays."""
        nrhs = b.shape[0]
        if x.shape != b.shape or b.stride(1) != 1 or x.stride(1) != 1:
            raise ValueError("b and x: same shape, contiguous rows")
        it = np.zeros(nrhs, dtype=np.int32)
        rel = np.zeros(nrhs, dtype=np.float64)
        _check(self._lib.spand_pcg_many(self._h, _dptr(b), _dptr(x), nrhs, b.stride(0), float(tol),
                                        it.ctypes.data, rel.ctypes.data, _stream_ptr(stream)),
               allow=(SPAND_ENOCONV,) if allow_noconv else ())
        return it, rel

    def pcg_noalloc(self, b, x, tol: float, stream=None):
        """spand_pcg without any allocation (work vectors in the library's static array)."""
        it = ctypes.c_int32()
        rel = ctypes.c_double()
        _check(self._lib.spand_pcg_noalloc(self._h, _dptr(b), _dptr(x), float(tol), ctypes.byref(it),
                                           ctypes.byref(rel), _stream_ptr(stream)))
        return int(it.value), float(rel.value)

    def pcg_host(self, b: np.ndarray, tol: float, stream=None, out: np.ndarray | None = None):
        """PCG from host buffers; out (optional): the float64 host array that receives
        x (e.g. a view of pinned memory), else a new one."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        if out is None:
            x = np.empty_like(b)
        else:
            x = out
            if x.dtype != np.float64 or x.shape != b.shape or not x.flags.c_contiguous:
                raise ValueError("out must be a contiguous float64 array shaped like b")
        it = ctypes.c_int32()
        rel = ctypes.c_double()
        _check(self._lib.spand_pcg_host(self._h, b.ctypes.data, x.ctypes.data, float(tol),
                                        ctypes.byref(it), ctypes.byref(rel), _stream_ptr(stream)))
        return x, int(it.value), float(rel.value)

    def info(self) -> dict:
        s = _Stats()
        _check(self._lib.spand_info(self._h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in _Stats._fields_}

    def ranks(self) -> np.ndarray:
        """(size at stage start, rank or -1, near-tie flags) for every cluster of every stage."""
        cnt = ctypes.c_int64()
        self._lib.spand_ranks(self._h, None, 0, ctypes.byref(cnt))
        out = np.empty((cnt.value, 3), dtype=np.int32)
        _check(self._lib.spand_ranks(self._h, out.ctypes.data, cnt.value, ctypes.byref(cnt)))
        return out

    def set_profiling(self, on: bool):
        _check(self._lib.spand_set_profiling(self._h, 1 if on else 0))

    def kernel_stats(self) -> list[dict]:
        """Per kernel kind: launches, total_ms, algorithmic flops and bytes."""
        arr = (_KStat * 64)()
        cnt = ctypes.c_int()
        _check(self._lib.spand_kernel_stats(self._h, arr, 64, ctypes.byref(cnt)))
        return [{"name": arr[i].name.decode(), "launches": int(arr[i].launches),
                 "total_ms": float(arr[i].total_ms), "flops": float(arr[i].flops),
                 "bytes": float(arr[i].bytes)} for i in range(cnt.value)]

    def num_clusters(self, stage: int) -> int:
        c = ctypes.c_int32()
        _check(self._lib.spand_num_clusters(self._h, int(stage), ctypes.byref(c)))
        return int(c.value)

    def cluster_map(self, stage: int) -> np.ndarray:
        out = np.empty(self.n, dtype=np.int32)
        _check(self._lib.spand_cluster_map(self._h, int(stage), out.ctypes.data))
        return out


def measure_fma_peak(precision: int = 0) -> tuple[float, float]:
    """(TFLOP/s, best launch ms) of FMA chains on the current device (spand_measure_fma_peak)."""
    L = load_library()
    tf = ctypes.c_double()
    ms = ctypes.c_double()
    _check(L.spand_measure_fma_peak(int(precision), ctypes.byref(tf), ctypes.byref(ms)))
    return float(tf.value), float(ms.value)


def _kstats(fn, h) -> list[dict]:
    arr = (_KStat * 64)()
    cnt = ctypes.c_int()
    _check(fn(h, arr, 64, ctypes.byref(cnt)))
    return [{"name": arr[i].name.decode(), "launches": int(arr[i].launches),
             "total_ms": float(arr[i].total_ms), "flops": float(arr[i].flops),
             "bytes": float(arr[i].bytes)} for i in range(cnt.value)]


class SpandBatch:
    """Independent problems factored and solved together (spand_batch_*).

    The member ``Spand`` objects must stay open while the batch exists."""

    def __init__(self, members):
        self._lib = load_library()
        self.members = list(members)
        arr = (ctypes.c_void_p * len(self.members))(*[m._h.value for m in self.members])
        h = ctypes.c_void_p()
        _check(self._lib.spand_batch_create(arr, len(self.members), ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.spand_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def factor(self, stream=None):
        _check(self._lib.spand_batch_factor(self._h, _stream_ptr(stream)))

    def pcg(self, bs, xs, tol: float, stream=None, allow_noconv: bool = False):
        """bs, xs: lists of float64 CUDA tensors; returns (iterations, true relative residuals)."""
        k = len(self.members)
        if len(bs) != k or len(xs) != k:
            raise ValueError("one right-hand side and one solution vector per member")
        bp = (ctypes.c_void_p * k)(*[_dptr(b) for b in bs])
        xp = (ctypes.c_void_p * k)(*[_dptr(x) for x in xs])
        it = np.zeros(k, dtype=np.int32)
        rel = np.zeros(k, dtype=np.float64)
        _check(self._lib.spand_batch_pcg(self._h, bp, xp, float(tol), it.ctypes.data,
                                         rel.ctypes.data, _stream_ptr(stream)),
               allow=(SPAND_ENOCONV,) if allow_noconv else ())
        return it, rel

    def info(self) -> dict:
        fm, pm = ctypes.c_double(), ctypes.c_double()
        nl, nt = ctypes.c_int64(), ctypes.c_int64()
        _check(self._lib.spand_batch_info(self._h, ctypes.byref(fm), ctypes.byref(pm),
                                          ctypes.byref(nl), ctypes.byref(nt)))
        return {"factor_ms": fm.value, "pcg_ms": pm.value, "launches": int(nl.value),
                "ticks": int(nt.value)}

    def set_profiling(self, on: bool):
        _check(self._lib.spand_batch_set_profiling(self._h, 1 if on else 0))

    def kernel_stats(self) -> list[dict]:
        return _kstats(self._lib.spand_batch_kernel_stats, self._h)


class SpandServer:
    """Resident factored problems answering multi-RHS solve requests (spand_server_*).

    ``submit`` returns at once; ``wait`` blocks (without the GIL) until the
    request is done.  Added ``Spand`` objects must stay open while the server
    exists and must not be used directly meanwhile."""

    def __init__(self, hbm_budget: int = 0, max_entries: int = 0, max_segments: int = 0,
                 precision: int = 0, tol: float = 1e-10):
        self._lib = load_library()
        o = _ServerOpts(int(hbm_budget), int(max_entries), int(max_segments), int(precision),
                        float(tol))
        h = ctypes.c_void_p()
        _check(self._lib.spand_server_create(ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        self._mats = {}
        self._pending = {}

    def add(self, problem: "Spand", pinned: bool = False) -> int:
        mid = ctypes.c_int32()
        _check(self._lib.spand_server_add(self._h, problem._h, 1 if pinned else 0, ctypes.byref(mid)))
        self._mats[int(mid.value)] = problem
        return int(mid.value)

    def submit(self, mid: int, b: np.ndarray) -> int:
        """b: (n,) or (nrhs, n) float64; returns the request id."""
        n = self._mats[mid].n
        b = np.ascontiguousarray(np.atleast_2d(b), dtype=np.float64)
        if b.shape[1] != n:
            raise ValueError("right-hand sides must have n entries")
        x = np.empty_like(b)
        rid = ctypes.c_int64()
        _check(self._lib.spand_server_submit(self._h, int(mid), b.shape[0], b.ctypes.data,
                                             x.ctypes.data, ctypes.byref(rid)))
        self._pending[int(rid.value)] = (b, x)
        return int(rid.value)

    def wait(self, rid: int, allow_noconv: bool = False):
        """Returns (x (nrhs, n), iterations, true relative residuals, latency in ms)."""
        b, x = self._pending[rid]
        it = np.zeros(b.shape[0], dtype=np.int32)
        rel = np.zeros(b.shape[0], dtype=np.float64)
        lat = ctypes.c_double()
        try:
            _check(self._lib.spand_server_wait(self._h, int(rid), it.ctypes.data, rel.ctypes.data,
                                               ctypes.byref(lat)),
                   allow=(SPAND_ENOCONV,) if allow_noconv else ())
        finally:
            self._pending.pop(rid, None)
        return x, it, rel, float(lat.value)

    def stats(self) -> dict:
        s = _ServerStats()
        _check(self._lib.spand_server_get_stats(self._h, ctypes.byref(s)))
        out = {f: getattr(s, f) for f, _ in _ServerStats._fields_}
        out["max_split_ms"] = list(out["max_split_ms"])
        return out

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.spand_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
