"""Thin ctypes binding of libknor.so (include/knor.h).

Argument marshalling only: every step of Lloyd's iteration runs in the CUDA
kernels of libknor.so.  Tensors may live on the GPU (their device pointer is
passed through) or on the host.  There is no fallback: if libknor.so has not
been built, or cannot be loaded, every entry point raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libknor.so")
_lib = None

KNOR_OK, KNOR_ERR_ARG, KNOR_ERR_OOM, KNOR_ERR_CUDA, KNOR_ERR_TIMEOUT, KNOR_ERR_STATE = 0, -1, -2, -3, -4, -5
KNOR_INIT_FORGY, KNOR_INIT_EXPLICIT, KNOR_INIT_KMEANSPP = 0, 1, 2
INITS = {"forgy": KNOR_INIT_FORGY, "explicit": KNOR_INIT_EXPLICIT, "kmeans++": KNOR_INIT_KMEANSPP}
PRECISIONS = {"fp32": 0, "bf16": 1, "fp8": 2, "fp16": 3}


class KnorError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"knor status {status}: {msg}")
        self.status = status


class Opts(ctypes.Structure):
    _fields_ = [("no_prune", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("full_recompute_every", ctypes.c_int32), ("debug_invariants", ctypes.c_int32),
                ("elkan", ctypes.c_int32), ("points_in_host", ctypes.c_int32)]


class IterStats(ctypes.Structure):
    _fields_ = [("changed", ctypes.c_int64), ("clause1_skipped", ctypes.c_int64),
                ("dist_evals", ctypes.c_int64), ("rechecked", ctypes.c_int64),
                ("empty", ctypes.c_int32), ("iteration", ctypes.c_int32),
                ("violations", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64 * 8), ("ms", ctypes.c_double * 8)]


KERNELS = ("dense", "mti", "reduce", "table", "recheck", "sums", "select", "delta")


class BatchInstance(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("d", ctypes.c_int32), ("k", ctypes.c_int32),
                ("iterations", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("changed_last", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}

_SIGS = {
    "knor_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                   ctypes.c_int, ctypes.c_uint64, ctypes.POINTER(Opts),
                                   ctypes.POINTER(ctypes.c_void_p)]),
    "knor_set_init_centroids": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "knor_reset": (ctypes.c_int, [ctypes.c_void_p]),
    "knor_iterate": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(IterStats)]),
    "knor_run": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                ctypes.POINTER(IterStats)]),
    "knor_get_assignments": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "knor_get_centroids": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "knor_get_centroids_f32": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "knor_get_init_indices": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "knor_get_iteration": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32)]),
    "knor_stream": (ctypes.c_void_p, [ctypes.c_void_p]),
    "knor_get_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]),
    "knor_set_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    "knor_set_profiling": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "knor_kernel_name": (ctypes.c_char_p, [ctypes.c_void_p, ctypes.c_int32]),
    "knor_get_profile": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Profile), ctypes.c_int32]),
    "knor_lloyd_step_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                               ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_void_p, ctypes.c_void_p]),
    "knor_test_fail_alloc": (ctypes.c_int, [ctypes.c_int32]),
    "knor_test_raise_error_flag": (ctypes.c_int, [ctypes.c_void_p]),
    "knor_probe_alu": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_float)]),
    "knor_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "knor_destroy": (None, [ctypes.c_void_p]),
    "knor_version": (ctypes.c_char_p, []),
    "knor_batch_create": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(ctypes.c_void_p),
                                         ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32),
                                         ctypes.POINTER(ctypes.c_int32), ctypes.c_uint64, ctypes.POINTER(Opts),
                                         ctypes.POINTER(ctypes.c_void_p)]),
    "knor_batch_set_init_centroids": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    "knor_batch_reset": (ctypes.c_int, [ctypes.c_void_p]),
    "knor_batch_iterate": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(IterStats)]),
    "knor_batch_run": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(IterStats)]),
    "knor_batch_get_assignments": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    "knor_batch_get_centroids": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    "knor_batch_get_centroids_f32": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    "knor_batch_get_init_indices": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    "knor_batch_get_instance": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(BatchInstance)]),
    "knor_batch_get_work": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
                                           ctypes.POINTER(ctypes.c_int64)]),
    "knor_batch_set_profiling": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "knor_batch_get_profile": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Profile), ctypes.c_int32]),
    "knor_batch_kernel_name": (ctypes.c_char_p, [ctypes.c_void_p, ctypes.c_int32]),
    "knor_batch_describe": (ctypes.c_char_p, [ctypes.c_void_p]),
    "knor_batch_stream": (ctypes.c_void_p, [ctypes.c_void_p]),
    "knor_batch_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "knor_batch_destroy": (None, [ctypes.c_void_p]),
}


def load(path: str | None = None):
    """Loads libknor.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is not built; run paper_1606_08905_gb300.build.build() "
                           "(or __graft_entry__.build()) first")
    lib = ctypes.CDLL(p)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(st: int, ctx=None):
    if st != KNOR_OK:
        msg = load().knor_last_error(ctx)
        raise KnorError(st, msg.decode() if msg else "")


def _ptr(obj, dtype):
    """(pointer, keepalive) for a torch tensor or numpy array of `dtype`."""
    try:
        import torch
        if isinstance(obj, torch.Tensor):
            want = {np.float32: torch.float32, np.float64: torch.float64, np.int32: torch.int32,
                    np.int64: torch.int64}[dtype]
            if obj.dtype != want:
                raise TypeError(f"expected {want}, got {obj.dtype}")
            if not obj.is_contiguous():
                raise ValueError("tensor must be contiguous")
            return obj.data_ptr(), obj
    except ImportError:
        pass
    arr = np.ascontiguousarray(obj, dtype=dtype)
    return arr.ctypes.data, arr


class Context:
    """One k-means problem on the GPU (a knor_ctx)."""

    def __init__(self, points, k: int, init: str = "forgy", seed: int = 0, prune: bool = True,
                 precision: str = "fp32", full_recompute_every: int = 0,
                 debug_invariants: bool = False, elkan: bool = False, points_in_host: bool = False):
        lib = load()
        shape = tuple(points.shape)
        if len(shape) != 2:
            raise ValueError("points must be n x d")
        self.n, self.d = int(shape[0]), int(shape[1])
        self.k = int(k)
        ptr, keep = _ptr(points, np.float32)
        opts = Opts(0 if prune else 1, PRECISIONS[precision], int(full_recompute_every),
                    1 if debug_invariants else 0, 1 if elkan else 0, 1 if points_in_host else 0)
        out = ctypes.c_void_p()
        st = lib.knor_create(ptr, self.n, self.d, self.k,
                             INITS[init],
                             int(seed) & 0xFFFFFFFFFFFFFFFF, ctypes.byref(opts), ctypes.byref(out))
        # with points_in_host the library reads the caller's buffer for the
        # context's lifetime: keep it referenced
        self._points = keep if points_in_host else None
        del keep
        _check(st, None)
        self._ctx = out.value

    # -- lifecycle
    def close(self):
        if getattr(self, "_ctx", None):
            load().knor_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def test_raise_error_flag(self):
        """Fault injection (knor_test_raise_error_flag): the next iterate or
        run reports KNOR_ERR_TIMEOUT, as after a device wait that gave up."""
        _check(load().knor_test_raise_error_flag(self._ctx), self._ctx)

    # -- iteration
    def set_init_centroids(self, C):
        ptr, keep = _ptr(C, np.float64)
        _check(load().knor_set_init_centroids(self._ctx, ptr), self._ctx)

    def reset(self):
        _check(load().knor_reset(self._ctx), self._ctx)

    def iterate(self) -> dict:
        s = IterStats()
        _check(load().knor_iterate(self._ctx, ctypes.byref(s)), self._ctx)
        return s.as_dict()

    def run(self, max_iters: int):
        recs = (IterStats * max(1, max_iters))()
        done = ctypes.c_int32(0)
        _check(load().knor_run(self._ctx, int(max_iters), ctypes.byref(done), recs), self._ctx)
        return int(done.value), [recs[i].as_dict() for i in range(done.value)]

    # -- results
    def assignments(self, out=None):
        """int32[n]; `out` may be a device tensor (filled in place)."""
        if out is None:
            out = np.empty(self.n, np.int32)
        ptr, _ = _ptr(out, np.int32)
        _check(load().knor_get_assignments(self._ctx, ptr), self._ctx)
        return out

    def centroids(self, out=None):
        if out is None:
            out = np.empty((self.k, self.d), np.float64)
        ptr, _ = _ptr(out, np.float64)
        _check(load().knor_get_centroids(self._ctx, ptr), self._ctx)
        return out

    def centroids_f32(self, out=None):
        if out is None:
            out = np.empty((self.k, self.d), np.float32)
        ptr, _ = _ptr(out, np.float32)
        _check(load().knor_get_centroids_f32(self._ctx, ptr), self._ctx)
        return out

    def init_indices(self):
        out = np.empty(self.k, np.int64)
        _check(load().knor_get_init_indices(self._ctx, out.ctypes.data), self._ctx)
        return out

    def iteration(self) -> int:
        v = ctypes.c_int32(0)
        _check(load().knor_get_iteration(self._ctx, ctypes.byref(v)), self._ctx)
        return int(v.value)

    def kernel_name(self, kernel: str) -> str:
        """The CUDA kernel behind 'dense', 'mti', 'reduce' or 'table'."""
        return load().knor_kernel_name(self._ctx, KERNELS.index(kernel)).decode()

    def set_profiling(self, on: bool):
        _check(load().knor_set_profiling(self._ctx, 1 if on else 0), self._ctx)

    def profile(self, reset: bool = False) -> dict:
        """{kernel: (launches, summed CUDA-event ms)} since the last reset."""
        pr = Profile()
        _check(load().knor_get_profile(self._ctx, ctypes.byref(pr), 1 if reset else 0), self._ctx)
        return {name: (int(pr.launches[i]), float(pr.ms[i])) for i, name in enumerate(KERNELS)}

    @property
    def stream(self) -> int:
        return int(load().knor_stream(self._ctx) or 0)

    # -- checkpoint
    def get_state(self) -> bytes:
        size = ctypes.c_size_t(0)
        _check(load().knor_get_state(self._ctx, None, ctypes.byref(size)), self._ctx)
        buf = ctypes.create_string_buffer(size.value)
        _check(load().knor_get_state(self._ctx, buf, ctypes.byref(size)), self._ctx)
        return buf.raw

    def set_state(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check(load().knor_set_state(self._ctx, buf, len(blob)), self._ctx)


def _bcheck(st: int, b):
    if st != KNOR_OK:
        msg = load().knor_batch_last_error(b) if b else load().knor_last_error(None)
        raise KnorError(st, msg.decode() if msg else "")


class Batch:
    """m independent k-means problems advanced together (a knor_batch).

    `points` is a list of n_i x d_i FP32 arrays or tensors (host or device),
    `k` a list of cluster counts; instance i starts from Forgy with seed + i.
    """

    def __init__(self, points, k, seed: int = 0, prune: bool = True):
        lib = load()
        m = len(points)
        if len(k) != m:
            raise ValueError("one k per instance")
        keep = []
        ptrs = (ctypes.c_void_p * m)()
        ns = (ctypes.c_int64 * m)()
        ds = (ctypes.c_int32 * m)()
        ks = (ctypes.c_int32 * m)()
        self.shapes = []
        for i, X in enumerate(points):
            shape = tuple(X.shape)
            if len(shape) != 2:
                raise ValueError("points must be n x d")
            ptr, kp = _ptr(X, np.float32)
            keep.append(kp)
            ptrs[i] = ptr
            ns[i], ds[i], ks[i] = int(shape[0]), int(shape[1]), int(k[i])
            self.shapes.append((int(shape[0]), int(shape[1]), int(k[i])))
        opts = Opts(0 if prune else 1, 0, 0, 0)
        out = ctypes.c_void_p()
        st = lib.knor_batch_create(m, ptrs, ns, ds, ks, int(seed) & 0xFFFFFFFFFFFFFFFF, ctypes.byref(opts),
                                   ctypes.byref(out))
        del keep
        _bcheck(st, None)
        self._b = out.value
        self.m = m

    def close(self):
        if getattr(self, "_b", None):
            load().knor_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_init_centroids(self, i: int, C):
        ptr, keep = _ptr(C, np.float64)
        _bcheck(load().knor_batch_set_init_centroids(self._b, int(i), ptr), self._b)

    def reset(self):
        _bcheck(load().knor_batch_reset(self._b), self._b)

    def iterate(self) -> dict:
        s = IterStats()
        _bcheck(load().knor_batch_iterate(self._b, ctypes.byref(s)), self._b)
        return s.as_dict()

    def run(self, max_iters: int):
        recs = (IterStats * max(1, max_iters))()
        done = ctypes.c_int32(0)
        _bcheck(load().knor_batch_run(self._b, int(max_iters), ctypes.byref(done), recs), self._b)
        return int(done.value), [recs[i].as_dict() for i in range(done.value)]

    def assignments(self, i: int, out=None):
        if out is None:
            out = np.empty(self.shapes[i][0], np.int32)
        ptr, _ = _ptr(out, np.int32)
        _bcheck(load().knor_batch_get_assignments(self._b, int(i), ptr), self._b)
        return out

    def centroids(self, i: int):
        n, d, k = self.shapes[i]
        out = np.empty((k, d), np.float64)
        _bcheck(load().knor_batch_get_centroids(self._b, int(i), out.ctypes.data), self._b)
        return out

    def centroids_f32(self, i: int):
        n, d, k = self.shapes[i]
        out = np.empty((k, d), np.float32)
        _bcheck(load().knor_batch_get_centroids_f32(self._b, int(i), out.ctypes.data), self._b)
        return out

    def init_indices(self, i: int):
        out = np.empty(self.shapes[i][2], np.int64)
        _bcheck(load().knor_batch_get_init_indices(self._b, int(i), out.ctypes.data), self._b)
        return out

    def instance(self, i: int) -> dict:
        r = BatchInstance()
        _bcheck(load().knor_batch_get_instance(self._b, int(i), ctypes.byref(r)), self._b)
        return r.as_dict()

    def work(self):
        """(point-iterations, scan algorithmic bytes) since the last reset."""
        pi, by = ctypes.c_int64(0), ctypes.c_int64(0)
        _bcheck(load().knor_batch_get_work(self._b, ctypes.byref(pi), ctypes.byref(by)), self._b)
        return int(pi.value), int(by.value)

    def set_profiling(self, on: bool):
        _bcheck(load().knor_batch_set_profiling(self._b, 1 if on else 0), self._b)

    def profile(self, reset: bool = False) -> dict:
        pr = Profile()
        _bcheck(load().knor_batch_get_profile(self._b, ctypes.byref(pr), 1 if reset else 0), self._b)
        return {name: (int(pr.launches[i]), float(pr.ms[i])) for i, name in enumerate(KERNELS)}

    def kernel_name(self, kernel: str) -> str:
        return load().knor_batch_kernel_name(self._b, KERNELS.index(kernel)).decode()

    def describe(self) -> str:
        return load().knor_batch_describe(self._b).decode()

    @property
    def stream(self) -> int:
        return int(load().knor_batch_stream(self._b) or 0)


def lloyd_step_noalloc(points, centroids, assign_out, sums_out, counts_out, stream: int = 0):
    """One plain Lloyd step on caller-owned device tensors with no device
    allocation (knor_lloyd_step_noalloc): points n x d FP32, centroids k x d
    FP32; fills assign_out (n int32), sums_out (k x d FP64) and counts_out
    (k int64).  For callers that cannot allocate device memory; all tensors
    must be CUDA tensors on one device.  The C ABI cannot see buffer sizes,
    so every shape is checked here, before anything is launched."""
    import torch
    bufs = {"points": points, "centroids": centroids, "assign_out": assign_out, "sums_out": sums_out,
            "counts_out": counts_out}
    for name, t in bufs.items():
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise ValueError(f"lloyd_step_noalloc: {name} must be a CUDA tensor")
    dev = points.device
    for name, t in bufs.items():
        if t.device != dev:
            raise ValueError(f"lloyd_step_noalloc: {name} is on {t.device}, points on {dev}")
    if points.dim() != 2 or centroids.dim() != 2:
        raise ValueError("lloyd_step_noalloc: points and centroids must be 2-D")
    n, d = int(points.shape[0]), int(points.shape[1])
    k = int(centroids.shape[0])
    if int(centroids.shape[1]) != d:
        raise ValueError(f"lloyd_step_noalloc: centroids are {tuple(centroids.shape)}, points have d = {d}")
    if assign_out.numel() < n:
        raise ValueError(f"lloyd_step_noalloc: assign_out holds {assign_out.numel()} < n = {n} entries")
    if sums_out.numel() < k * d:
        raise ValueError(f"lloyd_step_noalloc: sums_out holds {sums_out.numel()} < k * d = {k * d} entries")
    if counts_out.numel() < k:
        raise ValueError(f"lloyd_step_noalloc: counts_out holds {counts_out.numel()} < k = {k} entries")
    p0, _ = _ptr(points, np.float32)
    p1, _ = _ptr(centroids, np.float32)
    p2, _ = _ptr(assign_out, np.int32)
    p3, _ = _ptr(sums_out, np.float64)
    p4, _ = _ptr(counts_out, np.int64)
    with torch.cuda.device(dev):
        _check(load().knor_lloyd_step_noalloc(p0, n, d, k, p1, p2, p3, p4, stream or None), None)


def test_fail_alloc(after: int):
    """Fault injection (knor_test_fail_alloc): the device allocation after
    `after` more successful ones fails with KNOR_ERR_OOM; after < 0 cancels."""
    _check(load().knor_test_fail_alloc(int(after)), None)


def probe_alu(kind: str) -> tuple[float, float]:
    """Measured FMA throughput of the current GPU (knor_probe_alu): kind
    'fp32', 'fp32x2' (packed) or 'fp64'.  Returns (TFLOP/s, ms of the timed
    kernel)."""
    tf, ms = ctypes.c_double(0.0), ctypes.c_float(0.0)
    _check(load().knor_probe_alu({"fp32": 0, "fp32x2": 1, "fp64": 2}[kind], ctypes.byref(tf), ctypes.byref(ms)),
           None)
    return float(tf.value), float(ms.value)


def version() -> str:
    return load().knor_version().decode()
