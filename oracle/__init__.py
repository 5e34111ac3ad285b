"""FP64 CPU oracle for Lloyd's k-means with MTI pruning (test infrastructure).

This package is TEST INFRASTRUCTURE.  Only the test suite, the smoke check in
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import it.  The
library under test never imports it, and it never imports the library: the
two share no code.  Its arithmetic lives in ``knor_oracle.c`` (plain C, FP64,
OpenMP); this module only compiles that file and marshals numpy arrays.

Paper sections followed (Mhembere et al., HPDC'17, arXiv 1606.08905):
"Nomenclature" (distance, drift), "Parallel Lloyd's Algorithm" with
Algorithm 1 (assignment with lowest-index ties, means), and "Minimal Triangle
Inequality (MTI) Pruning" (Clauses 1-3).  The readings taken where the paper
is silent are listed at the top of ``knor_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "knor_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_knor.so")
_lock = threading.Lock()
_lib = None

_f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


def build(force: bool = False, out: str | None = None, defines=()) -> str:
    """Compile knor_oracle.c into liboracle_knor.so next to it (gcc, OpenMP).
    `out`/`defines` build a variant elsewhere (the planted-mistake test)."""
    target = out or _LIB
    if (not force and not defines and os.path.exists(target)
            and os.path.getmtime(target) >= os.path.getmtime(_SRC)):
        return target
    tmp = target + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC"]
    cmd += [f"-D{d}" for d in defines]
    cmd += [_SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, target)
    return target


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = os.environ.get("KNOR_ORACLE_LIB") or build()
        lib = ctypes.CDLL(path)
        c = ctypes
        lib.oracle_splitmix64_next.argtypes = [c.POINTER(c.c_uint64)]
        lib.oracle_splitmix64_next.restype = c.c_uint64
        lib.oracle_forgy_indices.argtypes = [c.c_int64, c.c_int32, c.c_uint64, _i64p]
        lib.oracle_kmeanspp_indices.argtypes = [_f32p, c.c_int64, c.c_int32, c.c_int32, c.c_uint64, _i64p]
        lib.oracle_kmeanspp_indices.restype = c.c_int
        lib.oracle_forgy_indices.restype = c.c_int
        lib.oracle_assign.argtypes = [_f32p, c.c_int64, c.c_int32, c.c_int32, _f64p,
                                      _i32p, _f64p, _f64p, _f64p, c.c_int]
        lib.oracle_assign.restype = None
        lib.oracle_means.argtypes = [_f32p, c.c_int64, c.c_int32, c.c_int32, _i32p, _f64p,
                                     _f64p, _i64p]
        lib.oracle_means.restype = None
        lib.oracle_objective.argtypes = [_f32p, c.c_int64, c.c_int32, _f64p, _i32p]
        lib.oracle_objective.restype = c.c_double
        lib.oracle_mti_tables.argtypes = [_f64p, c.c_void_p, c.c_int32, c.c_int32, _f64p,
                                          _f64p, _f64p]
        lib.oracle_mti_tables.restype = None
        lib.oracle_mti_iter.argtypes = [_f32p, c.c_int64, c.c_int32, c.c_int32, _f64p, _f64p,
                                        _f64p, _f64p, _i32p, _f64p, c.POINTER(c.c_int64),
                                        c.POINTER(c.c_int64), c.c_int]
        lib.oracle_mti_iter.restype = c.c_int64
        lib.oracle_run.argtypes = [_f32p, c.c_int64, c.c_int32, c.c_int32, _f64p, c.c_int32,
                                   c.c_int, _f64p, _i32p, c.c_void_p, c.c_void_p, c.c_void_p,
                                   c.c_void_p, c.c_void_p, c.c_void_p, c.c_int]
        lib.oracle_run.restype = c.c_int
        lib.oracle_assign_f32.argtypes = [_f32p, c.c_int64, c.c_int32, c.c_int32, _f32p, _i32p,
                                          c.c_int]
        lib.oracle_assign_f32.restype = None
        lib.oracle_max_threads.argtypes = []
        lib.oracle_max_threads.restype = c.c_int
        _lib = lib
        return lib


def _X(X):
    X = np.ascontiguousarray(X, dtype=np.float32)
    if X.ndim != 2:
        raise ValueError("X must be n x d")
    return X


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def splitmix64(seed: int, count: int) -> np.ndarray:
    """The first `count` SplitMix64 outputs from state `seed`."""
    lib = _load()
    st = ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF)
    return np.array([lib.oracle_splitmix64_next(ctypes.byref(st)) for _ in range(count)],
                    dtype=np.uint64)


def forgy_indices(n: int, k: int, seed: int) -> np.ndarray:
    """k distinct indices of [0, n) by Floyd's algorithm on SplitMix64(seed)."""
    out = np.zeros(k, dtype=np.int64)
    if _load().oracle_forgy_indices(n, k, seed & 0xFFFFFFFFFFFFFFFF, out) != 0:
        raise ValueError("forgy_indices: need 1 <= k <= n")
    return out


def forgy_centroids(X, k: int, seed: int) -> np.ndarray:
    X = _X(X)
    idx = forgy_indices(X.shape[0], k, seed)
    return X[idx].astype(np.float64)


def kmeanspp_indices(X, k: int, seed: int) -> np.ndarray:
    """k-means++ seeding (D^2 sampling, reproducible readings in
    knor_oracle.c): the k row indices in the order drawn."""
    X = _X(X)
    n, d = X.shape
    out = np.zeros(k, np.int64)
    if _load().oracle_kmeanspp_indices(X, n, d, k, seed & 0xFFFFFFFFFFFFFFFF, out) != 0:
        raise ValueError("kmeanspp_indices: need 1 <= k <= n")
    return out


def assign(X, C, nthreads: int = 0):
    """Phase I: (a, d1, d2, scale) with d1 <= d2 the two smallest squared
    distances and scale = ||x||^2 + ||c_a||^2, all FP64."""
    X = _X(X)
    n, d = X.shape
    C = np.ascontiguousarray(C, dtype=np.float64)
    k = C.shape[0]
    a = np.zeros(n, np.int32)
    d1 = np.zeros(n, np.float64)
    d2 = np.zeros(n, np.float64)
    sc = np.zeros(n, np.float64)
    _load().oracle_assign(X, n, d, k, C, a, d1, d2, sc, nthreads)
    return a, d1, d2, sc


def assign_f32(X, C32, nthreads: int = 0) -> np.ndarray:
    """The argmin taken in FP32 (even/odd fmaf chains, then their sum), lowest
    index on ties."""
    X = _X(X)
    n, d = X.shape
    C32 = np.ascontiguousarray(C32, dtype=np.float32)
    a = np.zeros(n, np.int32)
    _load().oracle_assign_f32(X, n, d, C32.shape[0], C32, a, nthreads)
    return a


def means(X, a, C_prev):
    """Phase II: (C, counts); empty clusters keep C_prev."""
    X = _X(X)
    n, d = X.shape
    C_prev = np.ascontiguousarray(C_prev, dtype=np.float64)
    k = C_prev.shape[0]
    a = np.ascontiguousarray(a, dtype=np.int32)
    if a.size and (a.min() < 0 or a.max() >= k):
        raise ValueError("assignment out of range")
    C = np.zeros((k, d), np.float64)
    cnt = np.zeros(k, np.int64)
    _load().oracle_means(X, n, d, k, a, C_prev, C, cnt)
    return C, cnt


def objective(X, C, a) -> float:
    X = _X(X)
    n, d = X.shape
    return float(_load().oracle_objective(X, n, d, np.ascontiguousarray(C, dtype=np.float64),
                                          np.ascontiguousarray(a, dtype=np.int32)))


def mti_tables(C, C_prev=None):
    """(halfD, s, f): lower bounds on 1/2 d(c_a, c), their row minima over
    c != a, and upper bounds on the drift d(c^t, c^{t-1})."""
    C = np.ascontiguousarray(C, dtype=np.float64)
    k, d = C.shape
    halfD = np.zeros((k, k), np.float64)
    s = np.zeros(k, np.float64)
    f = np.zeros(k, np.float64)
    prev = None
    if C_prev is not None:
        prev = np.ascontiguousarray(C_prev, dtype=np.float64)
    _load().oracle_mti_tables(C, prev.ctypes.data if prev is not None else None, d, k,
                              halfD, s, f)
    return halfD, s, f


def mti_iter(X, C, halfD, s, f, a, u, nthreads: int = 0):
    """One MTI iteration; a and u (int32 / float64 arrays) are updated in place.
    Returns (changed, skipped_by_clause1, distance_evaluations)."""
    X = _X(X)
    n, d = X.shape
    sk = ctypes.c_int64(0)
    ev = ctypes.c_int64(0)
    ch = _load().oracle_mti_iter(X, n, d, C.shape[0], np.ascontiguousarray(C, np.float64),
                                 np.ascontiguousarray(halfD, np.float64),
                                 np.ascontiguousarray(s, np.float64),
                                 np.ascontiguousarray(f, np.float64), a, u,
                                 ctypes.byref(sk), ctypes.byref(ev), nthreads)
    return int(ch), int(sk.value), int(ev.value)


class RunResult:
    def __init__(self, **kw):
        self.__dict__.update(kw)


def run(X, C0, max_iters: int, prune, history: bool = False, nthreads: int = 0,
        check_bounds: bool = False) -> RunResult:
    """Lloyd's algorithm from C0 (k x d) until no assignment changes or
    max_iters.  prune: False (every distance), True (MTI) or "elkan" (MTI
    plus per-centroid lower bounds; with check_bounds=True the bounds are
    checked against exact distances every iteration, result.violations).
    With history=True also returns a_hist (iters x n) and C_hist
    ((iters+1) x k x d, C^0 first)."""
    mode = 2 if prune == "elkan" else (1 if prune else 0)
    X = _X(X)
    n, d = X.shape
    C0 = np.ascontiguousarray(C0, dtype=np.float64)
    k = C0.shape[0]
    C = np.zeros((k, d), np.float64)
    a = np.zeros(n, np.int32)
    ch = np.zeros(max_iters, np.int64)
    sk = np.zeros(max_iters, np.int64)
    ev = np.zeros(max_iters, np.int64)
    ah = np.zeros((max_iters, n), np.int32) if history else None
    Ch = np.zeros((max_iters + 1, k, d), np.float64) if history else None
    vi = np.zeros(max_iters, np.int64)
    it = _load().oracle_run(X, n, d, k, C0, max_iters, mode, C, a,
                            ah.ctypes.data if history else None,
                            Ch.ctypes.data if history else None,
                            ch.ctypes.data, sk.ctypes.data, ev.ctypes.data,
                            vi.ctypes.data if check_bounds else None, nthreads)
    return RunResult(iters=int(it), C=C, a=a, changed=ch[:it].copy(), skipped=sk[:it].copy(),
                     evals=ev[:it].copy(), violations=vi[:it].copy(),
                     a_hist=ah[:it].copy() if history else None,
                     C_hist=Ch[:it + 1].copy() if history else None)


def near_tie_mask(d1, d2, scale, rel: float = 1e-6) -> np.ndarray:
    """Points whose FP64 top-2 gap is below rel * (||x||^2 + ||c||^2): the
    points the parity rule exempts from exact assignment agreement."""
    return (d2 - d1) < rel * scale
