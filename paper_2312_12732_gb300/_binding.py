"""ctypes binding of ``include/fmm.h`` (argument marshalling only).

Every function here has the name of the C entry point it wraps.  Tensors are
``torch.Tensor`` objects (float64, contiguous, square); only their data
pointers and the current CUDA stream cross the boundary.  All arithmetic runs
in the library's CUDA kernels; if ``libfmm.so`` is missing the first call
raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfmm.so")

FMM_OK, FMM_ERR_INVALID, FMM_ERR_BRENT, FMM_ERR_UNSUPPORTED = 0, 1, 2, 3
FMM_ERR_OOM, FMM_ERR_CUDA, FMM_ERR_TIMEOUT, FMM_ERR_NOT_FOUND = 4, 5, 6, 7
FMM_ERR_SCRATCH_LIMIT = 8
FMM_F64, FMM_F64_OZAKI, FMM_C128, FMM_C128_3M, FMM_F32 = 0, 1, 2, 3, 4
FMM_SCHED_AUTO, FMM_SCHED_FUSED, FMM_SCHED_HYBRID = 0, 1, 2

DTYPES = {"f64": FMM_F64, "f64_ozaki": FMM_F64_OZAKI, "c128": FMM_C128, "c128_3m": FMM_C128_3M, "f32": FMM_F32}
COMPLEX_DTYPES = ("c128", "c128_3m")
SCHEDULES = {"auto": FMM_SCHED_AUTO, "fused": FMM_SCHED_FUSED, "hybrid": FMM_SCHED_HYBRID}
POST_ADDITIONS = {"auto": 0, "fused": 1, "levels": 2}

_i32p = ctypes.POINTER(ctypes.c_int32)


class fmm_algo_t(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("R", ctypes.c_int), ("U", _i32p), ("V", _i32p), ("W", _i32p)]


class fmm_algo_rect_t(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("k", ctypes.c_int), ("n", ctypes.c_int), ("R", ctypes.c_int), ("U", _i32p),
                ("V", _i32p), ("W", _i32p)]


class fmm_algo_rational_t(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("R", ctypes.c_int), ("U", _i32p), ("V", _i32p), ("W", _i32p),
                ("den_u", ctypes.c_int32), ("den_v", ctypes.c_int32), ("den_w", ctypes.c_int32)]


class fmm_plan_options_t(ctypes.Structure):
    _fields_ = [("schedule", ctypes.c_int), ("materialize_levels", ctypes.c_int), ("ozaki_slices", ctypes.c_int),
                ("wait_timeout_s", ctypes.c_double), ("debug_poison_chain", ctypes.c_int),
                ("record_kernel_time", ctypes.c_int), ("tile_n", ctypes.c_int), ("shard_count", ctypes.c_int),
                ("shard_index", ctypes.c_int), ("post_additions", ctypes.c_int)]


class fmm_plan_info_t(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("p", ctypes.c_int), ("depth", ctypes.c_int), ("P", ctypes.c_int64),
                ("R_total", ctypes.c_int64), ("m", ctypes.c_int64), ("n_core", ctypes.c_int64),
                ("tasks", ctypes.c_int64), ("materialized_levels", ctypes.c_int),
                ("flops_leaf", ctypes.c_double), ("flops_executed", ctypes.c_double),
                ("workspace_bytes", ctypes.c_size_t), ("ozaki_slices", ctypes.c_int), ("flops_lowp", ctypes.c_double),
                ("tile_n", ctypes.c_int), ("materialize_passes", ctypes.c_int), ("coef_scale", ctypes.c_double),
                ("product_begin", ctypes.c_int64), ("product_end", ctypes.c_int64), ("post_passes", ctypes.c_int)]


# (name, restype, argtypes) for every symbol declared in include/fmm.h.
SIGNATURES = [
    ("fmm_status_string", ctypes.c_char_p, [ctypes.c_int]),
    ("fmm_shard_range", ctypes.c_int, [ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                       ctypes.POINTER(ctypes.c_int64)]),
    ("fmm_algo_builtin", ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(fmm_algo_t)]),
    ("fmm_algo_brent_mismatches", ctypes.c_int64, [ctypes.POINTER(fmm_algo_t)]),
    ("fmm_algo_from_transposed_c", ctypes.c_int, [ctypes.c_int, ctypes.c_int, _i32p, _i32p]),
    ("fmm_algo_compose", ctypes.c_int, [ctypes.POINTER(fmm_algo_t), ctypes.POINTER(fmm_algo_t), _i32p, _i32p, _i32p,
                                        ctypes.POINTER(fmm_algo_t)]),
    ("fmm_plan_create", ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int64, ctypes.POINTER(fmm_algo_t),
                                       ctypes.c_int, ctypes.c_int]),
    ("fmm_plan_create_ex", ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int64,
                                          ctypes.POINTER(fmm_algo_t), ctypes.c_int, ctypes.c_int,
                                          ctypes.POINTER(fmm_plan_options_t)]),
    ("fmm_algo_rational_brent_mismatches", ctypes.c_int64, [ctypes.POINTER(fmm_algo_rational_t)]),
    ("fmm_algo_rect_brent_mismatches", ctypes.c_int64, [ctypes.POINTER(fmm_algo_rect_t)]),
    ("fmm_algo_rect_builtin", ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(fmm_algo_rect_t)]),
    ("fmm_algo_rect_classic", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _i32p, _i32p, _i32p,
                                             ctypes.POINTER(fmm_algo_rect_t)]),
    ("fmm_algo_rect_transpose", ctypes.c_int, [ctypes.POINTER(fmm_algo_rect_t), _i32p, _i32p, _i32p,
                                               ctypes.POINTER(fmm_algo_rect_t)]),
    ("fmm_algo_rect_cyclic", ctypes.c_int, [ctypes.POINTER(fmm_algo_rect_t), _i32p, _i32p, _i32p,
                                            ctypes.POINTER(fmm_algo_rect_t)]),
    ("fmm_algo_rect_compose", ctypes.c_int, [ctypes.POINTER(fmm_algo_rect_t), ctypes.POINTER(fmm_algo_rect_t), _i32p,
                                             _i32p, _i32p, ctypes.POINTER(fmm_algo_rect_t)]),
    ("fmm_algo_rect_as_square", ctypes.c_int, [ctypes.POINTER(fmm_algo_rect_t), ctypes.POINTER(fmm_algo_t)]),
    ("fmm_plan_create_rational", ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int64,
                                                ctypes.POINTER(fmm_algo_rational_t), ctypes.c_int, ctypes.c_int,
                                                ctypes.POINTER(fmm_plan_options_t)]),
    ("fmm_gemm", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                ctypes.c_void_p]),
    ("fmm_gemm_ex", ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]),
    ("fmm_gemm_batched_ex", ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                           ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_void_p),
                                           ctypes.c_int, ctypes.c_void_p]),
    ("fmm_gemm_f32_ex", ctypes.c_int, [ctypes.c_void_p, ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p]),
    ("fmm_gemm_host", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p]),
    ("fmm_gemm_batched", ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                        ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                        ctypes.c_int, ctypes.c_void_p]),
    ("fmm_sync_status", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("fmm_batch_graph_create", ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                              ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                              ctypes.POINTER(ctypes.c_void_p), ctypes.c_int]),
    ("fmm_batch_graph_launch", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("fmm_batch_graph_destroy", None, [ctypes.c_void_p]),
    ("fmm_autotune", ctypes.c_int, [ctypes.c_int64, ctypes.POINTER(ctypes.POINTER(fmm_algo_t)), ctypes.c_int,
                                    ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    ("fmm_plan_last_kernel_ms", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float),
                                               ctypes.POINTER(ctypes.c_float)]),
    ("fmm_measure_fp64_peak", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                             ctypes.POINTER(ctypes.c_double)]),
    ("fmm_gemm_noalloc", ctypes.c_int, [ctypes.c_int64, ctypes.POINTER(fmm_algo_t), ctypes.c_int, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("fmm_measure_e4m3_peak", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    ("fmm_noalloc_sync_status", ctypes.c_int, [ctypes.c_void_p]),
    ("fmm_host_alloc", ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_size_t]),
    ("fmm_host_free", ctypes.c_int, [ctypes.c_void_p]),
    ("fmm_host_huge_page_bytes", ctypes.c_int64, []),
    ("fmm_debug_fail_allocation", None, [ctypes.c_int64]),
    ("fmm_debug_live_allocations", ctypes.c_int64, []),
    ("fmm_noalloc_set_debug", ctypes.c_int, [ctypes.c_double, ctypes.c_int]),
    ("fmm_plan_last_phase_ms", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float), ctypes.c_int]),
    ("fmm_plan_get_info", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(fmm_plan_info_t)]),
    ("fmm_plan_workspace_bytes", ctypes.c_size_t, [ctypes.c_void_p]),
    ("fmm_plan_destroy", None, [ctypes.c_void_p]),
]

_lib = None


def lib():
    """The loaded ``libfmm.so`` (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; "
                               "g.build()'` (the library has no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class FmmError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {fmm_status_string(status)} (status {status})")


def _check(status: int, what: str):
    if status != FMM_OK:
        raise FmmError(status, what)


def fmm_status_string(status: int) -> str:
    return lib().fmm_status_string(int(status)).decode()


def fmm_shard_range(units: int, shard_count: int, shard_index: int) -> tuple[int, int]:
    """[begin, end) of `units` work units taken by shard `shard_index` of `shard_count` (host only)."""
    b, e = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().fmm_shard_range(int(units), int(shard_count), int(shard_index), ctypes.byref(b), ctypes.byref(e)),
           "fmm_shard_range")
    return int(b.value), int(e.value)


class Algo:
    """An algorithm <p,p,p;R>; keeps its int32 tables alive for the C struct."""

    def __init__(self, p: int, U, V, W, name: str = "custom"):
        self.p = int(p)
        self.U = np.ascontiguousarray(U, dtype=np.int32)
        self.V = np.ascontiguousarray(V, dtype=np.int32)
        self.W = np.ascontiguousarray(W, dtype=np.int32)
        if not (self.U.shape == self.V.shape == self.W.shape and self.U.ndim == 2
                and self.U.shape[0] == self.p * self.p):
            raise ValueError("U, V, W must all be p^2 x R")
        self.R = int(self.U.shape[1])
        self.name = name

    def c_struct(self) -> fmm_algo_t:
        return fmm_algo_t(self.p, self.R, self.U.ctypes.data_as(_i32p), self.V.ctypes.data_as(_i32p),
                          self.W.ctypes.data_as(_i32p))

    def __repr__(self):
        return f"Algo({self.name}, <{self.p},{self.p},{self.p};{self.R}>)"


class RationalAlgo:
    """An algorithm <p,p,p;R> with coefficients U / den_u, V / den_v, W / den_w (int32 numerators,
    one positive denominator per matrix); keeps the numerator tables alive for the C struct."""

    def __init__(self, p: int, U, V, W, dens, name: str = "rational"):
        self.p = int(p)
        self.U = np.ascontiguousarray(U, dtype=np.int32)
        self.V = np.ascontiguousarray(V, dtype=np.int32)
        self.W = np.ascontiguousarray(W, dtype=np.int32)
        if not (self.U.shape == self.V.shape == self.W.shape and self.U.ndim == 2
                and self.U.shape[0] == self.p * self.p):
            raise ValueError("U, V, W must all be p^2 x R")
        self.R = int(self.U.shape[1])
        self.dens = tuple(int(d) for d in dens)
        if len(self.dens) != 3:
            raise ValueError("dens must be (den_u, den_v, den_w)")
        self.name = name

    def c_struct(self) -> fmm_algo_rational_t:
        return fmm_algo_rational_t(self.p, self.R, self.U.ctypes.data_as(_i32p), self.V.ctypes.data_as(_i32p),
                                   self.W.ctypes.data_as(_i32p), *self.dens)

    def __repr__(self):
        return f"RationalAlgo({self.name}, <{self.p},{self.p},{self.p};{self.R}>, dens={self.dens})"


class RectAlgo:
    """A rectangular algorithm <m,k,n;R> (U over A's m x k block grid, V over B's k x n grid, W over
    C's m x n grid, row-major); keeps its int32 tables alive for the C struct."""

    def __init__(self, m: int, k: int, n: int, U, V, W, name: str = "rect"):
        self.m, self.k, self.n = int(m), int(k), int(n)
        self.U = np.ascontiguousarray(U, dtype=np.int32)
        self.V = np.ascontiguousarray(V, dtype=np.int32)
        self.W = np.ascontiguousarray(W, dtype=np.int32)
        R = self.U.shape[1] if self.U.ndim == 2 else -1
        if not (self.U.shape == (self.m * self.k, R) and self.V.shape == (self.k * self.n, R)
                and self.W.shape == (self.m * self.n, R)):
            raise ValueError("U, V, W must be (m k) x R, (k n) x R and (m n) x R")
        self.R = int(R)
        self.name = name

    def c_struct(self) -> fmm_algo_rect_t:
        return fmm_algo_rect_t(self.m, self.k, self.n, self.R, self.U.ctypes.data_as(_i32p),
                               self.V.ctypes.data_as(_i32p), self.W.ctypes.data_as(_i32p))

    def __repr__(self):
        return f"RectAlgo({self.name}, <{self.m},{self.k},{self.n};{self.R}>)"


def _rect_from(out: fmm_algo_rect_t, name: str) -> RectAlgo:
    m, k, n, R = out.m, out.k, out.n, out.R
    U = np.ctypeslib.as_array(out.U, shape=(m * k * R,)).reshape(m * k, R).copy()
    V = np.ctypeslib.as_array(out.V, shape=(k * n * R,)).reshape(k * n, R).copy()
    W = np.ctypeslib.as_array(out.W, shape=(m * n * R,)).reshape(m * n, R).copy()
    return RectAlgo(m, k, n, U, V, W, name=name)


def fmm_algo_rect_builtin(name: str) -> RectAlgo:
    out = fmm_algo_rect_t()
    _check(lib().fmm_algo_rect_builtin(name.encode(), ctypes.byref(out)), f"fmm_algo_rect_builtin({name!r})")
    return _rect_from(out, name)


def fmm_algo_rect_classic(m: int, k: int, n: int) -> RectAlgo:
    R = m * k * n
    U = np.empty((m * k, R), dtype=np.int32)
    V = np.empty((k * n, R), dtype=np.int32)
    W = np.empty((m * n, R), dtype=np.int32)
    out = fmm_algo_rect_t()
    _check(lib().fmm_algo_rect_classic(m, k, n, U.ctypes.data_as(_i32p), V.ctypes.data_as(_i32p),
                                       W.ctypes.data_as(_i32p), ctypes.byref(out)), "fmm_algo_rect_classic")
    return RectAlgo(m, k, n, U, V, W, name=f"classic_{m}x{k}x{n}")


def fmm_algo_rect_brent_mismatches(algo: RectAlgo) -> int:
    a = algo.c_struct()
    return int(lib().fmm_algo_rect_brent_mismatches(ctypes.byref(a)))


def _rect_unary(fn, algo: RectAlgo, sizes, tag: str) -> RectAlgo:
    U = np.empty(sizes[0], dtype=np.int32)
    V = np.empty(sizes[1], dtype=np.int32)
    W = np.empty(sizes[2], dtype=np.int32)
    a, out = algo.c_struct(), fmm_algo_rect_t()
    _check(fn(ctypes.byref(a), U.ctypes.data_as(_i32p), V.ctypes.data_as(_i32p), W.ctypes.data_as(_i32p),
              ctypes.byref(out)), tag)
    return RectAlgo(out.m, out.k, out.n, U.reshape(out.m * out.k, out.R), V.reshape(out.k * out.n, out.R),
                    W.reshape(out.m * out.n, out.R), name=f"{tag}({algo.name})")


def fmm_algo_rect_transpose(algo: RectAlgo) -> RectAlgo:
    """<n,k,m> from (A B)^T = B^T A^T."""
    m, k, n, R = algo.m, algo.k, algo.n, algo.R
    return _rect_unary(lib().fmm_algo_rect_transpose, algo, (n * k * R, k * m * R, n * m * R), "transpose")


def fmm_algo_rect_cyclic(algo: RectAlgo) -> RectAlgo:
    """<k,n,m> from the rotation of the trilinear form."""
    m, k, n, R = algo.m, algo.k, algo.n, algo.R
    return _rect_unary(lib().fmm_algo_rect_cyclic, algo, (k * n * R, n * m * R, k * m * R), "cyclic")


def fmm_algo_rect_compose(first: RectAlgo, second: RectAlgo) -> RectAlgo:
    """<m1 m2, k1 k2, n1 n2; R1 R2>, the first factor outermost."""
    m, k, n, R = first.m * second.m, first.k * second.k, first.n * second.n, first.R * second.R
    U = np.empty((m * k, R), dtype=np.int32)
    V = np.empty((k * n, R), dtype=np.int32)
    W = np.empty((m * n, R), dtype=np.int32)
    a1, a2, out = first.c_struct(), second.c_struct(), fmm_algo_rect_t()
    _check(lib().fmm_algo_rect_compose(ctypes.byref(a1), ctypes.byref(a2), U.ctypes.data_as(_i32p),
                                       V.ctypes.data_as(_i32p), W.ctypes.data_as(_i32p), ctypes.byref(out)),
           "fmm_algo_rect_compose")
    return RectAlgo(m, k, n, U, V, W, name=f"{first.name}x{second.name}")


def fmm_algo_rect_as_square(algo: RectAlgo) -> Algo:
    """The square algorithm <p,p,p;R> of a rectangular one with m = k = n (plans take square ones)."""
    a, out = algo.c_struct(), fmm_algo_t()
    _check(lib().fmm_algo_rect_as_square(ctypes.byref(a), ctypes.byref(out)), "fmm_algo_rect_as_square")
    return Algo(algo.m, algo.U, algo.V, algo.W, name=algo.name)


def fmm_algo_rational_brent_mismatches(algo: RationalAlgo) -> int:
    a = algo.c_struct()
    return int(lib().fmm_algo_rational_brent_mismatches(ctypes.byref(a)))


def fmm_algo_builtin(name: str) -> Algo:
    a = fmm_algo_t()
    _check(lib().fmm_algo_builtin(name.encode(), ctypes.byref(a)), f"fmm_algo_builtin({name!r})")
    p, R = a.p, a.R
    U = np.ctypeslib.as_array(a.U, shape=(p * p * R,)).reshape(p * p, R).copy()
    V = np.ctypeslib.as_array(a.V, shape=(p * p * R,)).reshape(p * p, R).copy()
    W = np.ctypeslib.as_array(a.W, shape=(p * p * R,)).reshape(p * p, R).copy()
    return Algo(p, U, V, W, name=name)


def fmm_algo_brent_mismatches(algo: Algo) -> int:
    a = algo.c_struct()
    return int(lib().fmm_algo_brent_mismatches(ctypes.byref(a)))


def fmm_algo_from_transposed_c(p: int, ct) -> np.ndarray:
    ct = np.ascontiguousarray(ct, dtype=np.int32)
    R = ct.shape[1]
    W = np.empty_like(ct)
    _check(lib().fmm_algo_from_transposed_c(p, R, ct.ctypes.data_as(_i32p), W.ctypes.data_as(_i32p)),
           "fmm_algo_from_transposed_c")
    return W


def fmm_algo_compose(first: Algo, second: Algo) -> Algo:
    p = first.p * second.p
    R = first.R * second.R
    U = np.empty((p * p, R), dtype=np.int32)
    V = np.empty_like(U)
    W = np.empty_like(U)
    a1, a2, out = first.c_struct(), second.c_struct(), fmm_algo_t()
    _check(lib().fmm_algo_compose(ctypes.byref(a1), ctypes.byref(a2), U.ctypes.data_as(_i32p),
                                  V.ctypes.data_as(_i32p), W.ctypes.data_as(_i32p), ctypes.byref(out)),
           "fmm_algo_compose")
    return Algo(p, U, V, W, name=f"{first.name}x{second.name}")


class Plan:
    """Owns an ``fmm_plan_t*``; destroyed by ``fmm_plan_destroy`` or garbage collection."""

    def __init__(self, handle: int, n: int, algo: Algo, depth: int, dtype: str):
        self.handle = ctypes.c_void_p(handle)
        self.n, self.algo, self.depth, self.dtype = n, algo, depth, dtype

    def info(self) -> dict:
        return fmm_plan_get_info(self)

    def __del__(self):
        try:
            fmm_plan_destroy(self)
        except Exception:
            pass


def fmm_plan_create(n: int, algo: Algo, depth: int, dtype: str = "f64", schedule: str = "auto",
                    materialize_levels: int = 0, ozaki_slices: int = 0, wait_timeout_s: float = 0.0,
                    debug_poison_chain: int = 0, record_kernel_time: bool = False, tile_n: int = 0,
                    shard_count: int = 0, shard_index: int = 0, post_additions: str = "auto") -> Plan:
    """A plan for ``algo`` (an :class:`Algo`, or a :class:`RationalAlgo` through
    fmm_plan_create_rational) with the given options; ``shard_count`` > 1 makes it compute shard
    ``shard_index`` of the leaf products only; ``post_additions`` is "auto", "fused" or "levels"
    (see fmm_plan_options_t)."""
    h = ctypes.c_void_p()
    a = algo.c_struct()
    opts = fmm_plan_options_t(SCHEDULES[schedule], int(materialize_levels), int(ozaki_slices),
                              float(wait_timeout_s), int(debug_poison_chain), int(bool(record_kernel_time)),
                              int(tile_n), int(shard_count), int(shard_index), POST_ADDITIONS[post_additions])
    create = lib().fmm_plan_create_rational if isinstance(algo, RationalAlgo) else lib().fmm_plan_create_ex
    _check(create(ctypes.byref(h), int(n), ctypes.byref(a), int(depth), DTYPES[dtype], ctypes.byref(opts)),
           f"fmm_plan_create(n={n}, {algo}, depth={depth})")
    return Plan(h.value, int(n), algo, int(depth), dtype)


def fmm_plan_destroy(plan: Plan):
    if plan is not None and plan.handle:
        lib().fmm_plan_destroy(plan.handle)
        plan.handle = ctypes.c_void_p()


def fmm_plan_get_info(plan: Plan) -> dict:
    info = fmm_plan_info_t()
    _check(lib().fmm_plan_get_info(plan.handle, ctypes.byref(info)), "fmm_plan_get_info")
    return {k: getattr(info, k) for k, _ in fmm_plan_info_t._fields_}


def fmm_plan_last_kernel_ms(plan: Plan):
    """(leaf-kernel ms, whole-call ms) of the plan's most recent fmm_gemm (needs record_kernel_time)."""
    a, b = ctypes.c_float(), ctypes.c_float()
    _check(lib().fmm_plan_last_kernel_ms(plan.handle, ctypes.byref(a), ctypes.byref(b)), "fmm_plan_last_kernel_ms")
    return float(a.value), float(b.value)


def fmm_measure_fp64_peak(stream=None):
    """(DMMA TFLOP/s, DFMA TFLOP/s) measured on the current device."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(lib().fmm_measure_fp64_peak(ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(a), ctypes.byref(b)),
           "fmm_measure_fp64_peak")
    return float(a.value), float(b.value)


def fmm_measure_e4m3_peak(stream=None) -> float:
    """TFLOP/s of mma.sync m16n8k32 e4m3 (FP32 accumulation) measured on the current device."""
    a = ctypes.c_double()
    _check(lib().fmm_measure_e4m3_peak(ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(a)), "fmm_measure_e4m3_peak")
    return float(a.value)


def fmm_plan_last_phase_ms(plan: Plan) -> dict:
    """{materialize, slice, leaf, peel, post} milliseconds of the plan's most recent fmm_gemm."""
    arr = (ctypes.c_float * 5)()
    _check(lib().fmm_plan_last_phase_ms(plan.handle, arr, 5), "fmm_plan_last_phase_ms")
    return dict(zip(("materialize", "slice", "leaf", "peel", "post"), (float(x) for x in arr)))


def fmm_plan_workspace_bytes(plan: Plan) -> int:
    return int(lib().fmm_plan_workspace_bytes(plan.handle))


def _stream_ptr(stream) -> int:
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _check_operand(X, n: int, name: str, device: bool = True, complex_: bool = False, f32: bool = False):
    import torch

    if not isinstance(X, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    want = torch.complex128 if complex_ else (torch.float32 if f32 else torch.float64)
    if X.dtype != want or X.shape != (n, n) or not X.is_contiguous():
        raise ValueError(f"{name} must be a contiguous {str(want).replace('torch.', '')} tensor of shape ({n}, {n})")
    if device and not X.is_cuda:
        raise ValueError(f"{name} must live on a CUDA device")
    if not device and X.is_cuda:
        raise ValueError(f"{name} must live in host memory")


def fmm_gemm(plan: Plan, A, B, C, stream=None):
    """C = A @ B on the GPU (asynchronous on ``stream``, default: torch's current stream); complex128
    tensors for a "c128" / "c128_3m" plan, float32 for "f32" (through fmm_gemm_f32_ex), float64
    otherwise."""
    if plan.dtype == "f32":
        return fmm_gemm_f32_ex(plan, 1.0, A, B, 0.0, C, stream)
    n = plan.n
    for X, nm in ((A, "A"), (B, "B"), (C, "C")):
        _check_operand(X, n, nm, complex_=plan.dtype in COMPLEX_DTYPES)
    _check(lib().fmm_gemm(plan.handle, ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                          ctypes.c_void_p(C.data_ptr()), ctypes.c_void_p(_stream_ptr(stream))), "fmm_gemm")
    return C


def fmm_gemm_ex(plan: Plan, alpha: float, A, B, beta: float, C, stream=None):
    """C = alpha * A @ B + beta * C on the GPU (beta = 0: C is not read; alpha = 0: A, B are not read);
    real alpha and beta, also for complex plans; an "f32" plan goes through fmm_gemm_f32_ex."""
    if plan.dtype == "f32":
        return fmm_gemm_f32_ex(plan, alpha, A, B, beta, C, stream)
    n = plan.n
    for X, nm in ((A, "A"), (B, "B"), (C, "C")):
        _check_operand(X, n, nm, complex_=plan.dtype in COMPLEX_DTYPES)
    _check(lib().fmm_gemm_ex(plan.handle, float(alpha), ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                             float(beta), ctypes.c_void_p(C.data_ptr()), ctypes.c_void_p(_stream_ptr(stream))),
           "fmm_gemm_ex")
    return C


def fmm_gemm_f32_ex(plan: Plan, alpha: float, A, B, beta: float, C, stream=None):
    """C = alpha * A @ B + beta * C for float32 CUDA tensors and an "f32" plan."""
    n = plan.n
    for X, nm in ((A, "A"), (B, "B"), (C, "C")):
        _check_operand(X, n, nm, f32=True)
    _check(lib().fmm_gemm_f32_ex(plan.handle, float(alpha), ctypes.c_void_p(A.data_ptr()),
                                 ctypes.c_void_p(B.data_ptr()), float(beta), ctypes.c_void_p(C.data_ptr()),
                                 ctypes.c_void_p(_stream_ptr(stream))), "fmm_gemm_f32_ex")
    return C


def fmm_gemm_host(plan: Plan, A, B, C, stream=None):
    """C = A @ B with host tensors; copies in and out inside the call (blocking)."""
    n = plan.n
    for X, nm in ((A, "A"), (B, "B"), (C, "C")):
        _check_operand(X, n, nm, device=False, complex_=plan.dtype in COMPLEX_DTYPES, f32=plan.dtype == "f32")
    _check(lib().fmm_gemm_host(plan.handle, ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                               ctypes.c_void_p(C.data_ptr()), ctypes.c_void_p(_stream_ptr(stream))),
           "fmm_gemm_host")
    return C


def fmm_host_alloc(nbytes: int) -> int:
    """Page-locked host memory (huge-page backed and registered where the system allows); returns the
    address, to be released with fmm_host_free."""
    p = ctypes.c_void_p()
    _check(lib().fmm_host_alloc(ctypes.byref(p), ctypes.c_size_t(int(nbytes))), "fmm_host_alloc")
    return int(p.value)


def fmm_host_free(addr: int):
    _check(lib().fmm_host_free(ctypes.c_void_p(int(addr) if addr else None)), "fmm_host_free")


def fmm_host_huge_page_bytes() -> int:
    return int(lib().fmm_host_huge_page_bytes())


class _HostBlock:
    """Owns one fmm_host_alloc block; released when the last tensor viewing it is gone."""

    def __init__(self, nbytes: int):
        self.addr = fmm_host_alloc(nbytes)
        self.nbytes = nbytes

    def __del__(self):
        if getattr(self, "addr", 0):
            try:
                fmm_host_free(self.addr)
            except Exception:
                pass
            self.addr = 0


def host_empty(shape, dtype=None):
    """An uninitialised CPU tensor in fmm_host_alloc memory (the buffers fmm_gemm_host copies fastest
    from and to); the memory is released with the tensor and its views."""
    import torch

    dtype = torch.float64 if dtype is None else dtype
    if torch.cuda.is_available():
        # torch reports a buffer as page-locked (and copies from it asynchronously) only once its own
        # CUDA state is initialised
        torch.cuda.init()
    shape = tuple(int(x) for x in (shape if isinstance(shape, (tuple, list)) else (shape,)))
    count = 1
    for x in shape:
        count *= x
    nbytes = max(count * torch.empty((), dtype=dtype).element_size(), 1)
    block = _HostBlock(nbytes)
    arr = (ctypes.c_byte * nbytes).from_address(block.addr)
    arr._fmm_block = block  # torch.frombuffer keeps arr, and so the block, alive
    return torch.frombuffer(arr, dtype=dtype, count=count).view(shape)


def fmm_gemm_noalloc(algo: Algo, depth: int, A, B, C, stream=None):
    """C = A @ B through the allocation-free entry point (fused schedule, static scratch)."""
    n = A.shape[0]
    for X, nm in ((A, "A"), (B, "B"), (C, "C")):
        _check_operand(X, n, nm)
    a = algo.c_struct()
    _check(lib().fmm_gemm_noalloc(int(n), ctypes.byref(a), int(depth), ctypes.c_void_p(A.data_ptr()),
                                  ctypes.c_void_p(B.data_ptr()), ctypes.c_void_p(C.data_ptr()),
                                  ctypes.c_void_p(_stream_ptr(stream))), "fmm_gemm_noalloc")
    return C


def fmm_debug_fail_allocation(k: int):
    """Testing only: the k-th next allocation of the library fails (k < 0: none)."""
    lib().fmm_debug_fail_allocation(int(k))


def fmm_debug_live_allocations() -> int:
    """Testing only: allocations of the library currently live."""
    return int(lib().fmm_debug_live_allocations())


def fmm_noalloc_sync_status(stream=None) -> int:
    """Synchronizes the stream and returns the device status of the latest fmm_gemm_noalloc call (0 = ok)."""
    return int(lib().fmm_noalloc_sync_status(ctypes.c_void_p(_stream_ptr(stream))))


def fmm_noalloc_set_debug(wait_timeout_s: float = 5.0, poison_chain: bool = False):
    """Testing only: wait bound and counter poisoning of later fmm_gemm_noalloc calls."""
    _check(lib().fmm_noalloc_set_debug(float(wait_timeout_s), int(bool(poison_chain))), "fmm_noalloc_set_debug")


def fmm_gemm_batched(plans, As, Bs, Cs, stream=None, alphas=None, betas=None):
    """C[i] = A[i] @ B[i] as one grouped launch; with ``alphas`` / ``betas`` (sequences of floats,
    default all 1 / all 0) C[i] = alpha[i] * A[i] @ B[i] + beta[i] * C[i] (fmm_gemm_batched_ex)."""
    count = len(plans)
    if not (len(As) == len(Bs) == len(Cs) == count):
        raise ValueError("plans, A, B, C must have the same length")
    if len({id(p) for p in plans}) != count:
        raise ValueError("each product of a batch needs its own plan")
    for p, A, B, C in zip(plans, As, Bs, Cs):
        for X, nm in ((A, "A"), (B, "B"), (C, "C")):
            _check_operand(X, p.n, nm, complex_=p.dtype in COMPLEX_DTYPES,
                           f32=p.dtype == "f32")  # the library rejects complex and f32 plans
    arr = ctypes.c_void_p * max(count, 1)
    hp = arr(*[p.handle.value for p in plans])
    ha = arr(*[A.data_ptr() for A in As])
    hb = arr(*[B.data_ptr() for B in Bs])
    hc = arr(*[C.data_ptr() for C in Cs])
    if alphas is None and betas is None:
        _check(lib().fmm_gemm_batched(hp, ha, hb, hc, count, ctypes.c_void_p(_stream_ptr(stream))),
               "fmm_gemm_batched")
        return Cs
    darr = ctypes.c_double * max(count, 1)
    al = None if alphas is None else darr(*[float(x) for x in alphas])
    be = None if betas is None else darr(*[float(x) for x in betas])
    if (alphas is not None and len(alphas) != count) or (betas is not None and len(betas) != count):
        raise ValueError("alphas and betas must have one entry per product")
    _check(lib().fmm_gemm_batched_ex(hp, al, ha, hb, be, hc, count, ctypes.c_void_p(_stream_ptr(stream))),
           "fmm_gemm_batched_ex")
    return Cs


class BatchGraph:
    """A captured fmm_gemm_batched; keeps its plans and tensors alive."""

    def __init__(self, handle, keep):
        self.handle = ctypes.c_void_p(handle)
        self._keep = keep

    def __del__(self):
        try:
            fmm_batch_graph_destroy(self)
        except Exception:
            pass


def fmm_batch_graph_create(plans, As, Bs, Cs) -> BatchGraph:
    count = len(plans)
    if not (len(As) == len(Bs) == len(Cs) == count) or count < 1:
        raise ValueError("plans, A, B, C must have the same nonzero length")
    for p, A, B, C in zip(plans, As, Bs, Cs):
        for X, nm in ((A, "A"), (B, "B"), (C, "C")):
            _check_operand(X, p.n, nm)
    arr = ctypes.c_void_p * count
    h = ctypes.c_void_p()
    _check(lib().fmm_batch_graph_create(ctypes.byref(h), arr(*[p.handle.value for p in plans]),
                                        arr(*[A.data_ptr() for A in As]), arr(*[B.data_ptr() for B in Bs]),
                                        arr(*[C.data_ptr() for C in Cs]), count), "fmm_batch_graph_create")
    return BatchGraph(h.value, (list(plans), list(As), list(Bs), list(Cs)))


def fmm_batch_graph_launch(graph: BatchGraph, stream=None):
    _check(lib().fmm_batch_graph_launch(graph.handle, ctypes.c_void_p(_stream_ptr(stream))), "fmm_batch_graph_launch")


def fmm_batch_graph_destroy(graph: BatchGraph):
    if graph is not None and graph.handle:
        lib().fmm_batch_graph_destroy(graph.handle)
        graph.handle = ctypes.c_void_p()


class fmm_tune_result_t(ctypes.Structure):
    _fields_ = [("algo_index", ctypes.c_int), ("depth", ctypes.c_int), ("ms", ctypes.c_double),
                ("tile_n", ctypes.c_int), ("schedule", ctypes.c_int), ("depth0_ms", ctypes.c_double),
                ("candidates", ctypes.c_int)]


_SCHEDULE_NAMES = {v: k for k, v in SCHEDULES.items()}


def fmm_autotune(n: int, algos, max_depth: int = 3, min_leaf: int = 64, reps: int = 5, stream=None) -> dict:
    """The fastest configuration for size n: {"algo", "depth", "tile_n", "schedule", "ms", "depth0_ms",
    "candidates"} ("algo" is one of ``algos``; depth 0 is the classic product)."""
    structs = [a.c_struct() for a in algos]
    ptrs = (ctypes.POINTER(fmm_algo_t) * len(algos))(*[ctypes.pointer(x) for x in structs])
    res = fmm_tune_result_t()
    _check(lib().fmm_autotune(int(n), ptrs, len(algos), int(max_depth), int(min_leaf), int(reps),
                              ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(res)), f"fmm_autotune(n={n})")
    return {"algo": algos[res.algo_index], "depth": res.depth, "tile_n": res.tile_n,
            "schedule": _SCHEDULE_NAMES[res.schedule], "ms": res.ms, "depth0_ms": res.depth0_ms,
            "candidates": res.candidates}


def fmm_sync_status(plan: Plan, stream=None) -> int:
    """Synchronizes the stream and returns the plan's device status code (0 = ok)."""
    return int(lib().fmm_sync_status(plan.handle, ctypes.c_void_p(_stream_ptr(stream))))
