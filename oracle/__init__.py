"""CPU oracle for recursive bilinear fast matrix multiplication (arXiv 2312.12732).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package; the library's product
path never does.  The arithmetic lives in ``fmm_oracle.c`` (plain C, binary64,
no FMA contraction); this module only builds and loads it and marshals numpy
arrays.

Functions (each follows the passage cited in ``fmm_oracle.c``):

* ``brent_mismatches(p, U, V, W)`` -- exact Brent-equation check, Section 2.
* ``brent_mismatches_rational(p, U, V, W, dens)`` / ``bilinear_rational(...)`` --
  the same for coefficients U / den_u, V / den_v, W / den_w (Section 2: the
  coefficients need not be integers).
* ``classic(A, B)`` -- textbook triple loop, ascending k (Section 2).
* ``bilinear(A, B, p, U, V, W, depth)`` -- recursive evaluation of equation
  `strassen`, level by level, with the peeling rule stated in the C source.
* ``sample_dot2(A, B, rows, cols)`` -- compensated dot products (Ogita, Rump,
  Oishi 2005) for sampled reference entries.
* ``rect_brent_mismatches(pm, pk, pn, U, V, W)`` / ``rect_bilinear(A, B, levels)``
  -- rectangular algorithms <pm,pk,pn;R> (the factor-6 and factor-12 discussion
  of Section 2), checked exactly and evaluated level by level, one algorithm per
  level, on M x K times K x N operands.
* ``classic_complex(A, B)`` / ``bilinear_complex(A, B, p, U, V, W, depth)`` --
  the same products for complex128 matrices (Section 1 names double complex
  among the deployable types): real coefficients act on both parts alike,
  leaf products use the textbook complex product.
* ``set_num_threads(k)`` -- OpenMP threads used by the loops (timing only).
* ``axpby(alpha, P, beta, C)`` / ``scaled(alpha, A, B, beta, C, ...)`` -- the
  update C = alpha A B + beta C (Section 3 states C = alpha A B; beta is the
  BLAS extension), with beta = 0 leaving C unread and alpha = 0 leaving A B
  unread.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fmm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (gcc, OpenMP, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
               "-std=c11", _SRC, "-o", _LIB + ".tmp", "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        i64, i32, dp = ctypes.c_int64, ctypes.c_int, ctypes.POINTER(ctypes.c_double)
        ip32 = ctypes.POINTER(ctypes.c_int32)
        ip64 = ctypes.POINTER(ctypes.c_int64)
        lib.fmm_oracle_brent_mismatches.restype = i64
        lib.fmm_oracle_brent_mismatches.argtypes = [i32, i32, ip32, ip32, ip32]
        lib.fmm_oracle_classic.restype = None
        lib.fmm_oracle_classic.argtypes = [i64, i64, i64, dp, i64, dp, i64, dp, i64]
        lib.fmm_oracle_bilinear.restype = ctypes.c_int
        lib.fmm_oracle_bilinear.argtypes = [i64, dp, i64, dp, i64, dp, i64, i32, i32, ip32, ip32,
                                            ip32, i32]
        lib.fmm_oracle_brent_mismatches_rational.restype = i64
        lib.fmm_oracle_brent_mismatches_rational.argtypes = [i32, i32, ip32, ip32, ip32, i32, i32, i32]
        lib.fmm_oracle_bilinear_rational.restype = ctypes.c_int
        lib.fmm_oracle_bilinear_rational.argtypes = [i64, dp, i64, dp, i64, dp, i64, i32, i32, ip32, ip32,
                                                     ip32, i32, i32, i32, i32]
        lib.fmm_oracle_dot2.restype = ctypes.c_double
        lib.fmm_oracle_dot2.argtypes = [i64, dp, i64, dp, i64]
        lib.fmm_oracle_sample_dot2.restype = None
        lib.fmm_oracle_sample_dot2.argtypes = [i64, dp, i64, dp, i64, i64, ip64, ip64, dp]
        lib.fmm_oracle_rect_brent_mismatches.restype = i64
        lib.fmm_oracle_rect_brent_mismatches.argtypes = [i32, i32, i32, i32, ip32, ip32, ip32]
        pp32 = ctypes.POINTER(ip32)
        lib.fmm_oracle_rect_bilinear.restype = ctypes.c_int
        lib.fmm_oracle_rect_bilinear.argtypes = [i64, i64, i64, dp, i64, dp, i64, dp, i64, i32, ip32, pp32, pp32,
                                                 pp32]
        lib.fmm_oracle_classic_complex.restype = None
        lib.fmm_oracle_classic_complex.argtypes = [i64, i64, i64, dp, i64, dp, i64, dp, i64]
        lib.fmm_oracle_bilinear_complex.restype = ctypes.c_int
        lib.fmm_oracle_bilinear_complex.argtypes = [i64, dp, i64, dp, i64, dp, i64, i32, i32, ip32, ip32, ip32,
                                                    i32]
        lib.fmm_oracle_axpby.restype = None
        lib.fmm_oracle_axpby.argtypes = [i64, ctypes.c_double, dp, ctypes.c_double, dp]
        lib.fmm_oracle_set_num_threads.restype = None
        lib.fmm_oracle_set_num_threads.argtypes = [i32]
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _alg(p, U, V, W):
    U = np.ascontiguousarray(U, dtype=np.int32)
    V = np.ascontiguousarray(V, dtype=np.int32)
    W = np.ascontiguousarray(W, dtype=np.int32)
    assert U.shape == V.shape == W.shape and U.shape[0] == p * p, "U, V, W must be p^2 x R"
    return U, V, W, int(U.shape[1])


def _ip32(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def brent_mismatches(p: int, U, V, W) -> int:
    """Number of Brent equations (out of p^6) that fail; 0 means (U,V,W) multiplies exactly."""
    U, V, W, R = _alg(p, U, V, W)
    return int(_load().fmm_oracle_brent_mismatches(p, R, _ip32(U), _ip32(V), _ip32(W)))


def _mat(A):
    A = np.ascontiguousarray(A, dtype=np.float64)
    assert A.ndim == 2
    return A


def classic(A, B) -> np.ndarray:
    """C = A B by the ascending-k triple loop."""
    A, B = _mat(A), _mat(B)
    M, K = A.shape
    K2, N = B.shape
    assert K == K2
    C = np.empty((M, N), dtype=np.float64)
    _load().fmm_oracle_classic(M, N, K, _dp(A), K, _dp(B), N, _dp(C), N)
    return C


def bilinear(A, B, p: int, U, V, W, depth: int) -> np.ndarray:
    """C = A B (square) by `depth` recursive levels of the bilinear algorithm (U, V, W)."""
    A, B = _mat(A), _mat(B)
    n = A.shape[0]
    assert A.shape == (n, n) and B.shape == (n, n)
    U, V, W, R = _alg(p, U, V, W)
    C = np.empty((n, n), dtype=np.float64)
    rc = _load().fmm_oracle_bilinear(n, _dp(A), n, _dp(B), n, _dp(C), n, p, R, _ip32(U), _ip32(V),
                                     _ip32(W), depth)
    if rc != 0:
        raise MemoryError("oracle: temporary allocation failed")
    return C


def brent_mismatches_rational(p: int, U, V, W, dens) -> int:
    """Number of failed Brent equations of the rational algorithm (U / du, V / dv, W / dw)."""
    U, V, W, R = _alg(p, U, V, W)
    du, dv, dw = (int(d) for d in dens)
    return int(_load().fmm_oracle_brent_mismatches_rational(p, R, _ip32(U), _ip32(V), _ip32(W), du, dv, dw))


def bilinear_rational(A, B, p: int, U, V, W, dens, depth: int) -> np.ndarray:
    """C = A B by `depth` recursive levels of the rational algorithm (U / du, V / dv, W / dw)."""
    A, B = _mat(A), _mat(B)
    n = A.shape[0]
    assert A.shape == (n, n) and B.shape == (n, n)
    U, V, W, R = _alg(p, U, V, W)
    du, dv, dw = (int(d) for d in dens)
    C = np.empty((n, n), dtype=np.float64)
    rc = _load().fmm_oracle_bilinear_rational(n, _dp(A), n, _dp(B), n, _dp(C), n, p, R, _ip32(U), _ip32(V),
                                              _ip32(W), du, dv, dw, depth)
    if rc == -2:
        raise ValueError("oracle: denominators must be positive")
    if rc != 0:
        raise MemoryError("oracle: temporary allocation failed")
    return C


def _rect(alg):
    pm, pk, pn, U, V, W = alg
    U = np.ascontiguousarray(U, dtype=np.int32)
    V = np.ascontiguousarray(V, dtype=np.int32)
    W = np.ascontiguousarray(W, dtype=np.int32)
    R = U.shape[1]
    assert U.shape == (pm * pk, R) and V.shape == (pk * pn, R) and W.shape == (pm * pn, R)
    return int(pm), int(pk), int(pn), R, U, V, W


def rect_brent_mismatches(pm: int, pk: int, pn: int, U, V, W) -> int:
    """Failed Brent equations of the rectangular algorithm <pm,pk,pn;R> (exact)."""
    pm, pk, pn, R, U, V, W = _rect((pm, pk, pn, U, V, W))
    return int(_load().fmm_oracle_rect_brent_mismatches(pm, pk, pn, R, _ip32(U), _ip32(V), _ip32(W)))


def rect_bilinear(A, B, levels) -> np.ndarray:
    """C = A B (M x K times K x N) by one recursion level per entry of ``levels``, each a
    rectangular algorithm (pm, pk, pn, U, V, W), outermost first."""
    A, B = _mat(A), _mat(B)
    M, K = A.shape
    K2, N = B.shape
    assert K == K2
    lv = [_rect(a) for a in levels]
    ip32 = ctypes.POINTER(ctypes.c_int32)
    arr = ip32 * max(len(lv), 1)
    dims = np.array([[a[0], a[1], a[2], a[3]] for a in lv] or [[1, 1, 1, 1]], dtype=np.int32).ravel()
    Us = arr(*[_ip32(a[4]) for a in lv])
    Vs = arr(*[_ip32(a[5]) for a in lv])
    Ws = arr(*[_ip32(a[6]) for a in lv])
    C = np.empty((M, N), dtype=np.float64)
    rc = _load().fmm_oracle_rect_bilinear(M, K, N, _dp(A), K, _dp(B), N, _dp(C), N, len(lv), _ip32(dims), Us, Vs, Ws)
    if rc == -2:
        raise ValueError("oracle: bad level description")
    if rc != 0:
        raise MemoryError("oracle: temporary allocation failed")
    return C


def _cmat(A):
    A = np.ascontiguousarray(A, dtype=np.complex128)
    assert A.ndim == 2
    return A


def _cdp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def classic_complex(A, B) -> np.ndarray:
    """C = A B for complex128 matrices by the ascending-k triple loop."""
    A, B = _cmat(A), _cmat(B)
    M, K = A.shape
    K2, N = B.shape
    assert K == K2
    C = np.empty((M, N), dtype=np.complex128)
    _load().fmm_oracle_classic_complex(M, N, K, _cdp(A), K, _cdp(B), N, _cdp(C), N)
    return C


def bilinear_complex(A, B, p: int, U, V, W, depth: int) -> np.ndarray:
    """C = A B (square complex128) by `depth` recursive levels of the integer algorithm (U, V, W)."""
    A, B = _cmat(A), _cmat(B)
    n = A.shape[0]
    assert A.shape == (n, n) and B.shape == (n, n)
    U, V, W, R = _alg(p, U, V, W)
    C = np.empty((n, n), dtype=np.complex128)
    rc = _load().fmm_oracle_bilinear_complex(n, _cdp(A), n, _cdp(B), n, _cdp(C), n, p, R, _ip32(U), _ip32(V),
                                             _ip32(W), depth)
    if rc != 0:
        raise MemoryError("oracle: temporary allocation failed")
    return C


def dot2(x, y) -> float:
    """Compensated dot product of two vectors (Dot2)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    assert x.shape == y.shape and x.ndim == 1
    return float(_load().fmm_oracle_dot2(x.shape[0], _dp(x), 1, _dp(y), 1))


def sample_dot2(A, B, rows, cols) -> np.ndarray:
    """Reference entries (A B)[rows[t], cols[t]] by compensated dot products."""
    A, B = _mat(A), _mat(B)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    cols = np.ascontiguousarray(cols, dtype=np.int64)
    assert rows.shape == cols.shape
    M, K = A.shape
    K2, N = B.shape
    assert K == K2
    assert rows.size == 0 or (rows.min() >= 0 and rows.max() < M and cols.min() >= 0 and cols.max() < N)
    out = np.empty(rows.shape[0], dtype=np.float64)
    ip64 = ctypes.POINTER(ctypes.c_int64)
    _load().fmm_oracle_sample_dot2(K, _dp(A), K, _dp(B), N, rows.shape[0], rows.ctypes.data_as(ip64),
                                   cols.ctypes.data_as(ip64), _dp(out))
    return out


def axpby(alpha: float, P, beta: float, C) -> np.ndarray:
    """alpha * P + beta * C elementwise, in a new array; P is not read when alpha == 0
    (it may be None) and C is not read when beta == 0."""
    C = np.array(C, dtype=np.float64, order="C", copy=True)
    pp = None
    if alpha != 0.0:
        P = np.ascontiguousarray(P, dtype=np.float64)
        assert P.shape == C.shape
        pp = _dp(P)
    _load().fmm_oracle_axpby(C.size, float(alpha), pp, float(beta), _dp(C))
    return C


def set_num_threads(threads: int) -> None:
    """OpenMP threads of the parallel loops (classic, Dot2 samples); results do not depend on it."""
    _load().fmm_oracle_set_num_threads(int(threads))


def scaled(alpha: float, A, B, beta: float, C, p: int, U, V, W, depth: int) -> np.ndarray:
    """alpha * bilinear(A, B, ...) + beta * C; the product is not formed when alpha == 0."""
    P = bilinear(A, B, p, U, V, W, depth) if alpha != 0.0 else None
    return axpby(alpha, P, beta, C)
