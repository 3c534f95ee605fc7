"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the oracle.

This module holds no arithmetic of the multiplication method: only the random
streams and the value distributions of the workloads.  Every stream is
SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): output i of seed s is mix(s + (i + 1) * 0x9E3779B97F4A7C15)
with the published finaliser.  Doubles in [0, 1) take the top 53 bits.

Workload recipes (square FP64 operands, row-major):
  * ``uniform``  -- i.i.d. uniform[-1, 1]
  * ``normal``   -- i.i.d. N(0, 1) by Box-Muller on two consecutive uniforms
  * ``integer``  -- round(uniform[-16.5, 16.5)) clamped to [-16, 16]
  * ``wide``     -- uniform[-1, 1] * 10**uniform(-phi, phi) per entry (Ozaki inputs)
The operand A of a workload uses ``seed``, B uses ``seed + 1``.
"""
from __future__ import annotations

import math

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 22


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs start .. start+count-1 of the SplitMix64 stream with the given seed (uint64)."""
    out = np.empty(count, dtype=np.uint64)
    s = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        for c0 in range(0, count, _CHUNK):
            c1 = min(count, c0 + _CHUNK)
            idx = np.arange(start + c0 + 1, start + c1 + 1, dtype=np.uint64)
            z = s + idx * _GAMMA
            z = (z ^ (z >> np.uint64(30))) * _M1
            z = (z ^ (z >> np.uint64(27))) * _M2
            out[c0:c1] = z ^ (z >> np.uint64(31))
    return out


def uniform01(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Doubles in [0, 1) with 53 random bits each."""
    return (splitmix64(seed, count, start) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def matrix(n: int, kind: str = "uniform", seed: int = 1, phi: float = 0.0, m: int | None = None) -> np.ndarray:
    """An n x m (default square) float64 matrix of the named distribution."""
    rows, cols = n, (n if m is None else m)
    count = rows * cols
    if kind == "uniform":
        x = 2.0 * uniform01(seed, count) - 1.0
    elif kind == "normal":
        u = uniform01(seed, 2 * count)
        u1, u2 = u[0::2], u[1::2]
        x = np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)
    elif kind == "integer":
        x = np.floor(33.0 * uniform01(seed, count)) - 16.0
    elif kind == "wide":
        u = uniform01(seed, 2 * count)
        x = (2.0 * u[0::2] - 1.0) * np.power(10.0, phi * (2.0 * u[1::2] - 1.0))
    else:
        raise ValueError(f"unknown input kind {kind!r}")
    return np.ascontiguousarray(x.reshape(rows, cols))


def operands(n: int, kind: str = "uniform", seed: int = 1, phi: float = 0.0):
    """(A, B) for one workload: A from ``seed``, B from ``seed + 1``."""
    return matrix(n, kind, seed, phi), matrix(n, kind, seed + 1, phi)


def sample_indices(n: int, count: int = 4096, seed: int = 7):
    """``count`` (row, col) pairs in [0, n) x [0, n) from one SplitMix64 stream."""
    z = splitmix64(seed, 2 * count)
    rows = (z[0::2] % np.uint64(n)).astype(np.int64)
    cols = (z[1::2] % np.uint64(n)).astype(np.int64)
    return rows, cols


def batch_sizes(count: int = 256, lo: int = 128, hi: int = 4096, seed: int = 3) -> list[int]:
    """Sizes n_i = round(exp(uniform[ln lo, ln hi])) for the batched workload."""
    u = uniform01(seed, count)
    return [int(round(math.exp(math.log(lo) + (math.log(hi) - math.log(lo)) * float(x)))) for x in u]
