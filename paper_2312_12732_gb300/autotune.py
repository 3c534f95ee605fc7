"""Per-size choice of algorithm and recursion depth for batches of products.

Sizes are grouped into half-octave buckets; for each bucket the library's
``fmm_autotune`` times every candidate (algorithm, depth) once at the bucket's
largest size and the fastest wins.  Choices are cached per GPU name in memory
and, if ``cache_path`` is given, in a JSON file.  The leaf tile shape of the
FP64 kernel is fixed (128 x 128 x 16), so the tuned parameters are the
algorithm and the depth (depth 0 = the classic product).
"""
from __future__ import annotations

import json
import math
import os

from . import _binding as B

_memo: dict[tuple, tuple[str, int, float]] = {}


def bucket(n: int) -> int:
    """Half-octave bucket index of n."""
    return int(math.floor(2.0 * math.log2(max(n, 1))))


def bucket_top(b: int) -> int:
    return int(math.floor(2.0 ** ((b + 1) / 2.0)))


def _gpu_name() -> str:
    try:
        import torch

        return torch.cuda.get_device_name()
    except Exception:
        return "unknown"


def choose(n: int, candidates=("strassen", "winograd"), max_depth: int = 3, min_leaf: int = 128,
           cache_path: str | None = None) -> tuple[str, int, float]:
    """(algorithm name, depth, measured ms at the bucket's top size) for size n."""
    b = bucket(n)
    key = (_gpu_name(), b, tuple(candidates), max_depth, min_leaf)
    if key in _memo:
        return _memo[key]
    disk = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            disk = json.load(f)
    skey = json.dumps(list(key))
    if skey in disk:
        _memo[key] = tuple(disk[skey])
        return _memo[key]
    algos = [B.fmm_algo_builtin(c) for c in candidates]
    top = max(n, bucket_top(b))
    algo, depth, ms = B.fmm_autotune(top, algos, max_depth=max_depth, min_leaf=min_leaf)
    _memo[key] = (algo.name, depth, ms)
    if cache_path:
        disk[skey] = list(_memo[key])
        with open(cache_path, "w") as f:
            json.dump(disk, f, indent=1)
    return _memo[key]


def plan_batch(sizes, candidates=("strassen", "winograd"), max_depth: int = 3, min_leaf: int = 128,
               cache_path: str | None = None):
    """One plan per size, each with its bucket's tuned algorithm and depth."""
    plans, picks = [], []
    for n in sizes:
        name, depth, _ = choose(n, candidates, max_depth, min_leaf, cache_path)
        plans.append(B.fmm_plan_create(n, B.fmm_algo_builtin(name), depth))
        picks.append((name, depth))
    return plans, picks
