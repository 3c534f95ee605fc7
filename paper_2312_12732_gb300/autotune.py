"""Per-size choice of algorithm, recursion depth, leaf tile and schedule for batches of products.

Sizes are grouped into half-octave buckets.  For each bucket the library's ``fmm_autotune`` times every
candidate at the bucket's largest size: the classic product (depth 0) and each algorithm at each depth
whose leaf stays at least ``min_leaf``, each with both leaf tile widths of the FP64 kernel (128 x 64 with
two CTAs per SM, 128 x 128 with one) and, at depth 1, both the materialized and the fused pre-additions.
Each candidate's time is the median of ``reps`` runs; the fastest wins.  Choices are cached per GPU name
in memory and, if ``cache_path`` is given, in a JSON file, so that later calls (and later processes
reading the file) reuse them without timing anything.
"""
from __future__ import annotations

import json
import math
import os

from . import _binding as B

_memo: dict[tuple, dict] = {}
# how many times fmm_autotune ran in this process (a cached choice does not add to it)
tuned_count = 0


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
           cache_path: str | None = None, reps: int = 5) -> dict:
    """The tuned configuration for size n: {"algo": name, "depth", "tile_n", "schedule", "ms" (median at
    the bucket's top size), "depth0_ms" (the classic product there), "top": that size}."""
    global tuned_count
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
        _memo[key] = dict(disk[skey])
        return _memo[key]
    algos = [B.fmm_algo_builtin(c) for c in candidates]
    top = max(n, bucket_top(b))
    r = B.fmm_autotune(top, algos, max_depth=max_depth, min_leaf=min_leaf, reps=reps)
    tuned_count += 1
    pick = {"algo": r["algo"].name, "depth": r["depth"], "tile_n": r["tile_n"], "schedule": r["schedule"],
            "ms": r["ms"], "depth0_ms": r["depth0_ms"], "top": top, "candidates": r["candidates"]}
    _memo[key] = pick
    if cache_path:
        disk[skey] = pick
        with open(cache_path, "w") as f:
            json.dump(disk, f, indent=1)
    return pick


def plan_for(n: int, pick: dict):
    """A plan of size n with a tuned configuration (post-additions in the planner's form, as tuned)."""
    return B.fmm_plan_create(n, B.fmm_algo_builtin(pick["algo"]), pick["depth"], schedule=pick["schedule"],
                             tile_n=pick["tile_n"])


def plan_batch(sizes, candidates=("strassen", "winograd"), max_depth: int = 3, min_leaf: int = 128,
               cache_path: str | None = None, reps: int = 5):
    """One plan per size, each with its bucket's tuned configuration; returns (plans, picks)."""
    plans, picks = [], []
    for n in sizes:
        pick = choose(n, candidates, max_depth, min_leaf, cache_path, reps)
        plans.append(plan_for(n, pick))
        picks.append(pick)
    return plans, picks
