#!/usr/bin/env python
"""Benchmark: effective FP64 TFLOP/s (2 n^3 / t) of a fast bilinear algorithm
against the classic product, on one GB300.

Default workload: C = A B with n = 8192 FP64 operands, entries uniform[-1, 1]
(SplitMix64 seeds 1 and 2), Strassen's algorithm as printed in the paper
(Section 2) at the default depth, the planner's default schedule.  One step is
one fmm_gemm call: pre-additions, leaf products and post-additions, i.e. the
whole hot path.  Inputs (3 x 512 MiB) are larger than L2 (129 MB), so no
flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W]       # one JSON line
    python bench.py --impl reference ...                      # CPU oracle arm
    python bench.py --sweep                                   # per-algorithm table

With N > 1 (launched by torchrun) the ranks shard one multiplication by its
leaf products (Section 2: the products are independent) and sum their partial
C with one all-reduce; the value is that one multiplication's flops / the
slowest rank's time (strong scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "effective FP64 TFLOP/s (2n³/t), fast algorithm vs classic GEMM, same GB300"
NOMINAL_FP64_TFLOPS = 1.25     # GB300 nominal FP64 (= FP64 tensor) rate
NOMINAL_BF16_TFLOPS = 2250.0   # GB300 nominal dense bf16 rate
FALLBACK_BF16_TFLOPS = 1900.0  # recipe fallback when no measured peaks exist
L2_BYTES = 129e6


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=8192)
    ap.add_argument("--algo", default="strassen^2", help="built-in name; suffix ^2 for its Kronecker square")
    ap.add_argument("--depth", type=int, default=2)
    ap.add_argument("--schedule", default="auto", choices=["auto", "fused", "hybrid"])
    ap.add_argument("--materialize-levels", type=int, default=0)
    ap.add_argument("--kind", default="uniform", choices=["uniform", "normal", "integer", "wide"])
    ap.add_argument("--phi", type=float, default=0.0, help="decades of spread for --kind wide")
    ap.add_argument("--dtype", default="f64", choices=["f64", "f64_ozaki"])
    ap.add_argument("--slices", type=int, default=0, help="emulated leaf: slices per operand (0 = default)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-classic", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-cublas", action="store_true", help="skip the cuBLAS DGEMM context timing")
    ap.add_argument("--cpu-n", type=int, default=4096, help="size of the CPU-oracle sample")
    ap.add_argument("--sweep", action="store_true", help="print one JSON line per algorithm/depth/schedule")
    ap.add_argument("--only", default="", help="sweep: comma-separated algorithm names to keep (default: all)")
    ap.add_argument("--batched", action="store_true",
                    help="batched workload: 256 products, n log-uniform in [128, 4096], one captured graph")
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--batch-max-depth", type=int, default=4, help="batched workload: deepest depth the tuner tries")
    ap.add_argument("--no-emulated", action="store_true",
                    help="skip the emulated-FP64 (Ozaki, Strassen depth 2) measurement added to the JSON line")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched workload (256 autotuned products in one graph) added to the JSON line")
    return ap.parse_args(argv)


# ----------------------------------------------------------------------------- helpers


def workload_name(a) -> str:
    kind = a.kind if a.kind != "wide" else f"wide{a.phi:g}"
    leaf = "fp64" if a.dtype == "f64" else f"ozaki{a.slices or 12}"
    return f"{a.algo.replace('^2', 'x2')}_d{a.depth}_n{a.n}_{kind}_{leaf}"


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return None


def fp64_peak_tflops():
    """FP64 tensor peak: the measured bf16 burst peak times the nominal FP64:bf16 ratio."""
    pk = measured_peaks()
    if pk and pk.get("bf16_tflops"):
        return pk["bf16_tflops"] * NOMINAL_FP64_TFLOPS / NOMINAL_BF16_TFLOPS, \
            "of measured (MEASURED_PEAKS.json bf16 burst x nominal FP64/bf16 ratio 1.25/2250)"
    return FALLBACK_BF16_TFLOPS * NOMINAL_FP64_TFLOPS / NOMINAL_BF16_TFLOPS, \
        "of fallback (1.9 PFLOP/s bf16 x nominal FP64/bf16 ratio 1.25/2250)"


def fp8_peak_tflops():
    """e4m3 tensor peak: the measured bf16 burst peak times the nominal fp8/bf16 ratio (4.5/2.25)."""
    pk = measured_peaks()
    if pk and pk.get("bf16_tflops"):
        return pk["bf16_tflops"] * 4.5 / 2.25, \
            "of measured (MEASURED_PEAKS.json bf16 burst x nominal fp8/bf16 ratio 4.5/2.25)"
    return FALLBACK_BF16_TFLOPS * 2.0, "of fallback (1.9 PFLOP/s bf16 x nominal fp8/bf16 ratio 2)"


KERNEL_SOURCES = {"fmm_f64_kernel": "fmm_f64.cu", "ozaki_tc_kernel": "fmm_ozaki_tc.cu",
                  "ozaki_tc_pair_kernel": "fmm_ozaki_tc.cu"}


def source_digest(kernel: str):
    import hashlib

    src = os.path.join(ROOT, "paper_2312_12732_gb300", "csrc", KERNEL_SOURCES.get(kernel, "fmm_f64.cu"))
    try:
        return hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None


def profile_traffic(kernel: str, workload: str):
    """DRAM bytes per launch of `kernel` on `workload` from an ncu capture summarised in profiles/, if it
    was taken on the current kernel source; else None.  A capture of a smaller case of the same kernel
    names the bench workload it scales to (`scaled_workload`) and the scaled bytes
    (`scaled_dram_bytes_per_launch`, by the units of work the launch processes, as the summary states);
    a capture of the workload itself gives `dram_bytes_per_launch` directly."""
    digest = source_digest(kernel)
    if digest is None:
        return None
    pdir = os.path.join(ROOT, "profiles")
    if not os.path.isdir(pdir):
        return None
    for fn in sorted(os.listdir(pdir)):
        if not fn.endswith(".md"):
            continue
        kv = {}
        for line in open(os.path.join(pdir, fn)):
            if line.startswith("- ") and ":" in line:
                k, v = line[2:].split(":", 1)
                kv[k.strip()] = v.strip().strip("`")
        if kv.get("kernel") != kernel or kv.get("source_sha256_16") != digest:
            continue
        try:
            if kv.get("scaled_workload") == workload:
                return float(kv["scaled_dram_bytes_per_launch"])
            if kv.get("workload") == workload:
                return float(kv["dram_bytes_per_launch"])
        except (KeyError, ValueError):
            return None
    return None


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []
        self.thread = None

    def __enter__(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self.thread:
                self.thread.join(timeout=2)

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable: nvidia-smi gave no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def gpu_uuid(torch, dev):
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return None


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The largest value across ranks (identity without a process group)."""
    if dist is None:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, max_seconds: float) -> float:
    """Whole-job rate: the units of all ranks over the slowest rank's time."""
    return units_per_rank * world / max_seconds


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ----------------------------------------------------------------------------- CPU oracle arm


def golden_algo(name: str):
    """(p, U, V, W) of a built-in algorithm name from the text fixtures in tests/golden (the tables the
    oracle is pinned with), never from the product library: "strassen" is the paper's table with its
    c^t rows placed by their labels, "name^2" its Kronecker square with row-major block re-indexing."""
    from tests.golden import algos as golden

    base = name[:-2] if name.endswith("^2") else name
    table = {"strassen": golden.paper_strassen, "strassen1969": golden.strassen1969, "winograd": golden.winograd,
             "laderman": golden.laderman, "classic2": golden.classic_from_graph}
    if base not in table:
        raise ValueError(f"no golden table for {name!r}")
    alg = table[base]()
    return golden.kron_compose(alg, alg) if name.endswith("^2") else alg


def cpu_oracle_run(a, n_sample: int, reps: int, threads: int | None = None):
    """Times the oracle's recursive evaluation of the same algorithm and depth on
    an n_sample x n_sample sample of the workload distribution, on `threads`
    OpenMP threads (default: all host cores).  Loads only oracle/ (tables from
    tests/golden, inputs from the shared generator module)."""
    import oracle
    from paper_2312_12732_gb300 import inputs

    oracle.build()
    cores = threads or int(os.environ.get("OMP_NUM_THREADS") or os.cpu_count() or 1)
    oracle.set_num_threads(cores)
    p, U, V, W = golden_algo(a.algo)
    A, B = inputs.operands(n_sample, a.kind, seed=1)
    depth = a.depth
    while depth > 0 and p ** depth > n_sample:
        depth -= 1
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        oracle.bilinear(A, B, p, U, V, W, depth)
        times.append(time.perf_counter() - t0)
    return times, cores, depth


def oracle_error(A, B, C_gpu_sampled, rows, cols):
    """Normalised error max |C - C_ref| / (n max|A| max|B|) of sampled GPU entries against the oracle's
    compensated (Dot2) reference entries of the same positions (an accuracy check, not a timed step)."""
    import numpy as np

    import oracle

    ref = oracle.sample_dot2(A, B, rows, cols)
    n = A.shape[0]
    return float(np.max(np.abs(C_gpu_sampled - ref)) / (n * np.abs(A).max() * np.abs(B).max()))


def run_reference(a):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    times, cores, depth = cpu_oracle_run(a, a.cpu_n, a.warmup + a.steps)
    timed = times[a.warmup:] if len(times) > a.warmup else times
    t = statistics.mean(timed)
    value = 2.0 * a.cpu_n ** 3 / t / 1e12
    sample = (f"oracle bilinear evaluation ({a.algo}, depth {depth}) of one {a.cpu_n}x{a.cpu_n} product "
              f"per step, {a.kind} entries, {cores} OpenMP threads; the GPU arm's n={a.n} product is "
              f"sampled at this size to bound CPU time")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(a), "sample_n": a.cpu_n},
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- GPU arm


def make_algo(fmm, name):
    if name.endswith("^2"):
        return fmm.algorithm(name[:-2], 2)
    if name in ("rect_12", "rect_6"):
        # square algorithms composed from rectangular ones: <2,2,3;11> (x) <2,3,2;11> (x) <3,2,2;11> = <12;1331>,
        # <2,2,3;11> (x) classic <3,3,2;18> = <6;198>
        s = fmm.fmm_algo_rect_builtin("strassen_2x2x3")
        c = fmm.fmm_algo_rect_cyclic(s)
        if name == "rect_12":
            r = fmm.fmm_algo_rect_compose(fmm.fmm_algo_rect_compose(s, c), fmm.fmm_algo_rect_cyclic(c))
        else:
            r = fmm.fmm_algo_rect_compose(s, fmm.fmm_algo_rect_classic(3, 3, 2))
        return fmm.fmm_algo_rect_as_square(r)
    if name in ("strassen_dyadic", "strassen_thirds"):
        # Strassen in a basis with non-integer coefficients (exact change of basis, test fixture)
        from tests.golden import rational_algos

        p, U, V, W, dens = getattr(rational_algos, name)()
        return fmm.RationalAlgo(p, U, V, W, dens, name=name)
    return fmm.fmm_algo_builtin(name)


def ozaki_launches(passes: int, peeled: bool) -> int:
    """Kernels of one emulated-leaf call: each materialization pass for both operands, row and column
    slicing, the slice GEMM, the post-additions and (for peeled sizes) the FP64 peel tasks."""
    return 2 * passes + 4 + (1 if peeled else 0)


def f64_launches(info: dict, peeled: bool) -> int:
    """Kernels of one FP64 call: each materialization pass for both operands, the leaf kernel and, when
    the plan stores its leaf products, the post-addition passes and (for peeled sizes) the rank-q launch."""
    passes = info.get("post_passes", 0)
    return 1 + 2 * info["materialize_passes"] + passes + (1 if peeled and passes else 0)


def materialized_bytes(n_core: int, p: int, R_total: int, depth: int, levels: int) -> float:
    """Algorithmic HBM bytes of the materialized pre-additions of both operands: level l reads the
    R^(l-1) blocks of side n_core/p^(l-1) once and writes R^l blocks of side n_core/p^l."""
    if depth <= 0 or levels <= 0:
        return 0.0
    R = round(R_total ** (1.0 / depth))
    total, b = 0.0, float(n_core)
    for lev in range(1, levels + 1):
        total += R ** (lev - 1) * b * b + R ** lev * (b / p) ** 2
        b /= p
    return 2 * 8 * total


def time_plan(torch, fmm, plan, dA, dB, dC, warmup, steps, dist=None, stream=None, after=None):
    """(ms per step over the timed region, mean leaf-kernel ms per launch).  `after(dC)` runs after every
    call on the same stream (the sum of the shards' partial products when the product is sharded)."""
    stream = stream or torch.cuda.current_stream()
    for _ in range(warmup):
        fmm.fmm_gemm(plan, dA, dB, dC, stream)
        if after is not None:
            after(dC)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    leaf = []
    phases = []
    e0.record(stream)
    for _ in range(steps):
        fmm.fmm_gemm(plan, dA, dB, dC, stream)
        if after is not None:
            after(dC)
        leaf.append(fmm.fmm_plan_last_kernel_ms(plan)[0])
        if plan.dtype in ("f64", "f64_ozaki"):  # complex and f32 plans time the whole call only
            phases.append(fmm.fmm_plan_last_phase_ms(plan))
    e1.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    st = fmm.fmm_sync_status(plan, stream)
    if st != 0:
        raise RuntimeError("device status after timed region: " + fmm.fmm_status_string(st))
    time_plan.last_phases = {k: statistics.mean(p[k] for p in phases) for k in phases[0]} if phases else None
    return e0.elapsed_time(e1) / steps, statistics.mean(leaf)


def run_sweep(a):
    import torch

    import paper_2312_12732_gb300 as fmm
    from paper_2312_12732_gb300 import _build, inputs

    _build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    configs = [("strassen", 0, "auto", 0)]
    for algo in ("strassen", "winograd"):
        for d in (1, 2, 3):
            configs += [(algo, d, "fused", 0), (algo, d, "auto", 0)]
    configs += [("strassen^2", 1, "fused", 0), ("strassen^2", 1, "auto", 0), ("strassen^2", 2, "auto", 0),
                ("strassen", 4, "auto", 0), ("strassen", 5, "auto", 0), ("strassen", 6, "auto", 0)]
    configs = [c + ("f64",) for c in configs]
    # both post-addition forms where the planner's choice is close or the depth is large
    configs += [(al, d, "auto", 0, "f64", post) for al, d in (("strassen", 3), ("strassen^2", 2), ("strassen", 5),
                                                              ("strassen", 6)) for post in ("fused", "levels")]
    configs += [("strassen", d, "auto", 0, "f64_ozaki") for d in (0, 1, 2, 3)]
    if a.n >= 16384:
        # large sizes: the materialized schedules only (a fused row takes seconds per call)
        configs = [c for c in configs if c[2] == "auto" and c[0] in ("strassen", "strassen^2", "winograd")
                   and (c[0] != "winograd" or c[1] == 3) and not (len(c) > 5 and c[5] == "fused" and c[1] >= 5)
                   and c[1] <= 5]
    else:
        configs += [("strassen_dyadic", d, "auto", 0, "f64") for d in (1, 2, 3)]
        configs += [("strassen_thirds", 2, "auto", 0, "f64"), ("strassen_dyadic", 2, "auto", 0, "f64_ozaki")]
        configs += [("rect_12", 1, "auto", 0, "f64"), ("rect_6", 1, "auto", 0, "f64"), ("rect_6", 2, "auto", 0, "f64")]
    if a.only:
        keep = set(a.only.split(","))
        configs = [c for c in configs if c[0] in keep]
    n = a.n
    A, B = inputs.operands(n, a.kind, seed=1)
    dA, dB = torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev)
    dC = torch.empty_like(dA)
    rows = [(n, c) for c in configs]
    if a.n == 8192:
        rows += [(6912, ("laderman", d, s, 0, "f64")) for d in (1, 2) for s in ("fused", "auto")]
        rows += [(6912, ("strassen", 0, "auto", 0, "f64"))]
        rows += [(16384, ("strassen", d, "auto", 0, "f64_ozaki")) for d in (0, 2)]
    if a.only:
        rows = [r for r in rows if r[1][0] in set(a.only.split(","))]
    cache = {n: (dA, dB, dC)}
    for nn, cfg in rows:
        algo_name, depth, sched, ml, dt = cfg[:5]
        post = cfg[5] if len(cfg) > 5 else "auto"
        if nn not in cache:
            A2, B2 = inputs.operands(nn, a.kind, seed=1)
            xA2 = torch.from_numpy(A2).to(dev)
            cache = {nn: (xA2, torch.from_numpy(B2).to(dev), torch.empty_like(xA2))}
        xA, xB, xC = cache[nn]
        algo = make_algo(fmm, algo_name)
        plan = fmm.fmm_plan_create(nn, algo, depth, dtype=dt, schedule=sched, materialize_levels=ml,
                                   record_kernel_time=True, post_additions=post if dt == "f64" else "auto")
        ms, leaf = time_plan(torch, fmm, plan, xA, xB, xC, 1, 2)
        info = plan.info()
        lowp = info["flops_lowp"] / leaf / 1e9 if dt == "f64_ozaki" else None
        print(json.dumps({"n": nn, "algo": algo_name, "depth": depth, "schedule": sched, "dtype": dt,
                          "post": ("levels" if info["post_passes"] else "fused") if dt == "f64" else "separate",
                          "lowp_tflops_leaf_kernel": round(lowp, 1) if lowp else None,
                          "materialized": info["materialized_levels"], "ms": round(ms, 3),
                          "leaf_ms": round(leaf, 3), "eff_tflops": round(2.0 * nn ** 3 / ms / 1e9, 4),
                          "exec_tflops_leaf_kernel": round(info["flops_leaf"] / leaf / 1e9, 4),
                          "phases_ms": {k: round(v, 3) for k, v in (time_plan.last_phases or {}).items()}}),
              flush=True)
        fmm.fmm_plan_destroy(plan)
    if a.n <= 8192 and (not a.only or "complex" in a.only.split(",")):
        # double complex: <4,4,4;49> depth 2 through four or three real fast products, and cuBLAS ZGEMM
        # (torch.matmul on complex128) as context; effective complex flops 8 n^3
        del cache
        nn = a.n
        Z1 = torch.complex(torch.from_numpy(inputs.matrix(nn, a.kind, seed=1)),
                           torch.from_numpy(inputs.matrix(nn, a.kind, seed=3))).to(dev)
        Z2 = torch.complex(torch.from_numpy(inputs.matrix(nn, a.kind, seed=2)),
                           torch.from_numpy(inputs.matrix(nn, a.kind, seed=4))).to(dev)
        Z3 = torch.empty_like(Z1)
        for dt in ("c128", "c128_3m"):
            plan = fmm.fmm_plan_create(nn, make_algo(fmm, "strassen^2"), 2, dtype=dt, record_kernel_time=True)
            ms, _ = time_plan(torch, fmm, plan, Z1, Z2, Z3, 1, 2)
            print(json.dumps({"n": nn, "algo": "strassen^2", "depth": 2, "schedule": "auto", "dtype": dt,
                              "ms": round(ms, 3), "eff_complex_tflops": round(8.0 * nn ** 3 / ms / 1e9, 4)}),
                  flush=True)
            fmm.fmm_plan_destroy(plan)
        torch.matmul(Z1, Z2, out=Z3)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(2):
            torch.matmul(Z1, Z2, out=Z3)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 2
        print(json.dumps({"n": nn, "algo": "cuBLAS ZGEMM (context)", "depth": 0, "schedule": "-", "dtype": "c128",
                          "ms": round(ms, 3), "eff_complex_tflops": round(8.0 * nn ** 3 / ms / 1e9, 4)}), flush=True)
        del Z1, Z2, Z3
    if a.n <= 8192 and (not a.only or "f32" in a.only.split(",")):
        # single precision through the emulated leaf (6 slices), and cuBLAS SGEMM in true FP32 (TF32 off) as context
        nn = a.n
        X1 = torch.from_numpy(inputs.matrix(nn, a.kind, seed=1)).float().to(dev)
        X2 = torch.from_numpy(inputs.matrix(nn, a.kind, seed=2)).float().to(dev)
        X3 = torch.empty_like(X1)
        for d in (0, 1, 2, 3):
            plan = fmm.fmm_plan_create(nn, make_algo(fmm, "strassen"), d, dtype="f32", record_kernel_time=True)
            ms, _ = time_plan(torch, fmm, plan, X1, X2, X3, 1, 2)
            print(json.dumps({"n": nn, "algo": "strassen", "depth": d, "schedule": "auto", "dtype": "f32",
                              "ozaki_slices": plan.info()["ozaki_slices"], "ms": round(ms, 3),
                              "eff_tflops": round(2.0 * nn ** 3 / ms / 1e9, 4)}), flush=True)
            fmm.fmm_plan_destroy(plan)
        torch.backends.cuda.matmul.allow_tf32 = False
        torch.matmul(X1, X2, out=X3)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            torch.matmul(X1, X2, out=X3)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 3
        print(json.dumps({"n": nn, "algo": "cuBLAS SGEMM, TF32 off (context)", "depth": 0, "schedule": "-",
                          "dtype": "f32", "ms": round(ms, 3), "eff_tflops": round(2.0 * nn ** 3 / ms / 1e9, 4)}),
              flush=True)
    return 0


def batched_measurement(torch, fmm, dev, count: int, steps: int, warmup: int, tune_reps: int = 5,
                        max_depth: int = 3):
    """The batched workload: `count` products with n_i log-uniform in [128, 4096] (SplitMix64 seed 3),
    entries uniform[-1, 1] (seeded on the device), each planned with its bucket's autotuned (algorithm,
    depth, leaf tile, schedule), all of them run by one CUDA graph (per-plan counter resets and
    materialization passes, then one grouped persistent leaf launch per tile width).  Returns the
    measurement as a dict; the same batch at depth 0 in one graph is timed beside it."""
    import collections

    from paper_2312_12732_gb300 import autotune, inputs

    sizes = inputs.batch_sizes(count, 128, 4096, seed=3)
    t0 = time.perf_counter()
    plans, picks = autotune.plan_batch(sizes, candidates=("strassen", "winograd"), max_depth=max_depth,
                                       min_leaf=128, reps=tune_reps)
    tune_s = time.perf_counter() - t0
    gen = torch.Generator(device=dev)
    gen.manual_seed(1000)
    As, Bs, Cs = [], [], []
    for n in sizes:
        As.append(torch.rand(n, n, dtype=torch.float64, device=dev, generator=gen) * 2 - 1)
        Bs.append(torch.rand(n, n, dtype=torch.float64, device=dev, generator=gen) * 2 - 1)
        Cs.append(torch.empty_like(As[-1]))
    flops = sum(2.0 * n ** 3 for n in sizes)
    flops_exec = sum(p.info()["flops_executed"] for p in plans)

    def time_graph(g, k, warm):
        stream = torch.cuda.current_stream()
        for _ in range(warm):
            fmm.fmm_batch_graph_launch(g, stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fmm.fmm_batch_graph_launch(g, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    g = fmm.fmm_batch_graph_create(plans, As, Bs, Cs)
    sampler = ClockSampler(gpu_uuid(torch, dev))
    with sampler:
        ms = time_graph(g, steps, max(warmup, 3))
    st = fmm.fmm_sync_status(plans[0])
    if st != 0:
        raise RuntimeError("device status: " + fmm.fmm_status_string(st))
    # accuracy: 64 sampled entries of eight products against the oracle's Dot2 references
    errs = []
    for i in range(0, len(sizes), max(1, len(sizes) // 8)):
        A, B = As[i].cpu().numpy(), Bs[i].cpu().numpy()
        rows, cols = inputs.sample_indices(sizes[i], 64, seed=11 + i)
        got = Cs[i].cpu().numpy()[rows, cols]
        errs.append(oracle_error(A, B, got, rows, cols))
    plans0 = [fmm.fmm_plan_create(n, fmm.fmm_algo_builtin("strassen"), 0) for n in sizes]
    g0 = fmm.fmm_batch_graph_create(plans0, As, Bs, Cs)
    ms0 = time_graph(g0, max(2, steps // 2), 1)
    hist = collections.Counter(f"{p['algo']}:d{p['depth']}:t{p['tile_n']}:{p['schedule']}" for p in picks)
    launches = 0
    for p in plans:
        launches += 2 * p.info()["materialize_passes"] + p.info()["post_passes"]
    launches += len({p.info()["tile_n"] for p in plans})
    launches += len({p.info()["tile_n"] for p in plans if p.info()["post_passes"] and p.info()["n_core"] < p.n})
    return {
        "workload": f"batched_{len(sizes)}_loguniform_128_4096_uniform_fp64", "value": flops / (ms * 1e-3) / 1e12,
        "unit": "TFLOP/s", "ms_per_step": ms, "steps": steps, "warmup": max(warmup, 3), "products": len(sizes),
        "sizes_min_max": [min(sizes), max(sizes)], "picks": dict(hist), "autotune_s": round(tune_s, 2),
        "autotune_buckets": len({autotune.bucket(n) for n in sizes}),
        "launch": "one CUDA graph: per-plan counter resets and materialization passes, one grouped persistent "
                  "leaf launch per tile width, then the post-addition passes of the plans that store their leaf "
                  "products and one grouped launch of their rank-q fix-ups",
        "stored_products": sum(1 for p in plans if p.info()["post_passes"]),
        "gpu_launches": steps * launches,
        "classic_depth0_graph": {"value": flops / (ms0 * 1e-3) / 1e12, "ms_per_step": ms0},
        "speedup_vs_classic": ms0 / ms,
        "flops_executed_per_step": flops_exec, "executed_tflops": flops_exec / (ms * 1e-3) / 1e12,
        "normalised_error_sampled_max": max(errs),
        "clocks": sampler.summary(),
    }


def run_batched(a):
    import torch

    import paper_2312_12732_gb300 as fmm
    from paper_2312_12732_gb300 import _build

    _build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    b = batched_measurement(torch, fmm, dev, a.batch_count, a.steps, a.warmup, max_depth=a.batch_max_depth)
    line = {
        "metric": METRIC, "value": b["value"], "unit": "TFLOP/s", "n_gpus": 1, "steps": a.steps,
        "warmup": b["warmup"], "ms_per_step": b["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": b["workload"], "products": b["products"], "sizes_min_max": b["sizes_min_max"],
                   "picks": b["picks"], "autotune_s": b["autotune_s"], "launch": b["launch"],
                   "stored_products": b["stored_products"]},
        "classic_depth0_graph": b["classic_depth0_graph"], "flops_executed_per_step": b["flops_executed_per_step"],
        "executed_tflops": b["executed_tflops"], "speedup_vs_classic": b["speedup_vs_classic"],
        "normalised_error_sampled_max": b["normalised_error_sampled_max"], "clocks": b["clocks"],
        "gpu_launches": b["gpu_launches"],
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(a):
    import numpy as np
    import torch

    import paper_2312_12732_gb300 as fmm
    from paper_2312_12732_gb300 import _build, inputs

    ws, rank, local = dist_env()
    dist = None
    if ws > 1:
        import torch.distributed as dist_mod

        torch.cuda.set_device(local)
        dist_mod.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist = dist_mod
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    if rank == 0:
        _build.build()
    if dist is not None:
        dist.barrier()

    n = a.n
    algo = make_algo(fmm, a.algo)
    A, B = inputs.operands(n, a.kind, seed=1, phi=a.phi)
    dA, dB = torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev)
    dC = torch.empty_like(dA)
    # one GPU: the whole product; N GPUs: rank k computes shard k of the leaf products and the partial
    # products are summed by one all-reduce per step (strong scaling: one product per step for the job)
    sharded = ws > 1
    from paper_2312_12732_gb300 import sharded as shard_mod

    plan = fmm.fmm_plan_create(n, algo, a.depth, dtype=a.dtype, schedule=a.schedule,
                               materialize_levels=a.materialize_levels, ozaki_slices=a.slices,
                               record_kernel_time=True, shard_count=ws if sharded else 0,
                               shard_index=rank if sharded else 0)
    after = shard_mod.reduce_partials if sharded else None
    info = plan.info()

    dmma_peak, dfma_peak = fmm.fmm_measure_fp64_peak()
    e4m3_peak = fmm.fmm_measure_e4m3_peak() if a.dtype == "f64_ozaki" else None
    sampler = ClockSampler(gpu_uuid(torch, dev))
    with sampler:
        ms, leaf_ms = time_plan(torch, fmm, plan, dA, dB, dC, max(a.warmup, 3), a.steps, dist, after=after)
    clocks = sampler.summary()
    main_phases = time_plan.last_phases

    ms = max_over_ranks(ms, dist, dev)
    flops_eff = 2.0 * n ** 3
    value = (flops_eff / (ms * 1e-3) if sharded else job_throughput(flops_eff, ws, ms * 1e-3)) / 1e12

    # accuracy: 4096 sampled entries against the oracle's compensated dot products of the same inputs
    s_rows, s_cols = inputs.sample_indices(n, 4096, seed=7)
    t_rows, t_cols = torch.from_numpy(s_rows).to(dev), torch.from_numpy(s_cols).to(dev)
    err = oracle_error(A, B, dC[t_rows, t_cols].cpu().numpy(), s_rows, s_cols) if rank == 0 else None

    classic = None
    if not a.no_classic and a.depth > 0 and not sharded:
        p0 = fmm.fmm_plan_create(n, algo, 0, record_kernel_time=True)
        ms0, leaf0 = time_plan(torch, fmm, p0, dA, dB, dC, 1, max(2, a.steps // 2), dist)
        classic = {"value": flops_eff / (ms0 * 1e-3) / 1e12, "ms_per_step": ms0, "leaf_kernel_ms": leaf0}
        fmm.fmm_plan_destroy(p0)
        fmm.fmm_gemm(plan, dA, dB, dC)  # leave the fast result in C
        torch.cuda.synchronize()

    e2e = None
    if not a.no_e2e:
        k_e2e = max(2, a.steps // 2)
        dev_ms, call_ms = [], []
        # the clock sampler covers the whole end-to-end section, host buffer set-up included
        sampler_e2e = ClockSampler(gpu_uuid(torch, dev))
        with sampler_e2e:
            # the library's page-locked buffers (huge-page backed where the host has transparent huge
            # pages): the host link keeps its rate from them after other processes have churned memory
            hA = fmm.host_empty((n, n), torch.float64)
            hB = fmm.host_empty((n, n), torch.float64)
            hC = fmm.host_empty((n, n), torch.float64)
            hA.copy_(torch.from_numpy(A))
            hB.copy_(torch.from_numpy(B))

            def e2e_step():
                if not sharded:
                    fmm.fmm_gemm_host(plan, hA, hB, hC)
                    return
                # every rank copies in both operands, computes its shard, the partials are summed on the
                # device, and rank 0 copies the product back
                dA.copy_(hA, non_blocking=True)
                dB.copy_(hB, non_blocking=True)
                shard_mod.gemm_sharded(plan, dA, dB, dC)
                if rank == 0:
                    hC.copy_(dC, non_blocking=True)
                torch.cuda.synchronize()

            e2e_step()  # the plan's host-path buffers are allocated by the first call
            if dist is not None:
                dist.barrier()
            t0 = time.perf_counter()
            for _ in range(k_e2e):
                tc = time.perf_counter()
                e2e_step()
                call_ms.append((time.perf_counter() - tc) * 1e3)
                dev_ms.append(fmm.fmm_plan_last_kernel_ms(plan)[1])  # the call's device work, copies excluded
            t1 = time.perf_counter()
        te = max_over_ranks((t1 - t0) / k_e2e, dist, dev)
        # the copies alone, same pinned buffers (context for the gap between e2e and device time), and the
        # host link's rate in each direction measured with CUDA events on the same buffers
        torch.cuda.synchronize()
        tc = time.perf_counter()
        dA.copy_(hA, non_blocking=True)
        dB.copy_(hB, non_blocking=True)
        hC.copy_(dC, non_blocking=True)
        torch.cuda.synchronize()
        copy_ms = (time.perf_counter() - tc) * 1e3
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record()
        dA.copy_(hA, non_blocking=True)
        ev[1].record()
        dB.copy_(hB, non_blocking=True)
        ev[2].record()
        hC.copy_(dC, non_blocking=True)
        ev[3].record()
        torch.cuda.synchronize()
        gbs = [n * n * 8 / (ev[i].elapsed_time(ev[i + 1]) * 1e-3) / 1e9 for i in range(3)]
        h2d_gbs, d2h_gbs = min(gbs[0], gbs[1]), gbs[2]
        # context: the same copies from a plain cudaHostAlloc buffer (torch's pinned memory)
        hP = torch.empty((n, n), dtype=torch.float64, pin_memory=True)
        evp = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        evp[0].record()
        dA.copy_(hP, non_blocking=True)
        evp[1].record()
        hP.copy_(dC, non_blocking=True)
        evp[2].record()
        torch.cuda.synchronize()
        gbs_pinned = [n * n * 8 / (evp[i].elapsed_time(evp[i + 1]) * 1e-3) / 1e9 for i in range(2)]
        del hP
        dA.copy_(hA)  # restore the operand the copy above overwrote
        e2e = {"value": (flops_eff / te if sharded else job_throughput(flops_eff, ws, te)) / 1e12, "unit": "TFLOP/s",
               "h2d_bytes_per_step": ws * 2 * n * n * 8, "d2h_bytes_per_step": (1 if sharded else ws) * n * n * 8,
               "ms_per_step": te * 1e3, "steps": k_e2e,
               "device_ms_per_step": statistics.mean(dev_ms), "call_ms": [round(x, 2) for x in call_ms],
               "device_ms": [round(x, 2) for x in dev_ms], "copies_alone_ms": round(copy_ms, 2),
               "h2d_gbs": round(h2d_gbs, 1), "d2h_gbs": round(d2h_gbs, 1),
               "copy_gbs_A_B_C": [round(x, 1) for x in gbs],
               "host_buffers": "fmm_host_alloc (huge pages: %d bytes)" % fmm.fmm_host_huge_page_bytes(),
               "context_cudahostalloc_gbs_h2d_d2h": [round(x, 1) for x in gbs_pinned],
               "clocks": sampler_e2e.summary(),
               "path": "fmm_gemm_host (fmm_host_alloc buffers, copies inside the timed region)" if not sharded else
               "per rank: copies of A and B in, its shard (fmm_gemm), all-reduce of C, rank 0 copies C out"}

    nc = info["n_core"]
    q = n - nc
    if a.dtype == "f64":
        peak, peak_note = fp64_peak_tflops()
        contraction_flops = info["flops_leaf"] + 2.0 * (nc * q * n + q * n * n + nc * nc * q)
        kernel_name = "fmm_f64_kernel"
        extra = {"dmma_peak_measured_here": dmma_peak, "dfma_peak_measured_here": dfma_peak}
        ref_rate = dmma_peak
    else:
        peak, peak_note = fp8_peak_tflops()
        contraction_flops = info["flops_lowp"]
        kernel_name = "ozaki_tc_pair_kernel"
        extra = {"e4m3_mma_sync_peak_measured_here": e4m3_peak, "dmma_peak_measured_here": dmma_peak,
                 "ozaki_slices": info["ozaki_slices"]}
        ref_rate = e4m3_peak
    achieved = contraction_flops / (leaf_ms * 1e-3) / 1e12
    traffic = profile_traffic(kernel_name, workload_name(a))
    roofline = {"bound": "tensor", "kernel": kernel_name, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic, "peak_note": peak_note,
                "algorithmic_flops_per_launch": contraction_flops, "avg_launch_ms": leaf_ms,
                "kernel_share_of_step": leaf_ms / ms if ms > 0 else None,
                "phase_ms": main_phases,
                "frac_of_instruction_rate_measured_here": achieved / ref_rate if ref_rate else None, **extra}

    emulated = None
    if a.dtype == "f64" and not a.no_emulated and not sharded:
        e_algo = fmm.fmm_algo_builtin("strassen")
        e_plan = fmm.fmm_plan_create(n, e_algo, 2, dtype="f64_ozaki", record_kernel_time=True)
        e_ms, e_leaf = time_plan(torch, fmm, e_plan, dA, dB, dC, max(a.warmup, 3), a.steps, dist)
        e_ms = max_over_ranks(e_ms, dist, dev)
        e_info = e_plan.info()
        e_err = oracle_error(A, B, dC[t_rows, t_cols].cpu().numpy(), s_rows, s_cols) if rank == 0 else None
        fp8_peak, fp8_note = fp8_peak_tflops()
        e4m3_rate = fmm.fmm_measure_e4m3_peak()
        e_achieved = e_info["flops_lowp"] / (e_leaf * 1e-3) / 1e12
        emulated = {
            "workload": f"strassen_d2_n{n}_{a.kind}_ozaki{e_info['ozaki_slices']}",
            "value": job_throughput(flops_eff, ws, e_ms * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_step": e_ms,
            "speedup_vs_classic": (flops_eff / (e_ms * 1e-3) / 1e12) / classic["value"] if classic else None,
            "normalised_error_sampled": e_err, "ozaki_slices": e_info["ozaki_slices"],
            "gpu_launches": a.steps * ozaki_launches(e_info["materialize_passes"], e_info["n_core"] < n),
            "roofline": {"bound": "tensor", "kernel": "ozaki_tc_pair_kernel", "achieved": e_achieved, "peak": fp8_peak,
                         "unit": "TFLOP/s", "frac": e_achieved / fp8_peak, "peak_note": fp8_note,
                         "traffic": profile_traffic("ozaki_tc_pair_kernel",
                                                    f"strassen_d2_n{n}_{a.kind}_ozaki{e_info['ozaki_slices']}"),
                         "algorithmic_flops_per_launch": e_info["flops_lowp"], "avg_launch_ms": e_leaf,
                         "kernel_share_of_step": e_leaf / e_ms, "phase_ms": time_plan.last_phases,
                         "e4m3_mma_sync_rate_measured_here": e4m3_rate},
            "note": f"same FP64 operands; S_r/T_r and post-additions in FP64, leaf products from "
                    f"{e_info['ozaki_slices']} e4m3 slices with exact FP32/int64 sums (precision configuration)"}
        fmm.fmm_plan_destroy(e_plan)

    # the batched workload (256 autotuned products of log-uniform size in one CUDA graph), three timed steps
    batched = None
    if a.dtype == "f64" and not a.no_batched and not sharded:
        batched = batched_measurement(torch, fmm, dev, a.batch_count, 3, 3, max_depth=a.batch_max_depth)
        batched["gpu_launches_note"] = "counted separately from the main step's gpu_launches"

    # context only, not on the product path: the vendor FP64 GEMM (cuBLAS DGEMM through torch.matmul)
    dgemm = None
    if not a.no_cublas and not sharded:
        torch.matmul(dA, dB, out=dC)
        torch.cuda.synchronize()
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record()
        for _ in range(3):
            torch.matmul(dA, dB, out=dC)
        c1.record()
        torch.cuda.synchronize()
        ms_blas = c0.elapsed_time(c1) / 3
        dgemm = {"value": flops_eff / (ms_blas * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_step": ms_blas,
                 "path": "torch.matmul float64 (cuBLAS DGEMM), context only"}
        fmm.fmm_gemm(plan, dA, dB, dC)  # leave the fast result in C
        torch.cuda.synchronize()

    # HBM side: measured DRAM bytes of the dominant kernel (single-pass ncu capture) per launch over its
    # live duration, and the algorithmic bytes of the materialized pre-additions over their phase time
    hbm_gbs = (measured_peaks() or {}).get("hbm_gbs") or 6800.0
    phases = main_phases or {}
    hbm = {"peak_gbs": hbm_gbs, "peak_note": "of measured (MEASURED_PEAKS.json hbm_gbs)" if measured_peaks() else
           "of fallback (6.8 TB/s)"}
    if traffic:
        hbm["leaf_kernel_gbs"] = traffic / (leaf_ms * 1e-3) / 1e9
        hbm["leaf_kernel_frac"] = hbm["leaf_kernel_gbs"] / hbm_gbs
    mat_bytes = materialized_bytes(nc, info["p"], info["R_total"], info["depth"], info["materialized_levels"])
    if mat_bytes and phases.get("materialize"):
        hbm["pre_additions_bytes"] = mat_bytes
        hbm["pre_additions_gbs"] = mat_bytes / (phases["materialize"] * 1e-3) / 1e9
        hbm["pre_additions_frac"] = hbm["pre_additions_gbs"] / hbm_gbs

    cpu = None
    if rank == 0 and ws == 1 and not a.no_cpu_baseline:
        times, cores, cdepth = cpu_oracle_run(a, a.cpu_n, 1)
        t = times[0]
        cpu = {"value": 2.0 * a.cpu_n ** 3 / t / 1e12, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
               "sample": f"oracle bilinear ({a.algo}, depth {cdepth}) on one {a.cpu_n}x{a.cpu_n} {a.kind} "
                         f"product, {t:.1f} s on {cores} threads"}
        # the same oracle on one core (the paper's 1-core vs 16-core comparison), on a smaller sample
        n1 = max(2, a.cpu_n // 2)
        times1, _, cdepth1 = cpu_oracle_run(a, n1, 1, threads=1)
        cpu["one_core"] = {"value": 2.0 * n1 ** 3 / times1[0] / 1e12, "unit": "TFLOP/s", "cores": 1,
                           "sample": f"oracle bilinear ({a.algo}, depth {cdepth1}) on one {n1}x{n1} {a.kind} "
                                     f"product, {times1[0]:.1f} s on 1 thread"}
        import oracle

        oracle.set_num_threads(cores)

    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": ws, "steps": a.steps,
        "warmup": max(a.warmup, 3), "ms_per_step": ms, "higher_is_better": True,
        "scaling": "strong" if sharded else "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(a), "n": n, "algorithm": a.algo, "depth": a.depth,
                   "leaf": "fp64 DMMA" if a.dtype == "f64" else f"emulated FP64, {info['ozaki_slices']} e4m3 slices",
                   "schedule": a.schedule, "materialized_levels": info["materialized_levels"],
                   "leaf_m": info["m"], "products": info["R_total"], "entries": a.kind,
                   "l2": "inputs 3 x %.0f MiB > L2 (129 MB), no flush" % (n * n * 8 / 2 ** 20),
                   "parallelism": f"{ws} GPUs, leaf products sharded (ranges {info['product_begin']}.."
                                  f"{info['product_end']} on rank {rank}), one all-reduce of C per step"
                   if sharded else "single GPU"},
        "classic_depth0": classic,
        "speedup_vs_classic": value / classic["value"] if classic else None,
        "context_cublas_dgemm": dgemm,
        "hbm": hbm,
        "normalised_error_sampled": err,
        "clocks": clocks,
        "e2e": e2e,
        "gpu_launches": a.steps * ozaki_launches(info["materialize_passes"], q > 0) if a.dtype == "f64_ozaki"
        else a.steps * f64_launches(info, q > 0),
        "roofline": roofline,
        "emulated_fp64": emulated,
        "batched": batched,
        "cpu_baseline": cpu,
        "flops_executed_per_step": info["flops_executed"],
        "executed_tflops": info["flops_executed"] / (ms * 1e-3) / 1e12,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    fmm.fmm_plan_destroy(plan)
    if dist is not None:
        dist.destroy_process_group()
    _ = np
    return 0


def main(argv=None):
    a = parse_args(argv)
    if a.impl == "reference":
        return run_reference(a)
    if a.sweep:
        return run_sweep(a)
    if a.batched:
        return run_batched(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())
