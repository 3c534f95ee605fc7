"""GB300-native fast FP64 matrix multiplication by recursive bilinear algorithms
(D'Alberto, "Strassen's Matrix Multiplication Algorithm Is Still Faster",
arXiv 2312.12732).

The C ABI (``include/fmm.h``) is the product; this package is its thin
binding (``_binding``) plus seeded workload generators (``inputs``) and the
build step (``_build``).  Importing the package loads nothing; the shared
library is opened on first use and its absence is an error.

Typical use::

    import torch, paper_2312_12732_gb300 as fmm
    algo = fmm.fmm_algo_builtin("strassen")
    plan = fmm.fmm_plan_create(8192, algo, depth=2)
    fmm.fmm_gemm(plan, A, B, C)          # A, B, C: float64 CUDA tensors
"""
from ._binding import (  # noqa: F401
    Algo,
    BatchGraph,
    fmm_autotune,
    fmm_batch_graph_create,
    fmm_batch_graph_destroy,
    fmm_batch_graph_launch,
    FmmError,
    Plan,
    fmm_algo_brent_mismatches,
    fmm_algo_builtin,
    fmm_algo_compose,
    fmm_algo_from_transposed_c,
    fmm_gemm,
    fmm_gemm_batched,
    fmm_gemm_host,
    fmm_gemm_noalloc,
    fmm_plan_create,
    fmm_plan_destroy,
    fmm_plan_get_info,
    fmm_plan_last_kernel_ms,
    fmm_plan_last_phase_ms,
    fmm_measure_e4m3_peak,
    fmm_measure_fp64_peak,
    fmm_plan_workspace_bytes,
    fmm_status_string,
    fmm_sync_status,
    lib,
)


def algorithm(name: str, power: int = 1):
    """A built-in algorithm, optionally Kronecker-composed with itself ``power`` times
    (e.g. ``algorithm("strassen", 2)`` is <4,4,4;49>)."""
    a = fmm_algo_builtin(name)
    out = a
    for _ in range(power - 1):
        out = fmm_algo_compose(out, a)
    return out
