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

or, with a plan created on first use and kept for later calls of the same shape::

    C = fmm.gemm(A, B, "strassen", depth=2)
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
    fmm_algo_rational_brent_mismatches,
    fmm_algo_rect_as_square,
    fmm_algo_rect_brent_mismatches,
    fmm_algo_rect_builtin,
    fmm_algo_rect_classic,
    fmm_algo_rect_compose,
    fmm_algo_rect_cyclic,
    fmm_algo_rect_transpose,
    RationalAlgo,
    RectAlgo,
    fmm_gemm,
    fmm_gemm_batched,
    fmm_gemm_ex,
    fmm_gemm_f32_ex,
    fmm_gemm_host,
    fmm_host_alloc,
    fmm_host_free,
    fmm_host_huge_page_bytes,
    host_empty,
    fmm_debug_fail_allocation,
    fmm_debug_live_allocations,
    fmm_gemm_noalloc,
    fmm_noalloc_set_debug,
    fmm_noalloc_sync_status,
    fmm_plan_create,
    fmm_plan_destroy,
    fmm_plan_get_info,
    fmm_plan_last_kernel_ms,
    fmm_plan_last_phase_ms,
    fmm_measure_e4m3_peak,
    fmm_measure_fp64_peak,
    fmm_plan_workspace_bytes,
    fmm_shard_range,
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


_PLANS = {}


def gemm(A, B, algo="strassen", depth=1, dtype="f64", out=None, stream=None, alpha=1.0, beta=0.0):
    """C = alpha * A @ B + beta * out for square float64, complex128 or float32 CUDA tensors by the
    bilinear algorithm ``algo`` (a built-in name, ``"name^k"`` for its k-th Kronecker power, or an
    :class:`Algo`) at recursion ``depth``.  Complex operands use the "c128" plan (or "c128_3m" when
    asked for), float32 operands the "f32" plan.

    The plan for (n, algorithm, depth, dtype, device) is created on first use and cached; a cached
    plan's workspace serves one call at a time, so calls on different streams that share a plan
    must not overlap.  ``out`` (optional) receives the result; otherwise a new tensor does, and
    ``beta`` must then be 0.
    """
    import torch

    if not isinstance(A, torch.Tensor) or A.dim() != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("A must be a square 2-D torch.Tensor")
    n = A.shape[0]
    if out is None and beta != 0.0:
        raise ValueError("beta != 0 needs out")
    if A.is_complex() and dtype not in ("c128", "c128_3m"):
        dtype = "c128"  # complex operands: four real fast products unless "c128_3m" is asked for
    if A.dtype == torch.float32:
        dtype = "f32"
    if isinstance(algo, str):
        name, _, k = algo.partition("^")
        alg = algorithm(name, int(k) if k else 1)
        key_algo = algo
    else:
        alg = algo
        key_algo = (alg.p, alg.U.tobytes(), alg.V.tobytes(), alg.W.tobytes(), getattr(alg, "dens", None))
    key = (n, key_algo, depth, dtype, A.device.index)
    plan = _PLANS.get(key)
    if plan is None:
        with torch.cuda.device(A.device):
            plan = fmm_plan_create(n, alg, depth, dtype=dtype)
        _PLANS[key] = plan
    C = out if out is not None else torch.empty_like(A)
    if alpha == 1.0 and beta == 0.0:
        fmm_gemm(plan, A, B, C, stream)
    else:
        fmm_gemm_ex(plan, alpha, A, B, beta, C, stream)
    return C
