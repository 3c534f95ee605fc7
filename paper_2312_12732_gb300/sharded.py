"""One fast multiplication sharded across GPUs by its leaf products.

The R^depth leaf products P_r = S_r T_r of a bilinear algorithm are independent (Section 2: each product
of the recursion can be computed on its own), and C_l = sum_r W[l][r] P_r is linear in them.  So with one
process per GPU, rank k plans shard k of the products (``shard_count`` = world size, see
fmm_plan_options_t): its plan forms the pre-additions of its own products from its full copy of A and B,
multiplies them, and leaves in C the partial sum over its own products (zero where they do not reach; the
rank holding product 0 also computes the peel fix-ups of a non-divisible n).  One all-reduce (sum) of the
partial C's over the ranks then gives C = A B on every rank.  That sum is the only exchange; it runs
through ``torch.distributed`` (NCCL between GPUs), after the plan's kernels on the same stream.
"""
from __future__ import annotations

from . import _binding as B


def world():
    """(rank, world size) of the default process group, (0, 1) without one."""
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized():
        return dist.get_rank(), dist.get_world_size()
    return 0, 1


def plan_shard(n: int, algo, depth: int, rank: int | None = None, world_size: int | None = None, **opts):
    """This rank's plan: shard ``rank`` of ``world_size`` (default: the process group's) of the leaf
    products of ``depth`` levels of ``algo``; an unsharded plan for one rank."""
    r0, w0 = world()
    rank = r0 if rank is None else rank
    world_size = w0 if world_size is None else world_size
    if world_size <= 1:
        return B.fmm_plan_create(n, algo, depth, **opts)
    return B.fmm_plan_create(n, algo, depth, shard_count=world_size, shard_index=rank, **opts)


def reduce_partials(C, group=None):
    """Sums the ranks' partial products in place (all-reduce over ``group``); a no-op on one rank."""
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(C, op=dist.ReduceOp.SUM, group=group)
    return C


def gemm_sharded(plan, A, Bm, C, group=None, stream=None):
    """C = A @ B on every rank: this rank's shard of the products into C, then the sum over the ranks.
    A and B are the full operands on every rank; C is overwritten."""
    import torch

    B.fmm_gemm(plan, A, Bm, C, stream)
    if stream is not None:
        with torch.cuda.stream(stream):
            return reduce_partials(C, group)
    return reduce_partials(C, group)
