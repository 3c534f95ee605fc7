"""Product sharding across ranks, on the CPU: two gloo ranks each take their shard of the flattened leaf
products (the library's partition, fmm_shard_range), form the partial C = sum over their own products of
W[l][r] P_r with the oracle computing every leaf product, and sum the partials with the same reduction the
GPU path uses (paper_2312_12732_gb300.sharded.reduce_partials).  Integer inputs must give the exact
product on both ranks.  Also checks the partition itself: contiguous, ordered, covering, balanced."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("units,world", [(49, 2), (49, 3), (7, 7), (2401, 8), (1, 1), (0, 3), (10, 4)])
def test_shard_ranges_cover_in_order_and_balance(units, world):
    from paper_2312_12732_gb300 import _build

    _build.build()
    import paper_2312_12732_gb300 as fmm

    ranges = [fmm.fmm_shard_range(units, world, k) for k in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == units
    for (b0, e0), (b1, e1) in zip(ranges, ranges[1:]):
        assert e0 == b1
    sizes = [e - b for b, e in ranges]
    assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 0
    with pytest.raises(fmm.FmmError):
        fmm.fmm_shard_range(units, world, world)


def _partial_product(A, B, p, U, V, W, begin, end):
    """sum over products r in [begin, end) of W[l][r] (S_r T_r), blocks on the p x p grid, leaf products
    by the oracle's classic loop."""
    import oracle

    n = A.shape[0]
    m = n // p
    blk = lambda X, i: X[(i // p) * m:(i // p + 1) * m, (i % p) * m:(i % p + 1) * m]
    C = np.zeros_like(A)
    for r in range(begin, end):
        S = sum(U[i, r] * blk(A, i) for i in range(p * p) if U[i, r])
        T = sum(V[j, r] * blk(B, j) for j in range(p * p) if V[j, r])
        P = oracle.classic(S, T)
        for l in range(p * p):
            if W[l, r]:
                blk(C, l)[...] += W[l, r] * P
    return C


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist

    for p in (ROOT, os.path.join(ROOT, "tests")):
        sys.path.insert(0, p)
    from golden import algos

    import oracle
    from paper_2312_12732_gb300 import _build, inputs, sharded

    _build.build()
    import paper_2312_12732_gb300 as fmm

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        s = algos.paper_strassen()
        p, U, V, W = algos.kron_compose(s, s)  # two Strassen levels flattened: <4,4,4;49>
        n = 64
        A, B = inputs.operands(n, "integer", seed=77)
        begin, end = fmm.fmm_shard_range(U.shape[1], world, rank)
        C = torch.from_numpy(_partial_product(A, B, p, U, V, W, begin, end))
        sharded.reduce_partials(C)
        ok = bool(np.array_equal(C.numpy(), oracle.classic(A, B)))
        q.put((rank, begin, end, ok))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_sum_their_shards_to_the_exact_product():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert [(g[1], g[2]) for g in got] == [(0, 24), (24, 49)]
    assert all(g[3] for g in got)
