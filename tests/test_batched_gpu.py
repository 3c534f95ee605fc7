"""GPU tests of the grouped batched launch, its CUDA-graph capture and the autotuner."""
import numpy as np
import pytest

from paper_2312_12732_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fmm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_12732_gb300 import _build

    _build.build()
    import paper_2312_12732_gb300 as m

    return m


def nerr(C, ref, A, B):
    n = A.shape[0]
    return float(np.max(np.abs(C - ref)) / (n * np.abs(A).max() * np.abs(B).max()))


def make_batch(fmm, sizes, kind, picks=None):
    plans, As, Bs, Cs, host = [], [], [], [], []
    for i, n in enumerate(sizes):
        name, depth = picks[i] if picks else (("strassen", 1) if n >= 256 else ("strassen", 0))
        plans.append(fmm.fmm_plan_create(n, fmm.fmm_algo_builtin(name), depth))
        A, B = inputs.operands(n, kind, seed=100 + 2 * i)
        host.append((A, B))
        As.append(torch.from_numpy(A).cuda())
        Bs.append(torch.from_numpy(B).cuda())
        Cs.append(torch.full_like(As[-1], float("nan")))
    return plans, As, Bs, Cs, host


def test_graph_replay_matches_oracle_and_direct_launch(fmm, oracle_mod):
    sizes = inputs.batch_sizes(24, 128, 700, seed=5)
    plans, As, Bs, Cs, host = make_batch(fmm, sizes, "integer")
    g = fmm.fmm_batch_graph_create(plans, As, Bs, Cs)
    for _ in range(2):  # replays reset their counters themselves
        for C in Cs:
            C.fill_(float("nan"))
        fmm.fmm_batch_graph_launch(g)
        torch.cuda.synchronize()
        assert fmm.fmm_sync_status(plans[0]) == 0
        for (A, B), C in zip(host, Cs):
            assert np.array_equal(C.cpu().numpy(), oracle_mod.classic(A, B))


def test_graph_replay_real_inputs(fmm, oracle_mod):
    sizes = [130, 257, 512, 999]
    plans, As, Bs, Cs, host = make_batch(fmm, sizes, "uniform")
    g = fmm.fmm_batch_graph_create(plans, As, Bs, Cs)
    fmm.fmm_batch_graph_launch(g)
    torch.cuda.synchronize()
    for (A, B), C, p in zip(host, Cs, plans):
        ref = oracle_mod.bilinear(A, B, p.algo.p, p.algo.U, p.algo.V, p.algo.W, p.depth) if p.depth else \
            oracle_mod.classic(A, B)
        assert nerr(C.cpu().numpy(), ref, A, B) <= 1e-13


def test_batched_rejects_repeated_plan(fmm):
    p = fmm.fmm_plan_create(64, fmm.fmm_algo_builtin("strassen"), 1)
    A = torch.zeros(64, 64, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        fmm.fmm_gemm_batched([p, p], [A, A], [A, A], [A.clone(), A.clone()])


def test_autotuner_picks_a_valid_choice(fmm):
    from paper_2312_12732_gb300 import autotune

    algos = [fmm.fmm_algo_builtin("strassen"), fmm.fmm_algo_builtin("winograd")]
    algo, depth, ms = fmm.fmm_autotune(1024, algos, max_depth=3, min_leaf=128)
    assert algo.name in ("strassen", "winograd") and 0 <= depth <= 3 and ms > 0
    name, d, ms2 = autotune.choose(300)
    assert name in ("strassen", "winograd") and 0 <= d <= 1
    plans, picks = autotune.plan_batch([150, 300, 2000])
    assert len(plans) == 3 and all(p.depth == k[1] for p, k in zip(plans, picks))
