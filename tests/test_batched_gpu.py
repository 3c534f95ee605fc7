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


def median_ms(fmm, plan, n, reps=5):
    A = torch.rand(n, n, dtype=torch.float64, device="cuda")
    B = torch.rand(n, n, dtype=torch.float64, device="cuda")
    C = torch.empty_like(A)
    fmm.fmm_gemm(plan, A, B, C)
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fmm.fmm_gemm(plan, A, B, C)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    assert fmm.fmm_sync_status(plan) == 0
    return sorted(times)[reps // 2]


@pytest.mark.parametrize("n", [1024, 2896])
def test_autotuner_pick_is_no_slower_than_the_classic_product(fmm, n):
    """The tuner searches algorithm, depth, tile width and schedule; re-timed independently (median of 5),
    its pick is no slower than the best depth-0 configuration at the same size."""
    algos = [fmm.fmm_algo_builtin("strassen"), fmm.fmm_algo_builtin("winograd")]
    r = fmm.fmm_autotune(n, algos, max_depth=3, min_leaf=128)
    assert r["algo"].name in ("strassen", "winograd") and 0 <= r["depth"] <= 3
    assert r["tile_n"] in (64, 128) and r["schedule"] in ("auto", "fused")
    assert r["candidates"] >= 2 + 2 * 4  # depth 0 at both tiles, and both algorithms at depth 1 (x2 x2)
    assert r["ms"] <= r["depth0_ms"]
    pick = fmm.fmm_plan_create(n, r["algo"], r["depth"], schedule=r["schedule"], tile_n=r["tile_n"])
    t_pick = median_ms(fmm, pick, n)
    t_classic = min(median_ms(fmm, fmm.fmm_plan_create(n, algos[0], 0, tile_n=t), n) for t in (64, 128))
    assert t_pick <= 1.05 * t_classic, (r, t_pick, t_classic)


def test_autotune_choice_is_cached_in_memory_and_on_disk(fmm, monkeypatch, tmp_path):
    from paper_2312_12732_gb300 import autotune

    autotune._memo.clear()
    path = str(tmp_path / "tune.json")
    first = autotune.choose(300, cache_path=path)
    assert first["algo"] in ("strassen", "winograd") and 0 <= first["depth"] <= 1
    count = autotune.tuned_count
    again = autotune.choose(310, cache_path=path)  # same half-octave bucket: from memory
    assert autotune.tuned_count == count and again == first

    def must_not_tune(*a, **k):
        raise AssertionError("a cached choice was tuned again")

    autotune._memo.clear()
    monkeypatch.setattr(autotune.B, "fmm_autotune", must_not_tune)
    from_disk = autotune.choose(300, cache_path=path)  # a fresh memo reads the file
    assert from_disk == first
    plans, picks = autotune.plan_batch([300, 305], cache_path=path)
    assert all(p.info()["tile_n"] == first["tile_n"] and p.depth == first["depth"] for p in plans)


def test_force_depth_and_plan_log(fmm, monkeypatch, capfd):
    """FMM_FORCE_DEPTH restricts the tuner to one depth; FMM_LOG=2 logs each plan and each multiplication."""
    algos = [fmm.fmm_algo_builtin("strassen"), fmm.fmm_algo_builtin("winograd")]
    monkeypatch.setenv("FMM_FORCE_DEPTH", "2")
    r = fmm.fmm_autotune(1024, algos, max_depth=3, min_leaf=128)
    assert r["depth"] == 2 and r["depth0_ms"] > 1e29 and r["candidates"] >= 4
    monkeypatch.delenv("FMM_FORCE_DEPTH")
    monkeypatch.setenv("FMM_LOG", "2")
    capfd.readouterr()
    plan = fmm.fmm_plan_create(512, algos[0], 1)
    A = torch.ones(512, 512, dtype=torch.float64, device="cuda")
    C = torch.empty_like(A)
    fmm.fmm_gemm(plan, A, A, C)
    assert fmm.fmm_sync_status(plan) == 0
    err = capfd.readouterr().err
    assert "fmm: fmm_plan_create n=512 p=2 R=7 depth=1 dtype=f64 leaf=256 products=0..7" in err, err
    assert "fmm: gemm n=512 depth=1 dtype=f64" in err, err
    assert bool(torch.all(C == 512.0))
