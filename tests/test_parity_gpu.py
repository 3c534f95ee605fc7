"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bar (fixed in advance, from the method's error behaviour):
  * integer-valued inputs (entries in [-16, 16]): bit-exact, because every
    intermediate is an integer below 2^53 (abstract of the paper: integer
    computations come out exact);
  * real inputs: normalised error max|C - C_ref| / (n max|A| max|B|) <= 1e-13
    at depth <= 2 and <= 1e-12 at depth 3-4, with C_ref the oracle's
    recursive evaluation of the same algorithm (or its classic product at
    depth 0), or Dot2 reference entries on large sizes.
"""
import numpy as np
import pytest

from paper_2312_12732_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def tol(depth):
    return 1e-13 if depth <= 2 else 1e-12


@pytest.fixture(scope="module")
def fmm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_12732_gb300 import _build

    _build.build()
    import paper_2312_12732_gb300 as m

    return m


def run(fmm, plan, A, B):
    dA = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(B).cuda()
    dC = torch.full_like(dA, float("nan"))
    fmm.fmm_gemm(plan, dA, dB, dC)
    st = fmm.fmm_sync_status(plan)
    assert st == 0, fmm.fmm_status_string(st)
    return dC.cpu().numpy()


def nerr(C, ref, A, B):
    n = A.shape[0]
    return float(np.max(np.abs(C - ref)) / (n * np.abs(A).max() * np.abs(B).max()))


def oracle_ref(oracle_mod, A, B, algo, depth):
    if depth == 0:
        return oracle_mod.classic(A, B)
    return oracle_mod.bilinear(A, B, algo.p, algo.U, algo.V, algo.W, depth)


@pytest.mark.parametrize("n", [1, 2, 7, 64, 127, 128, 129, 300, 512])
def test_classic_depth0(fmm, oracle_mod, n):
    algo = fmm.fmm_algo_builtin("strassen")
    plan = fmm.fmm_plan_create(n, algo, 0)
    A, B = inputs.operands(n, "integer", seed=n)
    assert np.array_equal(run(fmm, plan, A, B), oracle_mod.classic(A, B))
    A, B = inputs.operands(n, "uniform", seed=n)
    assert nerr(run(fmm, plan, A, B), oracle_mod.classic(A, B), A, B) <= tol(0)


def test_strassen_n512_depth1_vs_classic(fmm, oracle_mod):
    """The small configuration: n = 512, Strassen one level (leaf 256) vs the classic product."""
    algo = fmm.fmm_algo_builtin("strassen")
    plan = fmm.fmm_plan_create(512, algo, 1)
    assert plan.info()["m"] == 256
    A, B = inputs.operands(512, "integer", seed=1)
    C = run(fmm, plan, A, B)
    assert np.array_equal(C, oracle_mod.classic(A, B))
    assert np.array_equal(C, oracle_ref(oracle_mod, A, B, algo, 1))
    A, B = inputs.operands(512, "uniform", seed=1)
    C = run(fmm, plan, A, B)
    assert nerr(C, oracle_ref(oracle_mod, A, B, algo, 1), A, B) <= 1e-13
    assert nerr(C, oracle_mod.classic(A, B), A, B) <= 1e-13


CASES = [
    ("strassen", 1, 512, "fused"), ("strassen", 2, 512, "fused"), ("strassen", 3, 1024, "fused"),
    ("strassen", 2, 1024, "hybrid1"), ("strassen", 3, 1024, "auto"), ("strassen", 4, 1024, "auto"),
    ("winograd", 1, 512, "auto"), ("winograd", 2, 1024, "fused"), ("winograd", 3, 1024, "auto"),
    ("strassen1969", 2, 512, "auto"),
    ("laderman", 1, 576, "fused"), ("laderman", 1, 576, "auto"), ("laderman", 2, 576, "auto"),
    ("strassen^2", 1, 512, "fused"), ("strassen^2", 2, 1024, "auto"), ("classic2", 2, 512, "auto"),
]


def make_algo(fmm, name):
    if name.endswith("^2"):
        return fmm.algorithm(name[:-2], 2)
    return fmm.fmm_algo_builtin(name)


def make_plan(fmm, n, algo, depth, sched):
    if sched.startswith("hybrid"):
        return fmm.fmm_plan_create(n, algo, depth, schedule="hybrid", materialize_levels=int(sched[6:]))
    return fmm.fmm_plan_create(n, algo, depth, schedule=sched)


@pytest.mark.parametrize("name,depth,n,sched", CASES)
def test_fast_algorithms(fmm, oracle_mod, name, depth, n, sched):
    algo = make_algo(fmm, name)
    plan = make_plan(fmm, n, algo, depth, sched)
    A, B = inputs.operands(n, "integer", seed=depth + n)
    assert np.array_equal(run(fmm, plan, A, B), oracle_mod.classic(A, B))
    A, B = inputs.operands(n, "uniform", seed=depth)
    C = run(fmm, plan, A, B)
    assert nerr(C, oracle_ref(oracle_mod, A, B, algo, depth), A, B) <= tol(depth)


@pytest.mark.parametrize("n,depth,sched", [(1000, 1, "auto"), (1031, 1, "fused"), (1031, 2, "auto"),
                                           (777, 3, "auto"), (777, 3, "fused"), (3, 1, "auto"), (5, 2, "fused"),
                                           (129, 3, "auto"), (3001, 3, "auto")])
def test_peeled_sizes(fmm, oracle_mod, n, depth, sched):
    algo = fmm.fmm_algo_builtin("strassen")
    plan = make_plan(fmm, n, algo, depth, sched)
    info = plan.info()
    assert info["n_core"] == info["P"] * info["m"] and info["n_core"] <= n
    A, B = inputs.operands(n, "integer", seed=n)
    assert np.array_equal(run(fmm, plan, A, B), oracle_mod.classic(A, B))
    A, B = inputs.operands(n, "normal", seed=n)
    assert nerr(run(fmm, plan, A, B), oracle_ref(oracle_mod, A, B, algo, depth), A, B) <= tol(depth)


def test_repeat_runs_are_bitwise_identical(fmm):
    algo = fmm.fmm_algo_builtin("strassen")
    plan = fmm.fmm_plan_create(1024, algo, 2, schedule="fused")
    A, B = inputs.operands(1024, "normal", seed=3)
    C1 = run(fmm, plan, A, B)
    C2 = run(fmm, plan, A, B)
    assert np.array_equal(C1, C2)


@pytest.mark.parametrize("name,depth", [("strassen", 2), ("winograd", 3)])
def test_full_size_sampled_n8192(fmm, oracle_mod, name, depth):
    """n = 8192 in the launch configuration the benchmark times; 4096 Dot2 samples."""
    n = 8192
    algo = fmm.fmm_algo_builtin(name)
    plan = fmm.fmm_plan_create(n, algo, depth)
    rows, cols = inputs.sample_indices(n, 4096, seed=11)
    for kind in ("integer", "uniform"):
        A, B = inputs.operands(n, kind, seed=5)
        C = run(fmm, plan, A, B)
        ref = oracle_mod.sample_dot2(A, B, rows, cols)
        if kind == "integer":
            assert np.array_equal(C[rows, cols], ref)
        else:
            assert nerr(C[rows, cols], ref, A, B) <= tol(depth)


def test_laderman_n6912_sampled(fmm, oracle_mod):
    n = 6912
    algo = fmm.fmm_algo_builtin("laderman")
    plan = fmm.fmm_plan_create(n, algo, 2)
    assert plan.info()["m"] == 768
    A, B = inputs.operands(n, "uniform", seed=8)
    C = run(fmm, plan, A, B)
    rows, cols = inputs.sample_indices(n, 4096, seed=12)
    assert nerr(C[rows, cols], oracle_mod.sample_dot2(A, B, rows, cols), A, B) <= tol(2)


def test_wait_timeout_is_reported_and_context_survives(fmm, oracle_mod):
    """One ordering counter is set to a value no task writes: its waiters give up
    after the bounded wait, the plan reports FMM_ERR_TIMEOUT, and the device
    stays usable."""
    algo = fmm.fmm_algo_builtin("strassen")
    plan = fmm.fmm_plan_create(256, algo, 1, schedule="fused", wait_timeout_s=0.05, debug_poison_chain=1)
    A, B = inputs.operands(256, "integer", seed=2)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.empty_like(dA)
    fmm.fmm_gemm(plan, dA, dB, dC)
    assert fmm.fmm_sync_status(plan) == 6
    good = fmm.fmm_plan_create(256, algo, 1)
    assert np.array_equal(run(fmm, good, A, B), oracle_mod.classic(A, B))


def test_batched_grouped_launch(fmm, oracle_mod):
    specs = [(300, "strassen", 1), (512, "winograd", 2), (128, "strassen", 0), (700, "laderman", 1),
             (257, "strassen", 2), (1024, "strassen", 3)]
    plans, As, Bs, Cs, host = [], [], [], [], []
    for i, (n, name, depth) in enumerate(specs):
        algo = fmm.fmm_algo_builtin(name)
        plans.append(fmm.fmm_plan_create(n, algo, depth))
        A, B = inputs.operands(n, "integer" if i % 2 else "uniform", seed=40 + i)
        host.append((A, B, algo, depth))
        As.append(torch.from_numpy(A).cuda())
        Bs.append(torch.from_numpy(B).cuda())
        Cs.append(torch.full_like(As[-1], float("nan")))
    fmm.fmm_gemm_batched(plans, As, Bs, Cs)
    assert fmm.fmm_sync_status(plans[0]) == 0
    for i, (A, B, algo, depth) in enumerate(host):
        C = Cs[i].cpu().numpy()
        if i % 2:
            assert np.array_equal(C, oracle_mod.classic(A, B))
        else:
            assert nerr(C, oracle_ref(oracle_mod, A, B, algo, depth), A, B) <= tol(depth)


def test_composed_levels_materialize_by_factors(fmm):
    """<4,4,4;49> = Strassen x Strassen: the planner forms each 4x4 level in two Strassen steps, so
    depth 2 of the composed algorithm and depth 4 of Strassen execute the same adds and, with the same
    operation order in every step, give bit-identical results on real inputs."""
    n = 1024
    comp = fmm.algorithm("strassen", 2)
    p_comp = fmm.fmm_plan_create(n, comp, 2)
    p_str = fmm.fmm_plan_create(n, fmm.fmm_algo_builtin("strassen"), 4)
    i_comp, i_str = p_comp.info(), p_str.info()
    assert i_comp["flops_executed"] == i_str["flops_executed"]
    assert i_comp["R_total"] == i_str["R_total"] == 2401
    A, B = inputs.operands(n, "uniform", seed=31)
    assert np.array_equal(run(fmm, p_comp, A, B), run(fmm, p_str, A, B))


@pytest.mark.parametrize("first,second,depth,n", [("laderman", "strassen", 1, 576), ("strassen", "laderman", 1, 576),
                                                  ("strassen", "winograd", 2, 576)])
def test_mixed_compositions(fmm, oracle_mod, first, second, depth, n):
    """Kronecker products of different algorithms (p = 6, R = 161 and p = 4, R = 49 mixed): the
    planner splits their levels into unequal factors; results match the oracle's recursion on the
    composed tables."""
    algo = fmm.fmm_algo_compose(fmm.fmm_algo_builtin(first), fmm.fmm_algo_builtin(second))
    plan = fmm.fmm_plan_create(n, algo, depth)
    A, B = inputs.operands(n, "integer", seed=n + depth)
    assert np.array_equal(run(fmm, plan, A, B), oracle_mod.classic(A, B))
    A, B = inputs.operands(n, "uniform", seed=depth + 5)
    assert nerr(run(fmm, plan, A, B), oracle_ref(oracle_mod, A, B, algo, depth), A, B) <= tol(depth)


@pytest.mark.parametrize("name,power,depth,passes", [("strassen", 1, 1, 1), ("strassen", 1, 2, 1), ("strassen", 1, 3, 2),
                                                     ("strassen", 2, 2, 2), ("laderman", 1, 2, 2),
                                                     ("winograd", 1, 4, 2)])
def test_materialization_passes(fmm, name, power, depth, passes):
    """Pairs of 2 x 2 steps (Strassen-like factors) are formed in one pass; other steps one pass each."""
    algo = fmm.algorithm(name, power)
    n = algo.p ** depth * 8
    assert fmm.fmm_plan_create(n, algo, depth, schedule="hybrid", materialize_levels=depth).info()[
        "materialize_passes"] == passes


def test_gemm_convenience(fmm, oracle_mod):
    """fmm.gemm creates a plan on first use, reuses it, accepts '<name>^k' and checks its operands."""
    n = 256
    A, B = inputs.operands(n, "integer", seed=77)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    C1 = fmm.gemm(dA, dB, "strassen", depth=2)
    C2 = fmm.gemm(dA, dB, "strassen^2", depth=1, out=torch.empty_like(dA))
    C3 = fmm.gemm(dA, dB, "strassen", depth=2)
    ref = oracle_mod.classic(A, B)
    for C in (C1, C2, C3):
        assert np.array_equal(C.cpu().numpy(), ref)
    assert len([k for k in fmm._PLANS if k[0] == n]) >= 2
    with pytest.raises(ValueError):
        fmm.gemm(dA.float(), dB)
