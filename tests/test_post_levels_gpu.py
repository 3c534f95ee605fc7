"""GPU parity of FP64 plans whose leaf products are stored and whose post-additions run level by
level (fmm_plan_options_t.post_additions = 2).

Section 2 forms each recursion level's C blocks from the R products of the level below
(equation `eq:recursion`); the flattened sum C_l = sum_r W[l][r] P_r over all levels is the same
result with another summation order.  The stored form writes every P_r once and sums the Kronecker
factors of W from the leaf upwards, two 2 x 2 factors per pass where it can.  Bar, as for the
fused epilogue: integer-valued inputs bit-exact against the classic product; real inputs within
the depth's normalised tolerance of the oracle's recursion; the scaled form alpha A B + beta C
bit-exact on integers with small integer scalars.
"""
import numpy as np
import pytest

from golden import rational_algos
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


def run(fmm, plan, A, B, alpha=1.0, beta=0.0, C0=None):
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.full_like(dA, float("nan")) if C0 is None else torch.from_numpy(np.array(C0)).cuda()
    fmm.fmm_gemm_ex(plan, alpha, dA, dB, beta, dC)
    st = fmm.fmm_sync_status(plan)
    assert st == 0, fmm.fmm_status_string(st)
    return dC.cpu().numpy()


def nerr(C, ref, A, B):
    n = A.shape[0]
    return float(np.max(np.abs(C - ref)) / (n * np.abs(A).max() * np.abs(B).max()))


def make_algo(fmm, name):
    if name.endswith("^2"):
        return fmm.algorithm(name[:-2], 2)
    if "*" in name:
        a, b = name.split("*")
        return fmm.fmm_algo_compose(fmm.fmm_algo_builtin(a), fmm.fmm_algo_builtin(b))
    return fmm.fmm_algo_builtin(name)


# (algorithm, depth, n, passes): W's factors over all levels, summed two 2 x 2 factors at a time
CASES = [
    ("strassen", 1, 512, 1), ("strassen", 2, 1024, 1), ("strassen", 3, 1024, 2), ("strassen", 4, 1024, 2),
    ("strassen", 5, 1024, 3), ("winograd", 2, 1024, 1), ("winograd", 3, 1000, 2), ("strassen1969", 2, 512, 1),
    ("laderman", 1, 576, 1), ("laderman", 2, 576, 2), ("strassen^2", 1, 512, 1), ("strassen^2", 2, 1024, 2),
    ("classic2", 2, 512, 1), ("laderman*strassen", 1, 576, 2), ("strassen*laderman", 1, 576, 2),
]


@pytest.mark.parametrize("name,depth,n,passes", CASES)
def test_level_passes_match_the_oracle(fmm, oracle_mod, name, depth, n, passes):
    algo = make_algo(fmm, name)
    plan = fmm.fmm_plan_create(n, algo, depth, post_additions="levels")
    assert plan.info()["post_passes"] == passes
    A, B = inputs.operands(n, "integer", seed=depth + n)
    assert np.array_equal(run(fmm, plan, A, B), oracle_mod.classic(A, B))
    A, B = inputs.operands(n, "uniform", seed=depth)
    C = run(fmm, plan, A, B)
    assert nerr(C, oracle_mod.bilinear(A, B, algo.p, algo.U, algo.V, algo.W, depth), A, B) <= tol(depth)


@pytest.mark.parametrize("n,depth,sched", [(1000, 1, "auto"), (1031, 1, "fused"), (1031, 2, "auto"),
                                           (777, 3, "auto"), (777, 3, "fused"), (3, 1, "auto"), (5, 2, "fused"),
                                           (129, 3, "auto"), (3001, 3, "auto"), (67, 5, "auto")])
def test_peeled_sizes(fmm, oracle_mod, n, depth, sched):
    """Border products run in the leaf launch; the rank-q fix-ups add into C after the last pass."""
    algo = fmm.fmm_algo_builtin("strassen")
    plan = fmm.fmm_plan_create(n, algo, depth, schedule=sched, post_additions="levels")
    info = plan.info()
    assert info["n_core"] == info["P"] * info["m"] and info["n_core"] <= n
    A, B = inputs.operands(n, "integer", seed=n)
    assert np.array_equal(run(fmm, plan, A, B), oracle_mod.classic(A, B))
    A, B = inputs.operands(n, "normal", seed=n)
    assert nerr(run(fmm, plan, A, B), oracle_mod.bilinear(A, B, algo.p, algo.U, algo.V, algo.W, depth), A,
                B) <= tol(depth)


@pytest.mark.parametrize("name,depth,n", [("strassen", 2, 1000), ("strassen", 3, 515), ("laderman", 1, 384),
                                          ("strassen^2", 1, 512)])
def test_scaled_bit_exact_on_integers(fmm, oracle_mod, name, depth, n):
    algo = make_algo(fmm, name)
    plan = fmm.fmm_plan_create(n, algo, depth, post_additions="levels")
    A, B = inputs.operands(n, "integer", seed=n + 1)
    C0 = inputs.matrix(n, "integer", seed=n + 7)
    AB = oracle_mod.classic(A, B)
    for alpha, beta in [(2.0, -3.0), (-1.0, 1.0), (1.0, 1.0), (3.0, 0.0), (1.0, 2.0)]:
        assert np.array_equal(run(fmm, plan, A, B, alpha, beta, C0), oracle_mod.axpby(alpha, AB, beta, C0))


def test_beta_zero_does_not_read_c(fmm, oracle_mod):
    n = 515
    plan = fmm.fmm_plan_create(n, fmm.fmm_algo_builtin("strassen"), 2, post_additions="levels")
    A, B = inputs.operands(n, "integer", seed=9)
    C0 = np.full((n, n), np.nan)
    assert np.array_equal(run(fmm, plan, A, B, 1.0, 0.0, C0), oracle_mod.classic(A, B))


def test_rational_algorithm(fmm, oracle_mod):
    """Non-unit W numerators in the passes; the denominators' scale applied once in the last pass."""
    p, U, V, W, dens = rational_algos.strassen_dyadic()
    algo = fmm.RationalAlgo(p, U, V, W, dens, name="strassen_dyadic")
    for n, depth in [(300, 1), (517, 2), (1024, 3)]:
        plan = fmm.fmm_plan_create(n, algo, depth, post_additions="levels")
        assert plan.info()["post_passes"] >= 1
        A, B = inputs.operands(n, "integer", seed=n + depth)
        assert np.array_equal(run(fmm, plan, A, B), oracle_mod.classic(A, B))


def test_complex_inner_plan(fmm, oracle_mod):
    n = 300
    algo = fmm.fmm_algo_builtin("strassen")
    plan = fmm.fmm_plan_create(n, algo, 2, dtype="c128", post_additions="levels")
    A, B = inputs.operands(n, "integer", seed=4)
    A2, B2 = inputs.operands(n, "integer", seed=6)
    Az, Bz = A + 1j * A2, B + 1j * B2
    dA, dB = torch.from_numpy(Az).cuda(), torch.from_numpy(Bz).cuda()
    dC = torch.zeros_like(dA)
    fmm.fmm_gemm(plan, dA, dB, dC)
    assert fmm.fmm_sync_status(plan) == 0
    C = dC.cpu().numpy()
    re = oracle_mod.classic(A, B) - oracle_mod.classic(A2, B2)
    im = oracle_mod.classic(A, B2) + oracle_mod.classic(A2, B)
    assert np.array_equal(C.real, re) and np.array_equal(C.imag, im)


def test_levels_and_fused_agree_and_repeat_bitwise(fmm, oracle_mod):
    n = 1024
    algo = fmm.fmm_algo_builtin("strassen")
    lev = fmm.fmm_plan_create(n, algo, 3, post_additions="levels")
    fus = fmm.fmm_plan_create(n, algo, 3, post_additions="fused")
    assert lev.info()["post_passes"] == 2 and fus.info()["post_passes"] == 0
    assert lev.info()["flops_executed"] < fus.info()["flops_executed"]
    A, B = inputs.operands(n, "normal", seed=12)
    C1, C2 = run(fmm, lev, A, B), run(fmm, lev, A, B)
    assert np.array_equal(C1, C2)
    ref = oracle_mod.bilinear(A, B, algo.p, algo.U, algo.V, algo.W, 3)
    assert nerr(C1, ref, A, B) <= tol(3) and nerr(run(fmm, fus, A, B), ref, A, B) <= tol(3)


def test_composed_algorithm_matches_its_factor_depth(fmm):
    """<4,4,4;49> at depth 2 and Strassen at depth 4 sum the same four factors of W in the same
    passes: bit-identical results."""
    n = 1024
    a = fmm.fmm_plan_create(n, fmm.algorithm("strassen", 2), 2, post_additions="levels")
    b = fmm.fmm_plan_create(n, fmm.fmm_algo_builtin("strassen"), 4, post_additions="levels")
    A, B = inputs.operands(n, "uniform", seed=21)
    assert np.array_equal(run(fmm, a, A, B), run(fmm, b, A, B))


def test_unsupported_requests(fmm):
    algo = fmm.fmm_algo_builtin("strassen")
    for kw in ({"shard_count": 2, "shard_index": 0}, {"debug_poison_chain": 1}):
        with pytest.raises(fmm.FmmError) as e:
            fmm.fmm_plan_create(512, algo, 2, post_additions="levels", **kw)
        assert e.value.status == 3
    plan = fmm.fmm_plan_create(512, algo, 0, post_additions="levels")  # depth 0: nothing to sum
    assert plan.info()["post_passes"] == 0


def test_planner_choice_and_override(fmm, monkeypatch):
    """Stored when the fused adds reach 0.4 % of the leaf flops: Strassen depth 4 at n = 1024
    (ratio 0.13) is stored, depth 1 (ratio 0.002) fused; FMM_F64_POSTADD overrides the choice."""
    s = fmm.fmm_algo_builtin("strassen")
    monkeypatch.delenv("FMM_F64_POSTADD", raising=False)
    assert fmm.fmm_plan_create(1024, s, 4).info()["post_passes"] == 2
    assert fmm.fmm_plan_create(1024, s, 1).info()["post_passes"] == 0
    monkeypatch.setenv("FMM_F64_POSTADD", "fused")
    assert fmm.fmm_plan_create(1024, s, 4).info()["post_passes"] == 0
    monkeypatch.setenv("FMM_F64_POSTADD", "levels")
    assert fmm.fmm_plan_create(1024, s, 1).info()["post_passes"] == 1


def test_stored_plans_in_a_batched_launch(fmm, oracle_mod):
    """Stored and fused plans in one grouped launch: the stored ones write their products there, then
    run their passes and one grouped launch of their rank-q fix-ups (peeled sizes 1031 and 515)."""
    specs = [(1024, 4, "levels"), (515, 2, "levels"), (300, 1, "fused"), (1031, 3, "levels"), (777, 2, "fused"),
             (64, 0, "auto")]
    plans, As, Bs, Cs, C0s, host = [], [], [], [], [], []
    for i, (n, depth, post) in enumerate(specs):
        plans.append(fmm.fmm_plan_create(n, fmm.fmm_algo_builtin("strassen"), depth, post_additions=post))
        A, B = inputs.operands(n, "integer", seed=60 + i)
        C0 = inputs.matrix(n, "integer", seed=70 + i)
        host.append((A, B, C0))
        As.append(torch.from_numpy(A).cuda())
        Bs.append(torch.from_numpy(B).cuda())
        Cs.append(torch.full_like(As[-1], float("nan")))
        C0s.append(torch.from_numpy(C0).cuda())
    assert [p.info()["post_passes"] > 0 for p in plans] == [True, True, False, True, False, False]
    fmm.fmm_gemm_batched(plans, As, Bs, Cs)
    assert fmm.fmm_sync_status(plans[0]) == 0
    for (A, B, _), C in zip(host, Cs):
        assert np.array_equal(C.cpu().numpy(), oracle_mod.classic(A, B))
    alphas = [2.0, -1.0, 1.0, 3.0, 1.0, 2.0]
    betas = [-3.0, 1.0, 0.0, 2.0, 1.0, 0.0]
    fmm.fmm_gemm_batched(plans, As, Bs, C0s, alphas=alphas, betas=betas)
    assert fmm.fmm_sync_status(plans[0]) == 0
    for (A, B, C0), C, al, be in zip(host, C0s, alphas, betas):
        assert np.array_equal(C.cpu().numpy(), oracle_mod.axpby(al, oracle_mod.classic(A, B), be, C0))


@pytest.mark.parametrize("n,depth,passes", [(1030, 2, 1), (1027, 3, 2), (2048, 3, 2)])
def test_emulated_leaf_sums_by_the_same_passes(fmm, oracle_mod, monkeypatch, n, depth, passes):
    """The emulated leaf stores its products and, from depth 2, sums them by the level passes (the
    flattened order with FMM_OZAKI_POSTADD=flat): bit-exact on integers with and without alpha and beta,
    also at peeled sizes, whose rank-q fix-ups run after the passes."""
    algo = fmm.fmm_algo_builtin("strassen")
    monkeypatch.delenv("FMM_OZAKI_POSTADD", raising=False)
    level = fmm.fmm_plan_create(n, algo, depth, dtype="f64_ozaki")
    monkeypatch.setenv("FMM_OZAKI_POSTADD", "flat")
    flat = fmm.fmm_plan_create(n, algo, depth, dtype="f64_ozaki")
    monkeypatch.delenv("FMM_OZAKI_POSTADD")
    assert level.info()["post_passes"] == passes and flat.info()["post_passes"] == 0
    A, B = inputs.operands(n, "integer", seed=n + depth)
    C0 = inputs.matrix(n, "integer", seed=n + 3)
    AB = oracle_mod.classic(A, B)
    for alpha, beta in [(1.0, 0.0), (-2.0, 3.0), (0.5, 1.0)]:
        for plan in (level, flat):
            assert np.array_equal(run(fmm, plan, A, B, alpha, beta, C0), oracle_mod.axpby(alpha, AB, beta, C0))
    A, B = inputs.operands(n, "uniform", seed=n + 5)
    ref = oracle_mod.bilinear(A, B, algo.p, algo.U, algo.V, algo.W, depth)
    assert nerr(run(fmm, level, A, B), ref, A, B) <= tol(depth)
    assert nerr(run(fmm, flat, A, B), ref, A, B) <= tol(depth)
