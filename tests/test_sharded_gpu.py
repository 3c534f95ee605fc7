"""Product-sharded plans on one GPU: the shards of a multiplication run one after the other, each into its
own partial C, and their sum must equal the oracle's product (bit-exact on integer inputs, within the
depth's tolerance on real inputs).  Covers peeled sizes (only the shard that holds product 0 runs the peel
fix-ups), C blocks that a shard's products never reach (zero in its partial), and the rules of sharded
plans (beta = 0 only, no batched launch, FMM_F64 only, at most one shard per sub-problem)."""
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


def sharded_sum(fmm, n, algo, depth, shards, A, B, **opts):
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    total = torch.zeros_like(dA)
    covered = []
    for k in range(shards):
        plan = fmm.fmm_plan_create(n, algo, depth, shard_count=shards, shard_index=k, **opts)
        info = plan.info()
        covered.append((info["product_begin"], info["product_end"]))
        C = torch.full_like(dA, float("nan"))
        fmm.fmm_gemm(plan, dA, dB, C)
        assert fmm.fmm_sync_status(plan) == 0
        assert not torch.isnan(C).any()
        total += C
    return total.cpu().numpy(), covered


@pytest.mark.parametrize("name,power,depth,n,shards", [("strassen", 1, 2, 512, 3), ("strassen", 1, 2, 1001, 4),
                                                       ("strassen", 2, 1, 777, 5), ("winograd", 1, 3, 600, 8),
                                                       ("laderman", 1, 1, 301, 2), ("strassen", 1, 1, 256, 7)])
def test_shards_sum_to_the_exact_product(fmm, oracle_mod, name, power, depth, n, shards):
    algo = fmm.algorithm(name, power)
    A, B = inputs.operands(n, "integer", seed=n + shards)
    got, covered = sharded_sum(fmm, n, algo, depth, shards, A, B)
    assert np.array_equal(got, oracle_mod.classic(A, B))
    R = algo.R ** depth
    assert covered[0][0] == 0 and covered[-1][1] == R
    assert all(e0 == b1 for (_, e0), (b1, _) in zip(covered, covered[1:]))


@pytest.mark.parametrize("kind", ["uniform", "normal"])
def test_shards_of_real_inputs_within_tolerance(fmm, oracle_mod, kind):
    s = fmm.fmm_algo_builtin("strassen")
    n = 1030
    A, B = inputs.operands(n, kind, seed=9)
    got, _ = sharded_sum(fmm, n, s, 2, 6, A, B, tile_n=128)
    assert nerr(got, oracle_mod.bilinear(A, B, s.p, s.U, s.V, s.W, 2), A, B) <= 1e-13


def test_sharded_plan_rules(fmm):
    s = fmm.fmm_algo_builtin("strassen")
    A = torch.ones(256, 256, dtype=torch.float64, device="cuda")
    plan = fmm.fmm_plan_create(256, s, 1, shard_count=2, shard_index=1)
    with pytest.raises(fmm.FmmError) as e:  # beta != 0 would count C once per shard
        fmm.fmm_gemm_ex(plan, 1.0, A, A, 1.0, A.clone())
    assert e.value.status == 3
    with pytest.raises(fmm.FmmError):  # a sharded plan cannot join a grouped launch
        fmm.fmm_gemm_batched([plan], [A], [A], [A.clone()])
    with pytest.raises(fmm.FmmError) as e:  # more shards than the 7 sub-problems of one level
        fmm.fmm_plan_create(256, s, 1, shard_count=8, shard_index=0)
    assert e.value.status == 3
    with pytest.raises(fmm.FmmError) as e:  # the fused schedule has one sub-problem
        fmm.fmm_plan_create(256, s, 1, schedule="fused", shard_count=2, shard_index=0)
    assert e.value.status == 3
    with pytest.raises(fmm.FmmError) as e:
        fmm.fmm_plan_create(256, s, 1, dtype="f64_ozaki", shard_count=2, shard_index=0)
    assert e.value.status == 3
