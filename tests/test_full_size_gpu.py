"""Full-size GPU parity on sampled outputs, in the launch configurations the
benchmark times: 4096 entries per case against Dot2 (compensated) reference
entries computed by the oracle one by one; integer-valued inputs must match
those entries exactly."""
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


def make_algo(fmm, name):
    return fmm.algorithm(name[:-2], 2) if name.endswith("^2") else fmm.fmm_algo_builtin(name)


def sampled(fmm, oracle_mod, n, name, depth, kind, dtype="f64", seed=5, count=4096):
    algo = make_algo(fmm, name)
    plan = fmm.fmm_plan_create(n, algo, depth, dtype=dtype)
    A, B = inputs.operands(n, kind, seed=seed)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.full_like(dA, float("nan"))
    fmm.fmm_gemm(plan, dA, dB, dC)
    assert fmm.fmm_sync_status(plan) == 0
    rows, cols = inputs.sample_indices(n, count, seed=seed + 100)
    r_t, c_t = torch.from_numpy(rows).cuda(), torch.from_numpy(cols).cuda()
    got = dC[r_t, c_t].cpu().numpy()
    ref = oracle_mod.sample_dot2(A, B, rows, cols)
    del dA, dB, dC
    torch.cuda.empty_cache()
    return got, ref, float(np.abs(A).max() * np.abs(B).max())


def tol(depth):
    return 1e-13 if depth <= 2 else 1e-12


@pytest.mark.parametrize("n,name,depth,dtype", [
    (8192, "strassen^2", 2, "f64"),        # the default benchmark workload
    (8192, "strassen", 2, "f64_ozaki"),    # the emulated-leaf workload of the benchmark
    (16384, "strassen", 2, "f64_ozaki"),
    (16384, "strassen", 3, "f64"),
    (4096, "winograd", 3, "f64"),
    (6912, "laderman", 1, "f64"),
])
def test_benchmarked_configurations(fmm, oracle_mod, n, name, depth, dtype):
    got, ref, scale = sampled(fmm, oracle_mod, n, name, depth, "uniform", dtype)
    assert np.max(np.abs(got - ref)) / (n * scale) <= tol(depth)


@pytest.mark.parametrize("n,depth", [(7777, 3), (10007, 3), (10007, 1)])
def test_peeled_full_sizes(fmm, oracle_mod, n, depth):
    got, ref, _ = sampled(fmm, oracle_mod, n, "strassen", depth, "integer")
    assert np.array_equal(got, ref)
    got, ref, scale = sampled(fmm, oracle_mod, n, "strassen", depth, "normal", seed=9)
    assert np.max(np.abs(got - ref)) / (n * scale) <= tol(depth)


@pytest.mark.parametrize("phi", [4, 8])
def test_wide_range_emulated_leaf_at_full_size(fmm, oracle_mod, phi):
    """Entries uniform[-1,1] * 10^U(-phi, phi) at n = 8192, Strassen depth 2: the emulated leaf stays
    within the depth's tolerance and within 2x the FP64 path's error on the same sampled entries."""
    n = 8192
    algo = fmm.fmm_algo_builtin("strassen")
    A, B = inputs.operands(n, "wide", seed=13, phi=phi)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    rows, cols = inputs.sample_indices(n, 4096, seed=21)
    r_t, c_t = torch.from_numpy(rows).cuda(), torch.from_numpy(cols).cuda()
    ref = oracle_mod.sample_dot2(A, B, rows, cols)
    scale = n * float(np.abs(A).max() * np.abs(B).max())
    errs = {}
    for dtype in ("f64_ozaki", "f64"):
        plan = fmm.fmm_plan_create(n, algo, 2, dtype=dtype)
        dC = torch.full_like(dA, float("nan"))
        fmm.fmm_gemm(plan, dA, dB, dC)
        assert fmm.fmm_sync_status(plan) == 0
        errs[dtype] = float(np.max(np.abs(dC[r_t, c_t].cpu().numpy() - ref))) / scale
        del dC, plan
        torch.cuda.empty_cache()
    assert errs["f64_ozaki"] <= 1e-13
    assert errs["f64_ozaki"] <= 2.0 * errs["f64"], errs


def test_default_workload_normal_entries(fmm, oracle_mod):
    """The default benchmark workload (<4,4,4;49> depth 2, n = 8192) on N(0,1) entries."""
    got, ref, scale = sampled(fmm, oracle_mod, 8192, "strassen^2", 2, "normal", seed=17)
    assert np.max(np.abs(got - ref)) / (8192 * scale) <= 1e-13
