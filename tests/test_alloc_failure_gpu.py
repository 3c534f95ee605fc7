"""Every allocation point of plan creation, the host-buffer path and the grouped launch fails once on
demand (fmm_debug_fail_allocation): each call must return FMM_ERR_OOM, leave nothing allocated, and the
next call without injection must work.  The failures are injected in the library's allocation shim on the
host, so no GPU allocation actually fails."""
import numpy as np
import pytest

from paper_2312_12732_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

OOM = 4


@pytest.fixture(scope="module")
def fmm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_12732_gb300 import _build

    _build.build()
    import paper_2312_12732_gb300 as m

    return m


def sweep(fmm, make):
    """Fail allocation k = 0, 1, ... of `make` until it succeeds; returns the number of allocation points."""
    base = fmm.fmm_debug_live_allocations()
    k = 0
    try:
        while True:
            fmm.fmm_debug_fail_allocation(k)
            try:
                out = make()
            except fmm.FmmError as e:
                assert e.status == OOM, (k, e)
                assert fmm.fmm_debug_live_allocations() == base, k
                k += 1
                assert k < 64
                continue
            fmm.fmm_debug_fail_allocation(-1)
            return k, out
    finally:
        fmm.fmm_debug_fail_allocation(-1)


@pytest.mark.parametrize("dtype,depth,n", [("f64", 2, 300), ("f64", 0, 100), ("f64_ozaki", 2, 300),
                                           ("c128", 1, 130), ("c128_3m", 1, 130), ("f32", 1, 130)])
def test_every_plan_allocation_failure_is_clean(fmm, oracle_mod, dtype, depth, n):
    s = fmm.fmm_algo_builtin("strassen")
    base = fmm.fmm_debug_live_allocations()
    points, plan = sweep(fmm, lambda: fmm.fmm_plan_create(n, s, depth, dtype=dtype))
    assert points >= 2
    if dtype in ("f64", "f64_ozaki"):
        A, B = inputs.operands(n, "integer", seed=n)
        dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        dC = torch.empty_like(dA)
        fmm.fmm_gemm(plan, dA, dB, dC)
        assert fmm.fmm_sync_status(plan) == 0
        assert np.array_equal(dC.cpu().numpy(), oracle_mod.classic(A, B))
    fmm.fmm_plan_destroy(plan)
    assert fmm.fmm_debug_live_allocations() == base


def test_host_path_allocation_failures_are_clean(fmm, oracle_mod):
    s = fmm.fmm_algo_builtin("strassen")
    n = 260
    plan = fmm.fmm_plan_create(n, s, 1)
    A, B = inputs.operands(n, "integer", seed=5)
    hA, hB = torch.from_numpy(A), torch.from_numpy(B)
    hC = torch.empty_like(hA)
    with_plan = fmm.fmm_debug_live_allocations()
    points, _ = sweep(fmm, lambda: fmm.fmm_gemm_host(plan, hA, hB, hC))
    assert points >= 1
    assert np.array_equal(hC.numpy(), oracle_mod.classic(A, B))
    assert fmm.fmm_debug_live_allocations() >= with_plan  # the plan keeps its host-path buffers
    fmm.fmm_plan_destroy(plan)


def test_batched_launch_allocation_failure_is_clean(fmm, oracle_mod):
    s = fmm.fmm_algo_builtin("strassen")
    sizes = [200, 300]
    plans = [fmm.fmm_plan_create(n, s, 1) for n in sizes]
    host = [inputs.operands(n, "integer", seed=60 + n) for n in sizes]
    As = [torch.from_numpy(A).cuda() for A, _ in host]
    Bs = [torch.from_numpy(B).cuda() for _, B in host]
    Cs = [torch.empty_like(A) for A in As]
    points, _ = sweep(fmm, lambda: fmm.fmm_gemm_batched(plans, As, Bs, Cs))
    assert points >= 1
    assert fmm.fmm_sync_status(plans[0]) == 0
    for (A, B), C in zip(host, Cs):
        assert np.array_equal(C.cpu().numpy(), oracle_mod.classic(A, B))
