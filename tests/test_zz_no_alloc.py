"""The allocation-free entry point, fmm_gemm_noalloc.

It exists for callers that cannot allocate device memory (allocator or
memory-pool callbacks, frameworks that reserve all device memory up front,
real-time paths that forbid cudaMalloc): it keeps all scratch state in a
static device array.  These tests call it through the C ABI and compare it
with the plan-based fmm_gemm on the same inputs, for two calls in a row with
different shapes, so that state left in the shared array by the first call
cannot leak into the second.  The file is named to be collected last.
"""
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


def both(fmm, algo, depth, A, B):
    """(fmm_gemm_noalloc result, fmm_gemm result with the fused schedule)."""
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    c_noalloc = torch.full_like(dA, float("nan"))
    fmm.fmm_gemm_noalloc(algo, depth, dA, dB, c_noalloc)
    torch.cuda.synchronize()
    got = c_noalloc.cpu().numpy()
    plan = fmm.fmm_plan_create(A.shape[0], algo, depth, schedule="fused")
    c_plan = torch.full_like(dA, float("nan"))
    fmm.fmm_gemm(plan, dA, dB, c_plan)
    assert fmm.fmm_sync_status(plan) == 0
    return got, c_plan.cpu().numpy()


def test_noalloc_matches_plan_entry_point_two_calls_in_a_row(fmm):
    # first call: peeled size, real inputs, depth 2
    s = fmm.fmm_algo_builtin("strassen")
    A, B = inputs.operands(1000, "uniform", seed=31)
    got, ref = both(fmm, s, 2, A, B)
    assert not np.isnan(got).any()
    assert nerr(got, ref, A, B) <= 1e-13
    # second call right after it: other algorithm, other size, integer inputs
    w = fmm.fmm_algo_builtin("winograd")
    A, B = inputs.operands(777, "integer", seed=32)
    got, ref = both(fmm, w, 3, A, B)
    assert np.array_equal(got, ref)
    assert np.array_equal(got, A @ B)


def test_noalloc_rejects_requests_beyond_its_scratch(fmm):
    lad = fmm.fmm_algo_builtin("laderman")
    A, B = inputs.operands(81, "uniform", seed=1)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.empty_like(dA)
    with pytest.raises(fmm.FmmError) as e:
        fmm.fmm_gemm_noalloc(lad, 4, dA, dB, dC)
    assert e.value.status == 8
    assert "static scratch" in str(e.value)
