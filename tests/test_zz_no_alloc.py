"""The allocation-free entry point, fmm_gemm_noalloc.

It exists for callers that cannot allocate device memory (allocator or
memory-pool callbacks, frameworks that reserve all device memory up front,
real-time paths that forbid cudaMalloc): it keeps all scratch state in a
static device array.  These tests call it through the C ABI and check each
result against the plan-based fmm_gemm on the same inputs and against the
oracle, for calls in a row with different shapes and algorithms, so that state
left in the shared array by one call cannot leak into the next.  They also
read its device status (fmm_noalloc_sync_status), make a bounded wait run out
on purpose (a counter poisoned from the host, no GPU fault) and check that a
call made during stream capture is refused.  The file is named to be
collected last.
"""
import numpy as np
import pytest

from paper_2312_12732_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TIMEOUT = 6  # FMM_ERR_TIMEOUT
UNSUPPORTED = 3  # FMM_ERR_UNSUPPORTED


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
    assert fmm.fmm_noalloc_sync_status() == 0
    got = c_noalloc.cpu().numpy()
    plan = fmm.fmm_plan_create(A.shape[0], algo, depth, schedule="fused")
    c_plan = torch.full_like(dA, float("nan"))
    fmm.fmm_gemm(plan, dA, dB, c_plan)
    assert fmm.fmm_sync_status(plan) == 0
    return got, c_plan.cpu().numpy()


def test_noalloc_matches_plan_entry_point_and_oracle_calls_in_a_row(fmm, oracle_mod):
    # first call: real inputs, Strassen depth 2 at a size with a remainder (1001 = 4 * 250 + 1), so the
    # peel tasks run
    s = fmm.fmm_algo_builtin("strassen")
    A, B = inputs.operands(1001, "uniform", seed=31)
    got, ref = both(fmm, s, 2, A, B)
    assert not np.isnan(got).any()
    assert nerr(got, ref, A, B) <= 1e-13
    assert nerr(got, oracle_mod.bilinear(A, B, s.p, s.U, s.V, s.W, 2), A, B) <= 1e-13
    # second call right after it: other algorithm, other size, integer inputs, depth 3
    w = fmm.fmm_algo_builtin("winograd")
    A, B = inputs.operands(777, "integer", seed=32)
    got, ref = both(fmm, w, 3, A, B)
    assert np.array_equal(got, ref)
    assert np.array_equal(got, oracle_mod.classic(A, B))
    # third: Laderman (p = 3, so the flattening of a 3 x 3 grid), real inputs with a remainder
    lad = fmm.fmm_algo_builtin("laderman")
    A, B = inputs.operands(500, "normal", seed=33)
    got, ref = both(fmm, lad, 1, A, B)
    assert nerr(got, ref, A, B) <= 1e-13
    assert nerr(got, oracle_mod.bilinear(A, B, lad.p, lad.U, lad.V, lad.W, 1), A, B) <= 1e-13
    # fourth: depth 0, the classic product
    A, B = inputs.operands(300, "integer", seed=34)
    got, ref = both(fmm, s, 0, A, B)
    assert np.array_equal(got, ref) and np.array_equal(got, oracle_mod.classic(A, B))


def test_noalloc_rejects_requests_beyond_its_scratch(fmm):
    lad = fmm.fmm_algo_builtin("laderman")
    A, B = inputs.operands(81, "uniform", seed=1)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.empty_like(dA)
    with pytest.raises(fmm.FmmError) as e:
        fmm.fmm_gemm_noalloc(lad, 4, dA, dB, dC)
    assert e.value.status == 8
    assert "static scratch" in str(e.value)


def test_noalloc_rejects_coefficients_that_would_overflow(fmm):
    # Strassen with U's column 0 scaled by 2^16: at depth 2 a flattened coefficient reaches 2^32, beyond
    # int32.  The table also fails the Brent equations, but the range check runs first.
    s = fmm.fmm_algo_builtin("strassen")
    U = s.U.copy()
    U[:, 0] *= 1 << 16
    big = fmm.Algo(2, U, s.V, s.W, name="scaled")
    A = torch.zeros(64, 64, dtype=torch.float64, device="cuda")
    with pytest.raises(fmm.FmmError) as e:
        fmm.fmm_gemm_noalloc(big, 2, A, A.clone(), A.clone())
    assert e.value.status == UNSUPPORTED


def test_noalloc_timeout_is_reported_and_context_survives(fmm, oracle_mod):
    """One ordering counter is poisoned from the host after the call's reset: its waiters give up after a
    50 ms bounded wait, fmm_noalloc_sync_status reports FMM_ERR_TIMEOUT once, and the next call works."""
    s = fmm.fmm_algo_builtin("strassen")
    A, B = inputs.operands(256, "integer", seed=35)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.empty_like(dA)
    try:
        fmm.fmm_noalloc_set_debug(0.05, True)
        fmm.fmm_gemm_noalloc(s, 1, dA, dB, dC)
        assert fmm.fmm_noalloc_sync_status() == TIMEOUT
        assert fmm.fmm_noalloc_sync_status() == 0  # read once, then cleared
    finally:
        fmm.fmm_noalloc_set_debug(5.0, False)
    fmm.fmm_gemm_noalloc(s, 1, dA, dB, dC)
    assert fmm.fmm_noalloc_sync_status() == 0
    assert np.array_equal(dC.cpu().numpy(), oracle_mod.classic(A, B))


def test_noalloc_refuses_a_capturing_stream(fmm):
    s = fmm.fmm_algo_builtin("strassen")
    A = torch.ones(128, 128, dtype=torch.float64, device="cuda")
    B, C = A.clone(), torch.empty_like(A)
    fmm.fmm_gemm_noalloc(s, 1, A, B, C)  # the device's set-up happens outside any capture
    assert fmm.fmm_noalloc_sync_status() == 0
    stream = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    status = None
    with torch.cuda.graph(g, stream=stream, capture_error_mode="thread_local"):
        try:
            fmm.fmm_gemm_noalloc(s, 1, A, B, C, stream)
        except fmm.FmmError as e:
            status = e.status
    assert status == UNSUPPORTED
    fmm.fmm_gemm_noalloc(s, 1, A, B, C)
    assert fmm.fmm_noalloc_sync_status() == 0
    assert bool(torch.all(C == 128.0))
