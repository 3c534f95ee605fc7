"""fmm_host_alloc / fmm_host_free: page-locked host memory for the host-buffer path.  Buffers of at least
one transparent huge page come from a huge-page-aligned mapping registered with the driver, smaller ones
from cudaHostAlloc; both must be page-locked (so copies from them are asynchronous), hold what is written
to them, serve fmm_gemm_host with results equal to the oracle's, fail cleanly under an injected
allocation failure and refuse addresses they did not hand out."""
import gc

import numpy as np
import pytest

from paper_2312_12732_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

OOM, INVALID = 4, 1


@pytest.fixture(scope="module")
def fmm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_12732_gb300 import _build

    _build.build()
    import paper_2312_12732_gb300 as m

    return m


def test_small_and_huge_page_buffers_are_page_locked_and_round_trip(fmm):
    base = fmm.fmm_debug_live_allocations()
    hp = fmm.fmm_host_huge_page_bytes()
    sizes = [512] + ([hp // 8] if hp else [])
    for count in sizes:
        h = fmm.host_empty((count,), torch.float64)
        assert h.is_pinned()
        if count * 8 >= hp > 0:
            assert h.data_ptr() % hp == 0  # the huge-page path: one aligned mapping
        src = torch.arange(count, dtype=torch.float64, device="cuda") * 0.5 - 3.0
        h.copy_(src, non_blocking=True)
        torch.cuda.synchronize()
        assert torch.equal(h, src.cpu())
        back = torch.empty_like(src)
        back.copy_(h, non_blocking=True)
        torch.cuda.synchronize()
        assert torch.equal(back, src)
        del h
        gc.collect()
        assert fmm.fmm_debug_live_allocations() == base


def test_gemm_host_from_library_buffers_matches_oracle(fmm, oracle_mod):
    s = fmm.fmm_algo_builtin("strassen")
    for n, depth in ((260, 1), (517, 2)):
        plan = fmm.fmm_plan_create(n, s, depth)
        A, B = inputs.operands(n, "integer", seed=n)
        hA, hB, hC = (fmm.host_empty((n, n)) for _ in range(3))
        hA.copy_(torch.from_numpy(A))
        hB.copy_(torch.from_numpy(B))
        fmm.fmm_gemm_host(plan, hA, hB, hC)
        assert fmm.fmm_sync_status(plan) == 0
        assert np.array_equal(hC.numpy(), oracle_mod.classic(A, B))
        fmm.fmm_plan_destroy(plan)


def test_injected_failure_and_bad_addresses(fmm):
    base = fmm.fmm_debug_live_allocations()
    fmm.fmm_debug_fail_allocation(0)
    try:
        with pytest.raises(fmm.FmmError) as e:
            fmm.fmm_host_alloc(1 << 16)
        assert e.value.status == OOM
    finally:
        fmm.fmm_debug_fail_allocation(-1)
    assert fmm.fmm_debug_live_allocations() == base
    addr = fmm.fmm_host_alloc(1 << 16)
    assert fmm.fmm_debug_live_allocations() == base + 1
    fmm.fmm_host_free(addr)
    with pytest.raises(fmm.FmmError) as e:  # freed already
        fmm.fmm_host_free(addr)
    assert e.value.status == INVALID
    with pytest.raises(fmm.FmmError) as e:  # never handed out
        fmm.fmm_host_free(addr + 64)
    assert e.value.status == INVALID
    fmm.fmm_host_free(0)
    assert fmm.fmm_debug_live_allocations() == base
