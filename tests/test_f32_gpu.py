"""GPU parity of single-precision plans (FMM_F32: binary32 operands widened to binary64, the product
through the emulated leaf with 6 slices, one rounding to binary32; Section 1 lists single precision
among the deployable types).

Bar: integer-valued inputs whose products stay below 2^24 come out exactly (the product is exact
before its rounding, and the rounding is exact). Real inputs with the default 6 slices (30 bits,
rounding the pre-added S_r and T_r to 2^-31 of their row maxima) stay within one binary32 unit
roundoff normwise, max |C - ref| <= 2^-24 n max|A| max|B|, the accuracy class of binary32 GEMM. With
8 slices the product before its rounding is accurate enough that every entry is within binary32
rounding of the oracle's FP64 product: |C - ref| <= 2^-24 |ref| + 1e-9 n max|A| max|B|.
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


def run(fmm, plan, A, B, alpha=1.0, beta=0.0, C0=None):
    dA = torch.from_numpy(A.astype(np.float32)).cuda()
    dB = torch.from_numpy(B.astype(np.float32)).cuda()
    dC = (torch.full_like(dA, float("nan")) if C0 is None else torch.from_numpy(C0.astype(np.float32)).cuda())
    fmm.fmm_gemm_ex(plan, alpha, dA, dB, beta, dC)
    st = fmm.fmm_sync_status(plan)
    assert st == 0, fmm.fmm_status_string(st)
    return dC.cpu().numpy()


@pytest.mark.parametrize("name,depth,n", [("strassen", 0, 200), ("strassen", 1, 300), ("strassen", 2, 1000),
                                          ("winograd", 2, 515), ("laderman", 1, 384)])
def test_f32_exact_on_integers(fmm, oracle_mod, name, depth, n):
    plan = fmm.fmm_plan_create(n, fmm.fmm_algo_builtin(name), depth, dtype="f32")
    A, B = inputs.operands(n, "integer", seed=n + depth)
    ref = oracle_mod.classic(A, B)
    assert np.abs(ref).max() < 2 ** 24
    assert np.array_equal(run(fmm, plan, A, B), ref.astype(np.float32))


@pytest.mark.parametrize("slices", [0, 8])
@pytest.mark.parametrize("kind,n,depth", [("uniform", 1024, 2), ("normal", 1000, 2), ("uniform", 777, 3)])
def test_f32_real_inputs(fmm, oracle_mod, kind, n, depth, slices):
    plan = fmm.fmm_plan_create(n, fmm.fmm_algo_builtin("strassen"), depth, dtype="f32", ozaki_slices=slices)
    A, B = inputs.operands(n, kind, seed=n)
    A32, B32 = A.astype(np.float32), B.astype(np.float32)
    ref = oracle_mod.classic(A32.astype(np.float64), B32.astype(np.float64))
    C = run(fmm, plan, A32, B32).astype(np.float64)
    scale = n * np.abs(A32).max() * np.abs(B32).max()
    if slices == 0:
        assert np.max(np.abs(C - ref)) <= 2.0 ** -24 * scale
    else:
        assert np.all(np.abs(C - ref) <= 2.0 ** -24 * np.abs(ref) + 1e-9 * scale)


def test_f32_scalars_and_slices(fmm, oracle_mod):
    n = 300
    A, B = inputs.operands(n, "integer", seed=4)
    C0 = inputs.matrix(n, "integer", seed=5)
    ref = oracle_mod.axpby(2.0, oracle_mod.classic(A, B), -3.0, C0)
    for slices in (0, 8):
        plan = fmm.fmm_plan_create(n, fmm.fmm_algo_builtin("strassen"), 1, dtype="f32", ozaki_slices=slices)
        assert plan.info()["ozaki_slices"] == (slices or 6)
        assert np.array_equal(run(fmm, plan, A, B, 2.0, -3.0, C0), ref.astype(np.float32))
        assert np.array_equal(run(fmm, plan, A, B, 0.0, 0.5, C0), (0.5 * C0).astype(np.float32))


def test_f32_convenience_and_host_buffers(fmm, oracle_mod):
    n = 256
    A, B = inputs.operands(n, "integer", seed=6)
    ref = oracle_mod.classic(A, B).astype(np.float32)
    out = fmm.gemm(torch.from_numpy(A.astype(np.float32)).cuda(), torch.from_numpy(B.astype(np.float32)).cuda(),
                   algo="strassen", depth=2)
    assert out.dtype == torch.float32 and np.array_equal(out.cpu().numpy(), ref)
    plan = fmm.fmm_plan_create(n, fmm.fmm_algo_builtin("winograd"), 1, dtype="f32")
    hA = torch.from_numpy(A.astype(np.float32)).pin_memory()
    hB = torch.from_numpy(B.astype(np.float32)).pin_memory()
    hC = torch.empty_like(hA).pin_memory()
    fmm.fmm_gemm_host(plan, hA, hB, hC)
    assert np.array_equal(hC.numpy(), ref)
    X = torch.zeros(n, n, dtype=torch.float64, device="cuda")
    assert fmm.lib().fmm_gemm(plan.handle, X.data_ptr(), X.data_ptr(), X.data_ptr(), None) == 1
