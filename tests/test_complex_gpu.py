"""GPU parity of the double-complex products (FMM_C128: four real fast products per call;
FMM_C128_3M: three, Gauss's form) against the oracle's complex recursion.

Bar: integer-valued complex inputs are exact on both forms (every part product, sum and join is
an exact integer below 2^53), so they match the oracle bit for bit; real inputs stay within the
depth's normalised tolerance, n max|A| max|B| with complex moduli as the scale.
"""
import ctypes

import numpy as np
import pytest

from golden import rational_algos
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


def cmat(n, kind, seed):
    return inputs.matrix(n, kind, seed=seed) + 1j * inputs.matrix(n, kind, seed=seed + 1000)


def make_algo(fmm, name):
    return fmm.algorithm(name[:-2], 2) if name.endswith("^2") else fmm.fmm_algo_builtin(name)


def run(fmm, plan, A, B):
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.full_like(dA, complex(float("nan"), float("nan")))
    fmm.fmm_gemm(plan, dA, dB, dC)
    st = fmm.fmm_sync_status(plan)
    assert st == 0, fmm.fmm_status_string(st)
    return dC.cpu().numpy()


def nerr(C, ref, A, B):
    return float(np.max(np.abs(C - ref)) / (A.shape[0] * np.abs(A).max() * np.abs(B).max()))


CASES = [("strassen", 0, 130), ("strassen", 1, 256), ("strassen", 2, 1000), ("winograd", 2, 515),
         ("laderman", 1, 384), ("strassen^2", 1, 512)]


@pytest.mark.parametrize("dtype", ["c128", "c128_3m"])
@pytest.mark.parametrize("name,depth,n", CASES)
def test_complex_bit_exact_on_integers(fmm, oracle_mod, dtype, name, depth, n):
    plan = fmm.fmm_plan_create(n, make_algo(fmm, name), depth, dtype=dtype)
    A, B = cmat(n, "integer", n), cmat(n, "integer", n + 1)
    assert np.array_equal(run(fmm, plan, A, B), oracle_mod.classic_complex(A, B))


@pytest.mark.parametrize("dtype,tol", [("c128", 1e-13), ("c128_3m", 2e-13)])
@pytest.mark.parametrize("name,depth,n", [("strassen", 2, 1024), ("winograd", 1, 777), ("laderman", 1, 576)])
def test_complex_real_inputs_within_tolerance(fmm, oracle_mod, dtype, tol, name, depth, n):
    algo = make_algo(fmm, name)
    plan = fmm.fmm_plan_create(n, algo, depth, dtype=dtype)
    A, B = cmat(n, "uniform", 3), cmat(n, "normal", 5)
    C = run(fmm, plan, A, B)
    ref = oracle_mod.bilinear_complex(A, B, algo.p, algo.U, algo.V, algo.W, depth)
    assert nerr(C, ref, A, B) <= tol


def test_four_and_three_product_forms_differ_only_by_rounding(fmm):
    n = 512
    algo = fmm.fmm_algo_builtin("strassen")
    A, B = cmat(n, "uniform", 7), cmat(n, "uniform", 9)
    C4 = run(fmm, fmm.fmm_plan_create(n, algo, 2, dtype="c128"), A, B)
    C3 = run(fmm, fmm.fmm_plan_create(n, algo, 2, dtype="c128_3m"), A, B)
    assert 0 < nerr(C4, C3, A, B) <= 2e-13
    # the real parts come from the same two real products (ArBr, AiBi), subtracted in different places
    assert nerr(C4.real, C3.real, A, B) <= 1e-13


@pytest.mark.parametrize("dtype", ["c128", "c128_3m"])
def test_complex_scalars(fmm, oracle_mod, dtype):
    n = 300
    plan = fmm.fmm_plan_create(n, fmm.fmm_algo_builtin("strassen"), 1, dtype=dtype)
    A, B, C0 = cmat(n, "integer", 11), cmat(n, "integer", 12), cmat(n, "integer", 13)
    AB = oracle_mod.classic_complex(A, B)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    for alpha, beta in [(2.0, -3.0), (-1.0, 1.0), (1.0, 0.0), (0.0, 2.0), (0.0, 0.0)]:
        dC = torch.from_numpy(C0.copy()).cuda()
        fmm.fmm_gemm_ex(plan, alpha, dA, dB, beta, dC)
        assert fmm.fmm_sync_status(plan) == 0
        assert np.array_equal(dC.cpu().numpy(), alpha * AB + beta * C0), (alpha, beta)


def test_complex_rational_algorithm(fmm, oracle_mod):
    p, U, V, W, dens = rational_algos.strassen_dyadic()
    plan = fmm.fmm_plan_create(640, fmm.RationalAlgo(p, U, V, W, dens), 2, dtype="c128")
    A, B = cmat(640, "integer", 21), cmat(640, "integer", 22)
    assert np.array_equal(run(fmm, plan, A, B), oracle_mod.classic_complex(A, B))


def test_complex_host_buffers_info_and_convenience(fmm, oracle_mod):
    n = 256
    algo = fmm.fmm_algo_builtin("winograd")
    plan = fmm.fmm_plan_create(n, algo, 1, dtype="c128")
    real = fmm.fmm_plan_create(n, algo, 1)
    ic, ir = plan.info(), real.info()
    assert ic["flops_leaf"] == 4 * ir["flops_leaf"]
    assert fmm.fmm_plan_workspace_bytes(plan) >= fmm.fmm_plan_workspace_bytes(real) + 6 * n * n * 8
    A, B = cmat(n, "integer", 31), cmat(n, "integer", 32)
    hA, hB = torch.from_numpy(A).pin_memory(), torch.from_numpy(B).pin_memory()
    hC = torch.empty_like(hA).pin_memory()
    fmm.fmm_gemm_host(plan, hA, hB, hC)
    assert np.array_equal(hC.numpy(), oracle_mod.classic_complex(A, B))
    out = fmm.gemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), algo="strassen", depth=2)
    assert out.dtype == torch.complex128 and np.array_equal(out.cpu().numpy(), oracle_mod.classic_complex(A, B))
    out3 = fmm.gemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), algo="strassen", depth=2, dtype="c128_3m")
    assert np.array_equal(out3.cpu().numpy(), oracle_mod.classic_complex(A, B))


def test_complex_plans_are_rejected_where_unsupported(fmm):
    """Complex plans do not join grouped launches, report no per-phase times, and need 16-byte
    aligned operands (checked before anything is launched)."""
    n = 64
    plan = fmm.fmm_plan_create(n, fmm.fmm_algo_builtin("strassen"), 1, dtype="c128", record_kernel_time=True)
    X = torch.zeros(n, n, dtype=torch.complex128, device="cuda")
    with pytest.raises(fmm.FmmError):
        fmm.fmm_gemm_batched([plan], [X], [X], [X])
    fmm.fmm_gemm(plan, X, X, X.clone())
    torch.cuda.synchronize()
    with pytest.raises(fmm.FmmError):
        fmm.fmm_plan_last_phase_ms(plan)
    leaf, total = fmm.fmm_plan_last_kernel_ms(plan)
    assert total > 0
    lib = fmm.lib()
    st = lib.fmm_gemm_ex(plan.handle, 1.0, ctypes.c_void_p(X.data_ptr() + 8), ctypes.c_void_p(X.data_ptr()), 0.0,
                         ctypes.c_void_p(X.data_ptr()), None)
    assert st == 1
