"""GPU parity of plans for algorithms with rational coefficients (Section 2: the coefficients of
a, b, c need not be integers).

The library runs the integer numerator tables and applies (den_u den_v den_w)^-depth once per
leaf product with W; the oracle applies every fraction where it stands.  Bar: power-of-two
denominators make every step exact on integer inputs, so both sides agree bit for bit with the
classic product; denominators 3 and 9 are compared on real inputs by the depth's tolerance,
against Dot2 entries and against the oracle's own recursion.  The test tables come from
``tests/golden/rational_algos.py`` (exact change of basis of the paper's Strassen table).
"""
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


def run(fmm, plan, A, B):
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.full_like(dA, float("nan"))
    fmm.fmm_gemm(plan, dA, dB, dC)
    st = fmm.fmm_sync_status(plan)
    assert st == 0, fmm.fmm_status_string(st)
    return dC.cpu().numpy()


def ralgo(fmm, make):
    p, U, V, W, dens = make()
    return fmm.RationalAlgo(p, U, V, W, dens, name=make.__name__), (p, U, V, W, dens)


@pytest.mark.parametrize("dtype", ["f64", "f64_ozaki"])
@pytest.mark.parametrize("n,depth", [(64, 1), (300, 1), (1000, 2), (517, 2), (1024, 3)])
def test_dyadic_bit_exact_on_integers(fmm, oracle_mod, dtype, n, depth):
    algo, _ = ralgo(fmm, rational_algos.strassen_dyadic)
    plan = fmm.fmm_plan_create(n, algo, depth, dtype=dtype)
    assert plan.info()["coef_scale"] == 8.0 ** -depth
    A, B = inputs.operands(n, "integer", seed=n + depth)
    assert np.array_equal(run(fmm, plan, A, B), oracle_mod.classic(A, B))


@pytest.mark.parametrize("schedule,levels", [("fused", 0), ("hybrid", 1)])
def test_dyadic_other_schedules(fmm, oracle_mod, schedule, levels):
    """Pre-additions fused into the leaf's operand staging apply the non-unit numerators there."""
    algo, _ = ralgo(fmm, rational_algos.strassen_dyadic)
    n = 777
    plan = fmm.fmm_plan_create(n, algo, 2, schedule=schedule, materialize_levels=levels)
    A, B = inputs.operands(n, "integer", seed=5)
    assert np.array_equal(run(fmm, plan, A, B), oracle_mod.classic(A, B))


def test_halved_bit_exact_on_integers(fmm, oracle_mod):
    algo, _ = ralgo(fmm, rational_algos.strassen_halved)
    plan = fmm.fmm_plan_create(513, algo, 3)
    assert plan.info()["coef_scale"] == 0.125
    A, B = inputs.operands(513, "integer", seed=8)
    assert np.array_equal(run(fmm, plan, A, B), oracle_mod.classic(A, B))


@pytest.mark.parametrize("dtype", ["f64", "f64_ozaki"])
@pytest.mark.parametrize("make,n,depth", [(rational_algos.strassen_thirds, 1024, 1),
                                          (rational_algos.strassen_thirds, 1000, 2),
                                          (rational_algos.strassen_dyadic, 1024, 2)])
def test_real_inputs_within_tolerance(fmm, oracle_mod, dtype, make, n, depth):
    algo, (p, U, V, W, dens) = ralgo(fmm, make)
    plan = fmm.fmm_plan_create(n, algo, depth, dtype=dtype)
    A, B = inputs.operands(n, "uniform", seed=n + 3)
    C = run(fmm, plan, A, B)
    scale = n * np.abs(A).max() * np.abs(B).max()
    rows, cols = inputs.sample_indices(n, 4096, seed=9)
    ref = oracle_mod.sample_dot2(A, B, rows, cols)
    assert np.max(np.abs(C[rows, cols] - ref)) / scale <= 1e-13
    Co = oracle_mod.bilinear_rational(A, B, p, U, V, W, dens, depth)
    assert np.max(np.abs(C - Co)) / scale <= 1e-13


def test_rational_with_scalars_and_in_a_batch(fmm, oracle_mod):
    """alpha and beta compose with the coefficient scale; a rational plan shares a grouped
    launch with integer plans."""
    algo, _ = ralgo(fmm, rational_algos.strassen_dyadic)
    n = 640
    plan = fmm.fmm_plan_create(n, algo, 2)
    A, B = inputs.operands(n, "integer", seed=12)
    C0 = inputs.matrix(n, "integer", seed=13)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.from_numpy(C0.copy()).cuda()
    fmm.fmm_gemm_ex(plan, -2.0, dA, dB, 3.0, dC)
    assert fmm.fmm_sync_status(plan) == 0
    AB = oracle_mod.classic(A, B)
    assert np.array_equal(dC.cpu().numpy(), oracle_mod.axpby(-2.0, AB, 3.0, C0))

    plans = [fmm.fmm_plan_create(n, algo, 2), fmm.fmm_plan_create(n, fmm.fmm_algo_builtin("strassen"), 2),
             fmm.fmm_plan_create(300, algo, 1)]
    ops = [(A, B), inputs.operands(n, "integer", seed=14), inputs.operands(300, "integer", seed=15)]
    As = [torch.from_numpy(x).cuda() for x, _ in ops]
    Bs = [torch.from_numpy(y).cuda() for _, y in ops]
    Cs = [torch.full_like(x, float("nan")) for x in As]
    fmm.fmm_gemm_batched(plans, As, Bs, Cs)
    torch.cuda.synchronize()
    for pl, (x, y), C in zip(plans, ops, Cs):
        assert fmm.fmm_sync_status(pl) == 0
        assert np.array_equal(C.cpu().numpy(), oracle_mod.classic(x, y))
