"""GPU parity of square algorithms composed from rectangular ones (Section 2: a problem of split
factor 6 or 12 solved through non-square basic products, 2x2x3 with 2x3x2 and 3x2x2, composed by
Kronecker products).

The library's rectangular tables (<2,2,3;11> and its rotations, classic <3,3,2;18>) are composed
into square <12,12,12;1331> and <6,6,6;198> and planned like any square algorithm. Bar: integer
inputs bit-exact against the classic product; real inputs within the depth's tolerance of the
oracle's nested evaluation, one rectangular factor per level (the same algorithm, summed in a
different order). The oracle's tables come from tests/golden/rect_algos.py.
"""
import numpy as np
import pytest

from golden import rect_algos
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


def square_12(fmm):
    s = fmm.fmm_algo_rect_builtin("strassen_2x2x3")
    c = fmm.fmm_algo_rect_cyclic(s)
    return fmm.fmm_algo_rect_as_square(fmm.fmm_algo_rect_compose(fmm.fmm_algo_rect_compose(s, c),
                                                                 fmm.fmm_algo_rect_cyclic(c)))


def square_6(fmm):
    s = fmm.fmm_algo_rect_builtin("strassen_2x2x3")
    return fmm.fmm_algo_rect_as_square(fmm.fmm_algo_rect_compose(s, fmm.fmm_algo_rect_classic(3, 3, 2)))


@pytest.mark.parametrize("dtype,which,n,depth", [
    ("f64", "12", 1152, 1), ("f64", "12", 1000, 1), ("f64", "6", 600, 1), ("f64", "6", 727, 2),
    # the emulated leaf pads leaves to 128, so it runs the depth-1 cases only
    ("f64_ozaki", "12", 1152, 1), ("f64_ozaki", "6", 600, 1)])
def test_composed_rectangular_bit_exact_on_integers(fmm, oracle_mod, dtype, which, n, depth):
    algo = square_12(fmm) if which == "12" else square_6(fmm)
    plan = fmm.fmm_plan_create(n, algo, depth, dtype=dtype)
    A, B = inputs.operands(n, "integer", seed=n + depth)
    assert np.array_equal(run(fmm, plan, A, B), oracle_mod.classic(A, B))


def test_composed_rectangular_matches_nested_oracle_levels(fmm, oracle_mod):
    n = 1152
    plan = fmm.fmm_plan_create(n, square_12(fmm), 1)
    A, B = inputs.operands(n, "uniform", seed=17)
    C = run(fmm, plan, A, B)
    s = rect_algos.strassen_223()
    c = rect_algos.cyclic(s)
    ref = oracle_mod.rect_bilinear(A, B, [s, c, rect_algos.cyclic(c)])
    assert np.max(np.abs(C - ref)) / (n * np.abs(A).max() * np.abs(B).max()) <= 1e-13
    rows, cols = inputs.sample_indices(n, 2048, seed=3)
    exact = oracle_mod.sample_dot2(A, B, rows, cols)
    assert np.max(np.abs(C[rows, cols] - exact)) / (n * np.abs(A).max() * np.abs(B).max()) <= 1e-13
