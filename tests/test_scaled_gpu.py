"""GPU parity of the scaled product C = alpha A B + beta C (fmm_gemm_ex, fmm_gemm_batched_ex).

Section 3 states the product as C = alpha A B; beta C is the BLAS extension.  Bar: integer
inputs with small integer scalars come out bit-exact (every term and sum is exact in binary64);
real inputs stay within the depth's normalised tolerance of alpha * Dot2 + beta * C; beta = 0
never reads C and alpha = 0 never reads A or B (NaN placed there does not reach the result).
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


def run_ex(fmm, plan, alpha, A, B, beta, C0):
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.from_numpy(np.array(C0)).cuda()
    fmm.fmm_gemm_ex(plan, alpha, dA, dB, beta, dC)
    st = fmm.fmm_sync_status(plan)
    assert st == 0, fmm.fmm_status_string(st)
    return dC.cpu().numpy()


CASES = [("strassen", 0, 300), ("strassen", 1, 256), ("strassen", 2, 1000), ("winograd", 2, 515),
         ("laderman", 1, 384), ("strassen^2", 1, 512)]
SCALARS = [(2.0, -3.0), (-1.0, 1.0), (1.0, 1.0), (3.0, 0.0), (1.0, 2.0)]


def make_plan(fmm, name, n, depth, dtype="f64"):
    algo = fmm.algorithm(name[:-2], 2) if name.endswith("^2") else fmm.fmm_algo_builtin(name)
    return fmm.fmm_plan_create(n, algo, depth, dtype=dtype)


@pytest.mark.parametrize("name,depth,n", CASES)
def test_scaled_fp64_bit_exact_on_integers(fmm, oracle_mod, name, depth, n):
    plan = make_plan(fmm, name, n, depth)
    A, B = inputs.operands(n, "integer", seed=n + 1)
    C0 = inputs.matrix(n, "integer", seed=n + 7)
    AB = oracle_mod.classic(A, B)
    for alpha, beta in SCALARS:
        got = run_ex(fmm, plan, alpha, A, B, beta, C0)
        assert np.array_equal(got, oracle_mod.axpby(alpha, AB, beta, C0)), (alpha, beta)


@pytest.mark.parametrize("engine", ["pair", "tc1", "mma_sync"])
@pytest.mark.parametrize("name,depth,n", [("strassen", 1, 301), ("strassen", 2, 1000), ("strassen", 0, 200)])
def test_scaled_emulated_bit_exact_on_integers(fmm, oracle_mod, monkeypatch, engine, name, depth, n):
    """Every slice-GEMM engine: the tcgen05 ones apply alpha and beta in the post-addition gather,
    the mma.sync one in its fused epilogue; the peel tasks (n = 301) in the FP64 kernel."""
    if engine == "pair":
        monkeypatch.delenv("FMM_OZAKI_ENGINE", raising=False)
    else:
        monkeypatch.setenv("FMM_OZAKI_ENGINE", engine)
    plan = make_plan(fmm, name, n, depth, "f64_ozaki")
    A, B = inputs.operands(n, "integer", seed=2 * n + depth)
    C0 = inputs.matrix(n, "integer", seed=n + 11)
    AB = oracle_mod.classic(A, B)
    for alpha, beta in [(2.0, -3.0), (-1.0, 1.0), (1.0, 0.0)]:
        got = run_ex(fmm, plan, alpha, A, B, beta, C0)
        assert np.array_equal(got, oracle_mod.axpby(alpha, AB, beta, C0)), (alpha, beta)


@pytest.mark.parametrize("dtype", ["f64", "f64_ozaki"])
@pytest.mark.parametrize("name,depth,n", [("strassen", 2, 1024), ("strassen", 3, 1003), ("laderman", 1, 576)])
def test_scaled_real_inputs_within_tolerance(fmm, oracle_mod, dtype, name, depth, n):
    plan = make_plan(fmm, name, n, depth, dtype)
    A, B = inputs.operands(n, "uniform", seed=31)
    C0 = inputs.matrix(n, "normal", seed=33)
    alpha, beta = 0.7, -1.3
    got = run_ex(fmm, plan, alpha, A, B, beta, C0)
    rows, cols = inputs.sample_indices(n, 4096, seed=35)
    ref = oracle_mod.axpby(alpha, oracle_mod.sample_dot2(A, B, rows, cols), beta, C0[rows, cols])
    scale = abs(alpha) * n * np.abs(A).max() * np.abs(B).max() + abs(beta) * np.abs(C0).max()
    tol = 1e-13 if depth <= 2 else 1e-12
    assert np.max(np.abs(got[rows, cols] - ref)) / scale <= tol


@pytest.mark.parametrize("dtype", ["f64", "f64_ozaki"])
def test_zero_scalars_do_not_read_their_operands(fmm, oracle_mod, dtype):
    n = 257
    plan = make_plan(fmm, "strassen", n, 1, dtype)
    A, B = inputs.operands(n, "integer", seed=41)
    nanC = np.full((n, n), np.nan)
    # beta = 0: the NaN in C is overwritten, never read
    got = run_ex(fmm, plan, -2.0, A, B, 0.0, nanC)
    assert np.array_equal(got, oracle_mod.axpby(-2.0, oracle_mod.classic(A, B), 0.0, nanC))
    # alpha = 0: A and B (NaN) are not read; C = beta C, or zeros for beta = 0
    A_nan = A.copy()
    A_nan[5, 7] = np.nan
    C0 = inputs.matrix(n, "integer", seed=43)
    got = run_ex(fmm, plan, 0.0, A_nan, B, 3.0, C0)
    assert np.array_equal(got, 3.0 * C0)
    got = run_ex(fmm, plan, 0.0, A_nan, B, 0.0, nanC)
    assert np.array_equal(got, np.zeros((n, n)))
    got = run_ex(fmm, plan, 0.0, A_nan, B, 1.0, C0)
    assert np.array_equal(got, C0)


def test_scaled_is_deterministic(fmm):
    n = 1000
    plan = make_plan(fmm, "strassen", n, 2)
    A, B = inputs.operands(n, "normal", seed=51)
    C0 = inputs.matrix(n, "normal", seed=53)
    first = run_ex(fmm, plan, 0.3, A, B, 0.9, C0)
    for _ in range(3):
        assert np.array_equal(run_ex(fmm, plan, 0.3, A, B, 0.9, C0), first)


def test_rejects_non_finite_scalars(fmm):
    n = 64
    plan = make_plan(fmm, "strassen", n, 1)
    X = torch.zeros(n, n, dtype=torch.float64, device="cuda")
    for alpha, beta in [(float("nan"), 0.0), (1.0, float("inf"))]:
        with pytest.raises(fmm.FmmError):
            fmm.fmm_gemm_ex(plan, alpha, X, X, beta, X)


def test_batched_scaled_per_product(fmm, oracle_mod):
    """One grouped launch with a different (alpha, beta) per product, one of them alpha = 0
    (run as a scaling of its C, outside the launch), matches the oracle bit for bit."""
    sizes = [130, 257, 512, 300, 999]
    alphas = [2.0, -1.0, 0.0, 1.0, 3.0]
    betas = [-3.0, 0.0, 2.0, 1.0, 0.0]
    plans, As, Bs, Cs, expect = [], [], [], [], []
    for i, n in enumerate(sizes):
        plans.append(make_plan(fmm, "strassen", n, 1 if n >= 256 else 0))
        A, B = inputs.operands(n, "integer", seed=60 + 2 * i)
        C0 = inputs.matrix(n, "integer", seed=90 + i)
        if alphas[i] == 0.0:
            A = A.copy()
            A[0, 0] = np.nan
        As.append(torch.from_numpy(A).cuda())
        Bs.append(torch.from_numpy(B).cuda())
        Cs.append(torch.from_numpy(C0.copy()).cuda())
        AB = None if alphas[i] == 0.0 else oracle_mod.classic(A, B)
        expect.append(oracle_mod.axpby(alphas[i], AB, betas[i], C0))
    fmm.fmm_gemm_batched(plans, As, Bs, Cs, alphas=alphas, betas=betas)
    torch.cuda.synchronize()
    for p in plans:
        assert fmm.fmm_sync_status(p) == 0
    for C, e in zip(Cs, expect):
        assert np.array_equal(C.cpu().numpy(), e)


def test_gemm_convenience_scalars(fmm, oracle_mod):
    n = 384
    A, B = inputs.operands(n, "integer", seed=71)
    C0 = inputs.matrix(n, "integer", seed=73)
    out = torch.from_numpy(C0.copy()).cuda()
    fmm.gemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), algo="laderman", depth=1, out=out,
             alpha=-2.0, beta=1.0)
    assert np.array_equal(out.cpu().numpy(), oracle_mod.axpby(-2.0, oracle_mod.classic(A, B), 1.0, C0))
    with pytest.raises(ValueError):
        fmm.gemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), beta=1.0)
