"""GPU parity of the emulated-FP64 leaf (FMM_F64_OZAKI) against the oracle.

Bar: integer-valued inputs (entries in [-16, 16]) come out bit-exact -- their
slices are exact, each diagonal group is an exact integer in FP32, the int64
recombination keeps every bit and the FP64 post-additions stay below 2^53.
Real inputs: the normalised error against Dot2 reference entries stays within
the FP64 tolerance of its depth and within 2x the error of the plain FP64
path (FMM_F64) on the same inputs, with the default 12 slices.
"""
import numpy as np
import pytest

from paper_2312_12732_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
U = 2.0 ** -53


@pytest.fixture(scope="module")
def fmm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_12732_gb300 import _build

    _build.build()
    import paper_2312_12732_gb300 as m

    return m


def run(fmm, plan, A, B):
    dA = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(B).cuda()
    dC = torch.full_like(dA, float("nan"))
    fmm.fmm_gemm(plan, dA, dB, dC)
    st = fmm.fmm_sync_status(plan)
    assert st == 0, fmm.fmm_status_string(st)
    return dC.cpu().numpy()


def nerr(C, ref, A, B):
    n = A.shape[0]
    return float(np.max(np.abs(C - ref)) / (n * np.abs(A).max() * np.abs(B).max()))


def ref_entries(oracle_mod, A, B, count=4096, seed=3):
    n = A.shape[0]
    if n * n <= count:
        rows, cols = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
        rows, cols = rows.ravel(), cols.ravel()
    else:
        rows, cols = inputs.sample_indices(n, count, seed=seed)
    return rows, cols, oracle_mod.sample_dot2(A, B, rows, cols)


@pytest.mark.parametrize("name,depth,n", [("strassen", 0, 128), ("strassen", 0, 300), ("strassen", 1, 512),
                                          ("strassen", 2, 1000), ("winograd", 2, 1024), ("laderman", 1, 384),
                                          ("strassen", 1, 7)])
def test_ozaki_bit_exact_on_integers(fmm, oracle_mod, name, depth, n):
    algo = fmm.fmm_algo_builtin(name)
    plan = fmm.fmm_plan_create(n, algo, depth, dtype="f64_ozaki")
    A, B = inputs.operands(n, "integer", seed=n + depth)
    assert np.array_equal(run(fmm, plan, A, B), oracle_mod.classic(A, B))


@pytest.mark.parametrize("name,depth,n,kind,phi", [
    ("strassen", 0, 256, "uniform", 0), ("strassen", 1, 512, "uniform", 0), ("strassen", 2, 1024, "uniform", 0),
    ("strassen", 2, 1000, "normal", 0), ("strassen", 2, 1024, "wide", 4), ("strassen", 2, 1024, "wide", 8),
    ("strassen", 0, 512, "wide", 8), ("strassen", 1, 768, "wide", 4),
    ("winograd", 1, 640, "uniform", 0), ("laderman", 1, 576, "uniform", 0)])
def test_ozaki_accuracy_vs_fp64_path(fmm, oracle_mod, name, depth, n, kind, phi):
    algo = fmm.fmm_algo_builtin(name)
    A, B = inputs.operands(n, kind, seed=7, phi=phi)
    rows, cols, ref = ref_entries(oracle_mod, A, B)
    C_oz = run(fmm, fmm.fmm_plan_create(n, algo, depth, dtype="f64_ozaki"), A, B)
    C_64 = run(fmm, fmm.fmm_plan_create(n, algo, depth), A, B)
    e_oz = nerr(C_oz[rows, cols], ref, A, B)
    e_64 = nerr(C_64[rows, cols], ref, A, B)
    assert e_oz <= (1e-13 if depth <= 2 else 1e-12)
    assert e_oz <= 2.0 * e_64, (e_oz, e_64)


def test_fewer_slices_lose_accuracy(fmm, oracle_mod):
    """The slice count is the precision knob: each slice adds 5 bits, so 4 slices
    (20 bits) are far worse than the default 12 and still bounded by about 2^-18."""
    n = 256
    algo = fmm.fmm_algo_builtin("strassen")
    A, B = inputs.operands(n, "uniform", seed=9)
    rows, cols, ref = ref_entries(oracle_mod, A, B)
    e4 = nerr(run(fmm, fmm.fmm_plan_create(n, algo, 1, dtype="f64_ozaki", ozaki_slices=4), A, B)[rows, cols],
              ref, A, B)
    e12 = nerr(run(fmm, fmm.fmm_plan_create(n, algo, 1, dtype="f64_ozaki"), A, B)[rows, cols], ref, A, B)
    e8 = nerr(run(fmm, fmm.fmm_plan_create(n, algo, 1, dtype="f64_ozaki", ozaki_slices=8), A, B)[rows, cols],
              ref, A, B)
    assert e4 > 100 * e8 > 100 * 100 * e12
    assert e4 < 2.0 ** -18


def test_ozaki_plan_info(fmm):
    plan = fmm.fmm_plan_create(1000, fmm.fmm_algo_builtin("strassen"), 2, dtype="f64_ozaki", ozaki_slices=9)
    info = plan.info()
    assert info["ozaki_slices"] == 9 and info["materialized_levels"] == 2
    assert info["flops_lowp"] == 2.0 * 49 * 45 * 256 ** 3
    with pytest.raises(fmm.FmmError):
        fmm.fmm_plan_create(64, fmm.fmm_algo_builtin("strassen"), 1, dtype="f64_ozaki", ozaki_slices=13)


@pytest.mark.parametrize("engine", ["pair", "tc1", "mma_sync"])
@pytest.mark.parametrize("name,depth,n", [("strassen", 1, 7), ("strassen", 0, 300), ("strassen", 2, 1000),
                                          ("laderman", 1, 384)])
def test_every_slice_gemm_engine(fmm, oracle_mod, monkeypatch, engine, name, depth, n):
    """The CTA-pair kernel (default), the one-CTA tcgen05 kernel and the mma.sync kernel give the same
    bit-exact integer results; the engine is read when the plan is created.  Sizes cover an odd number of
    tile rows and columns (padding tiles in the last pair), K not a multiple of 256 and a single tile."""
    if engine == "pair":
        monkeypatch.delenv("FMM_OZAKI_ENGINE", raising=False)
    else:
        monkeypatch.setenv("FMM_OZAKI_ENGINE", engine)
    algo = fmm.fmm_algo_builtin(name)
    plan = fmm.fmm_plan_create(n, algo, depth, dtype="f64_ozaki")
    A, B = inputs.operands(n, "integer", seed=3 * n + depth)
    assert np.array_equal(run(fmm, plan, A, B), oracle_mod.classic(A, B))
    A, B = inputs.operands(n, "uniform", seed=n)
    rows, cols, ref = ref_entries(oracle_mod, A, B)
    assert nerr(run(fmm, plan, A, B)[rows, cols], ref, A, B) <= 1e-13


@pytest.mark.parametrize("name,n", [("strassen", 1030), ("winograd", 1024)])
def test_post_additions_level_by_level_and_flattened(fmm, oracle_mod, monkeypatch, name, n):
    """Two levels of a 2 x 2 algorithm: the post-additions run level by level (each leaf product read
    once, the inner sums forming the outer products' blocks, as the recursion of Section 2 defines them)
    unless FMM_OZAKI_POSTADD=flat asks for the flattened sums.  Both are bit-exact on integers, with and
    without alpha and beta, at a peeled size (1030 = 4 * 257 + 2), and within the depth-2 tolerance of the
    oracle's Dot2 entries on real inputs; they differ only by the rounding of the sums' association."""
    algo = fmm.fmm_algo_builtin(name)
    monkeypatch.delenv("FMM_OZAKI_POSTADD", raising=False)
    level = fmm.fmm_plan_create(n, algo, 2, dtype="f64_ozaki")
    monkeypatch.setenv("FMM_OZAKI_POSTADD", "flat")
    flat = fmm.fmm_plan_create(n, algo, 2, dtype="f64_ozaki")
    monkeypatch.delenv("FMM_OZAKI_POSTADD")
    A, B = inputs.operands(n, "integer", seed=n)
    C0 = inputs.matrix(n, "integer", seed=n + 1)
    AB = oracle_mod.classic(A, B)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    for alpha, beta in [(1.0, 0.0), (-2.0, 3.0), (0.5, 1.0)]:
        for plan in (level, flat):
            dC = torch.from_numpy(C0.copy()).cuda()
            fmm.fmm_gemm_ex(plan, alpha, dA, dB, beta, dC)
            assert fmm.fmm_sync_status(plan) == 0
            assert np.array_equal(dC.cpu().numpy(), oracle_mod.axpby(alpha, AB, beta, C0)), (alpha, beta)
    A, B = inputs.operands(n, "uniform", seed=n + 2)
    rows, cols, ref = ref_entries(oracle_mod, A, B)
    C_level, C_flat = run(fmm, level, A, B), run(fmm, flat, A, B)
    assert nerr(C_level[rows, cols], ref, A, B) <= 1e-13
    assert nerr(C_flat[rows, cols], ref, A, B) <= 1e-13
    assert nerr(C_level, C_flat, A, B) <= 1e-15


@pytest.mark.parametrize("kparts", [1, 2, 3, 4])
def test_slice_gemm_k_pieces(fmm, oracle_mod, monkeypatch, kparts):
    """The CTA-pair slice GEMM may take each slice pair's K range in pieces, each accumulated in TMEM and
    folded into the int64 sums on its own (FMM_OZAKI_KPARTS, read at plan creation; the default is about
    one piece per 1024 of K).  At n = 2051 (Strassen depth 1, leaf 1025 after peeling, K padded to 9
    stages of 128) two and four pieces are uneven; every piece count gives the exact product on integers
    and stays within the depth-1 tolerance of the oracle and within 2x of the FP64 path's error on real
    inputs."""
    monkeypatch.setenv("FMM_OZAKI_KPARTS", str(kparts))
    algo = fmm.fmm_algo_builtin("strassen")
    n = 2 * 1024 + 3
    plan = fmm.fmm_plan_create(n, algo, 1, dtype="f64_ozaki")
    monkeypatch.delenv("FMM_OZAKI_KPARTS")
    A, B = inputs.operands(n, "integer", seed=kparts)
    assert np.array_equal(run(fmm, plan, A, B), oracle_mod.classic(A, B))
    A, B = inputs.operands(n, "uniform", seed=10 + kparts)
    rows, cols, ref = ref_entries(oracle_mod, A, B)
    e_oz = nerr(run(fmm, plan, A, B)[rows, cols], ref, A, B)
    e_64 = nerr(run(fmm, fmm.fmm_plan_create(n, algo, 1), A, B)[rows, cols], ref, A, B)
    assert e_oz <= 1e-13 and e_oz <= 2.0 * e_64, (e_oz, e_64)
