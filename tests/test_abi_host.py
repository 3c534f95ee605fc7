"""Host-side checks of the C ABI (no GPU): the library loads, exports every
declared symbol, carries the paper's tables, and validates algorithms exactly."""
import ctypes
import os
import re

import numpy as np
import pytest

from golden import algos

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fmm():
    from paper_2312_12732_gb300 import _build

    _build.build()
    import paper_2312_12732_gb300 as m

    return m


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(fmm_\w+)\s*\(", text)
    return sorted(set(names))


def test_library_exports_every_declared_symbol(fmm):
    lib = ctypes.CDLL(os.path.join(ROOT, "paper_2312_12732_gb300", "libfmm.so"))
    names = declared_functions()
    assert len(names) >= 14
    for name in names:
        assert hasattr(lib, name), name
    bound = {s[0] for s in fmm._binding.SIGNATURES}
    assert set(names) <= bound, set(names) - bound


def test_status_strings(fmm):
    for s in range(8):
        assert fmm.fmm_status_string(s)
    assert fmm.fmm_status_string(2) == "algorithm fails the Brent equations"


@pytest.mark.parametrize("name,golden", [("strassen", algos.paper_strassen), ("winograd", algos.winograd),
                                         ("strassen1969", algos.strassen1969), ("laderman", algos.laderman),
                                         ("classic2", algos.classic_from_graph)])
def test_builtin_tables_equal_golden(fmm, name, golden):
    a = fmm.fmm_algo_builtin(name)
    p, U, V, W = golden()
    assert a.p == p
    assert np.array_equal(a.U, U) and np.array_equal(a.V, V) and np.array_equal(a.W, W)
    assert fmm.fmm_algo_brent_mismatches(a) == 0


def test_unknown_builtin(fmm):
    with pytest.raises(fmm.FmmError) as e:
        fmm.fmm_algo_builtin("bini")
    assert e.value.status == 7


def test_brent_rejects_paper_ct_without_relabel(fmm):
    a, b, ct, _ = algos.paper_strassen_as_printed()
    assert fmm.fmm_algo_brent_mismatches(fmm.Algo(2, a, b, ct)) == 8
    W = fmm.fmm_algo_from_transposed_c(2, ct)
    # the printed rows C0, C2, C1, C3 are exactly C transposed, row-major
    assert fmm.fmm_algo_brent_mismatches(fmm.Algo(2, a, b, W)) == 0
    assert np.array_equal(W, algos.paper_strassen()[3])


def test_brent_rejects_single_changes(fmm):
    s = fmm.fmm_algo_builtin("strassen")
    for X in ("U", "V", "W"):
        T = getattr(s, X)
        for idx in np.ndindex(*T.shape):
            M = {k: getattr(s, k).copy() for k in "UVW"}
            M[X][idx] += 1
            assert fmm.fmm_algo_brent_mismatches(fmm.Algo(2, M["U"], M["V"], M["W"])) > 0


def test_compose_matches_reindexed_kronecker(fmm):
    s = fmm.fmm_algo_builtin("strassen")
    lad = fmm.fmm_algo_builtin("laderman")
    for a1, a2, g1, g2 in ((s, s, algos.paper_strassen(), algos.paper_strassen()),
                           (s, lad, algos.paper_strassen(), algos.laderman())):
        c = fmm.fmm_algo_compose(a1, a2)
        p, U, V, W = algos.kron_compose(g1, g2)
        assert c.p == p and np.array_equal(c.U, U) and np.array_equal(c.V, V) and np.array_equal(c.W, W)
        assert fmm.fmm_algo_brent_mismatches(c) == 0
    assert fmm.algorithm("strassen", 2).R == 49


def test_plan_create_rejects_bad_requests_before_touching_the_gpu(fmm):
    s = fmm.fmm_algo_builtin("strassen")
    bad = fmm.Algo(2, s.U, s.V, s.W[[0, 2, 1, 3]])
    with pytest.raises(fmm.FmmError) as e:
        fmm.fmm_plan_create(64, bad, 1)
    assert e.value.status == 2
    for n, depth in ((0, 1), (64, -1), (3, 2)):
        with pytest.raises(fmm.FmmError) as e:
            fmm.fmm_plan_create(n, s, depth)
        assert e.value.status == 1
    with pytest.raises(fmm.FmmError) as e:
        fmm.fmm_plan_create(64, s, 1, schedule="hybrid", materialize_levels=2)
    assert e.value.status == 1


def test_binding_requires_built_library(monkeypatch, tmp_path):
    from paper_2312_12732_gb300 import _binding

    monkeypatch.setattr(_binding, "_lib", None)
    monkeypatch.setattr(_binding, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        _binding.lib()


def test_scaled_entry_points_validate_before_touching_the_gpu(fmm):
    """fmm_gemm_ex rejects a NULL plan or operand, and an empty fmm_gemm_batched_ex is a no-op;
    neither makes a CUDA call on these paths."""
    lib = fmm.lib()
    assert lib.fmm_gemm_ex(None, 1.0, None, None, 0.0, None, None) == 1
    assert lib.fmm_gemm_batched_ex(None, None, None, None, None, None, 0, None) == 0
    assert lib.fmm_gemm_batched_ex(None, None, None, None, None, None, -1, None) == 1


def test_rational_brent_agrees_with_the_oracle(fmm, oracle_mod):
    """The library's rational Brent check gives the oracle's count on the derived non-integer
    algorithms, on single-entry changes and on a wrong denominator; bad input gives -1."""
    from golden import rational_algos

    for make in (rational_algos.strassen_dyadic, rational_algos.strassen_thirds, rational_algos.strassen_halved):
        p, U, V, W, dens = make()
        assert fmm.fmm_algo_rational_brent_mismatches(fmm.RationalAlgo(p, U, V, W, dens)) == 0
        for wrong in ((dens[0] * 2, dens[1], dens[2]), (dens[0], dens[1], dens[2] + 1)):
            assert (fmm.fmm_algo_rational_brent_mismatches(fmm.RationalAlgo(p, U, V, W, wrong))
                    == oracle_mod.brent_mismatches_rational(p, U, V, W, wrong) > 0)
        U2 = U.copy()
        U2[1, 3] += 1
        assert (fmm.fmm_algo_rational_brent_mismatches(fmm.RationalAlgo(p, U2, V, W, dens))
                == oracle_mod.brent_mismatches_rational(p, U2, V, W, dens) > 0)
        assert fmm.fmm_algo_rational_brent_mismatches(fmm.RationalAlgo(p, U, V, W, (0, 1, 1))) == -1
    big = np.full((4, 7), 1 << 30, dtype=np.int32)
    assert fmm.fmm_algo_rational_brent_mismatches(fmm.RationalAlgo(2, big, big, big, (1, 1, 1))) == -1


def test_rational_plan_create_rejects_bad_algorithms_before_touching_the_gpu(fmm):
    from golden import rational_algos

    p, U, V, W, (du, dv, dw) = rational_algos.strassen_dyadic()
    with pytest.raises(fmm.FmmError) as e:
        fmm.fmm_plan_create(64, fmm.RationalAlgo(p, U, V, W, (du, dv, dw * 2)), 1)
    assert e.value.status == 2  # FMM_ERR_BRENT
    with pytest.raises(fmm.FmmError) as e:
        fmm.fmm_plan_create(64, fmm.RationalAlgo(p, U, V, W, (du, 0, dw)), 1)
    assert e.value.status == 1  # FMM_ERR_INVALID


def test_binding_checks_operands_before_calling_the_library(fmm):
    """Tensor checks happen in the binding, before any C call: dtype (float64 for real plans,
    complex128 for complex ones), shape, contiguity, and device."""
    import torch

    n = 8
    real = fmm.Plan(0, n, None, 1, "f64")
    cplx = fmm.Plan(0, n, None, 1, "c128")
    X = torch.zeros(n, n, dtype=torch.float64)
    Z = torch.zeros(n, n, dtype=torch.complex128)
    with pytest.raises(ValueError, match="CUDA device"):
        fmm.fmm_gemm(real, X, X, X)
    with pytest.raises(ValueError, match="float64"):
        fmm.fmm_gemm(real, Z, Z, Z)
    with pytest.raises(ValueError, match="complex128"):
        fmm.fmm_gemm_ex(cplx, 1.0, X, X, 0.0, X)
    with pytest.raises(ValueError, match="shape"):
        fmm.fmm_gemm(real, torch.zeros(n, n + 1, dtype=torch.float64), X, X)
    with pytest.raises(ValueError, match="contiguous"):
        fmm.fmm_gemm(real, X.t().contiguous().t()[:, :], X.t(), X)
    with pytest.raises(ValueError, match="float64"):
        fmm.fmm_gemm_host(real, Z, Z, Z)  # host path: a complex tensor for a real plan
    with pytest.raises(ValueError, match="needs out"):
        fmm.gemm(X, X, beta=1.0)
    real.handle = None
    cplx.handle = None


def test_rect_tables_match_the_golden_constructions(fmm, oracle_mod):
    """The library's <2,2,3;11>, its transpose and rotations, compositions and classic tables equal
    the independent constructions in tests/golden/rect_algos.py entry for entry, and both Brent
    implementations accept them."""
    from golden import rect_algos

    def same(lib_alg, gold):
        m, k, n, U, V, W = gold
        assert (lib_alg.m, lib_alg.k, lib_alg.n) == (m, k, n)
        assert np.array_equal(lib_alg.U, U) and np.array_equal(lib_alg.V, V) and np.array_equal(lib_alg.W, W)
        assert fmm.fmm_algo_rect_brent_mismatches(lib_alg) == 0 == oracle_mod.rect_brent_mismatches(*gold)

    s = fmm.fmm_algo_rect_builtin("strassen_2x2x3")
    g = rect_algos.strassen_223()
    same(s, g)
    same(fmm.fmm_algo_rect_transpose(s), rect_algos.transpose(g))
    same(fmm.fmm_algo_rect_cyclic(s), rect_algos.cyclic(g))
    c, gc = fmm.fmm_algo_rect_cyclic(s), rect_algos.cyclic(g)
    same(fmm.fmm_algo_rect_compose(s, c), rect_algos.compose(g, gc))
    same(fmm.fmm_algo_rect_classic(3, 1, 4), rect_algos.classic(3, 1, 4))
    sq = fmm.fmm_algo_rect_compose(fmm.fmm_algo_rect_compose(s, c), fmm.fmm_algo_rect_cyclic(c))
    same(sq, rect_algos.strassen_12())
    a = fmm.fmm_algo_rect_as_square(sq)
    assert (a.p, a.R) == (12, 1331) and fmm.fmm_algo_brent_mismatches(a) == 0


def test_rect_brent_agrees_with_the_oracle_on_changes(fmm, oracle_mod):
    s = fmm.fmm_algo_rect_builtin("strassen_2x2x3")
    for M in ("U", "V", "W"):
        for idx in [(0, 0), (1, 7), (3, 10)] if M == "U" else [(2, 7), (5, 10), (4, 3)]:
            t = fmm.RectAlgo(s.m, s.k, s.n, s.U.copy(), s.V.copy(), s.W.copy())
            getattr(t, M)[idx] += 1
            got = fmm.fmm_algo_rect_brent_mismatches(t)
            assert got == oracle_mod.rect_brent_mismatches(t.m, t.k, t.n, t.U, t.V, t.W) > 0


def test_rect_compose_of_square_tables_is_the_square_compose(fmm):
    a = fmm.fmm_algo_builtin("strassen")
    b = fmm.fmm_algo_builtin("laderman")
    ra = fmm.RectAlgo(2, 2, 2, a.U, a.V, a.W)
    rb = fmm.RectAlgo(3, 3, 3, b.U, b.V, b.W)
    rc = fmm.fmm_algo_rect_compose(ra, rb)
    sc = fmm.fmm_algo_compose(a, b)
    assert np.array_equal(rc.U, sc.U) and np.array_equal(rc.V, sc.V) and np.array_equal(rc.W, sc.W)


def test_rect_as_square_rejects_non_square(fmm):
    with pytest.raises(fmm.FmmError) as e:
        fmm.fmm_algo_rect_as_square(fmm.fmm_algo_rect_builtin("strassen_2x2x3"))
    assert e.value.status == 3  # FMM_ERR_UNSUPPORTED
    with pytest.raises(fmm.FmmError):
        fmm.fmm_algo_rect_builtin("no_such_algorithm")


def test_f32_entry_point_validates_before_touching_the_gpu(fmm):
    import torch

    assert fmm.lib().fmm_gemm_f32_ex(None, 1.0, None, None, 0.0, None, None) == 1
    plan = fmm.Plan(0, 8, None, 1, "f32")
    with pytest.raises(ValueError, match="float32"):
        fmm.fmm_gemm(plan, *(torch.zeros(8, 8, dtype=torch.float64) for _ in range(3)))
    plan.handle = None


@pytest.mark.parametrize("dtype", ["f64", "f64_ozaki", "c128", "c128_3m", "f32"])
def test_every_dtype_rejects_a_broken_algorithm_before_touching_the_gpu(fmm, dtype):
    """The complex and single-precision plans wrap a real plan whose exact Brent check runs first,
    so a broken table fails the same way for every dtype, with no CUDA call."""
    a = fmm.fmm_algo_builtin("strassen")
    U = a.U.copy()
    U[0, 0] += 1
    with pytest.raises(fmm.FmmError) as e:
        fmm.fmm_plan_create(64, fmm.Algo(2, U, a.V, a.W), 1, dtype=dtype)
    assert e.value.status == 2  # FMM_ERR_BRENT
    with pytest.raises(fmm.FmmError) as e:
        fmm.fmm_plan_create(0, a, 1, dtype=dtype)
    assert e.value.status == 1  # FMM_ERR_INVALID


def test_random_symmetry_and_composition_chains(fmm, oracle_mod):
    """Seeded random chains of transposes, rotations and compositions of <2,2,3;11> and classic
    tables: the library and the independent golden construction give the same tables, and both
    Brent implementations accept every result."""
    from golden import rect_algos

    rng = np.random.default_rng(2024)
    base_lib = [fmm.fmm_algo_rect_builtin("strassen_2x2x3"), fmm.fmm_algo_rect_classic(1, 2, 2),
                fmm.fmm_algo_rect_classic(2, 1, 1)]
    base_gold = [rect_algos.strassen_223(), rect_algos.classic(1, 2, 2), rect_algos.classic(2, 1, 1)]
    for _ in range(12):
        i = int(rng.integers(len(base_lib)))
        lib_a, gold_a = base_lib[i], base_gold[i]
        for _step in range(int(rng.integers(1, 4))):
            op = int(rng.integers(3))
            if op == 0:
                lib_a, gold_a = fmm.fmm_algo_rect_transpose(lib_a), rect_algos.transpose(gold_a)
            elif op == 1:
                lib_a, gold_a = fmm.fmm_algo_rect_cyclic(lib_a), rect_algos.cyclic(gold_a)
            elif lib_a.R * 11 <= 1500:
                j = int(rng.integers(len(base_lib)))
                lib_a = fmm.fmm_algo_rect_compose(lib_a, base_lib[j])
                gold_a = rect_algos.compose(gold_a, base_gold[j])
        m, k, n, U, V, W = gold_a
        assert (lib_a.m, lib_a.k, lib_a.n) == (m, k, n)
        assert np.array_equal(lib_a.U, U) and np.array_equal(lib_a.V, V) and np.array_equal(lib_a.W, W)
        assert fmm.fmm_algo_rect_brent_mismatches(lib_a) == 0
        assert oracle_mod.rect_brent_mismatches(m, k, n, U, V, W) == 0


@pytest.mark.parametrize("dtype", ["f64", "f64_ozaki", "c128", "c128_3m", "f32"])
def test_injected_allocation_failure_returns_oom_and_leaks_nothing(fmm, dtype):
    """The library's allocation shim fails the k-th next request on demand.  k = 0 fails the plan object
    itself, k = 1 the first device allocation (the coefficient tables, or an inner plan's object); both
    are injected before any CUDA call, so this runs without a GPU.  Each must give FMM_ERR_OOM and leave
    no allocation live."""
    s = fmm.fmm_algo_builtin("strassen")
    base = fmm.fmm_debug_live_allocations()
    try:
        for k in (0, 1):
            fmm.fmm_debug_fail_allocation(k)
            with pytest.raises(fmm.FmmError) as e:
                fmm.fmm_plan_create(256, s, 1, dtype=dtype)
            assert e.value.status == 4, (k, e.value)
            assert fmm.fmm_debug_live_allocations() == base, k
    finally:
        fmm.fmm_debug_fail_allocation(-1)


def test_host_alloc_rejects_what_it_did_not_hand_out(fmm):
    """fmm_host_free: NULL is a no-op, an unknown address is FMM_ERR_INVALID.  Without a CUDA driver
    fmm_host_alloc cannot lock pages: FMM_ERR_OOM, nothing left allocated."""
    fmm.fmm_host_free(0)
    with pytest.raises(fmm.FmmError) as e:
        fmm.fmm_host_free(4096)
    assert e.value.status == 1
    hp = fmm.fmm_host_huge_page_bytes()
    assert hp == 0 or (hp & (hp - 1)) == 0
    import torch

    if torch.cuda.is_available():
        return
    base = fmm.fmm_debug_live_allocations()
    for nbytes in (64, max(hp, 1 << 21)):
        with pytest.raises(fmm.FmmError) as e:
            fmm.fmm_host_alloc(nbytes)
        assert e.value.status == 4
    assert fmm.fmm_debug_live_allocations() == base


def test_fmm_log_reports_rejected_plans_on_stderr():
    """FMM_LOG=1: a plan rejected before any CUDA call (Brent failure, bad size) leaves one line on stderr
    naming the reason; without FMM_LOG nothing is printed."""
    import subprocess
    import sys

    code = ("import sys; sys.path.insert(0, %r)\n"
            "import paper_2312_12732_gb300 as f\n"
            "s = f.fmm_algo_builtin('strassen')\n"
            "bad = f.Algo(2, s.U, s.V, s.W[[0, 2, 1, 3]])\n"
            "for args in ((64, bad, 1), (0, s, 1)):\n"
            "    try:\n"
            "        f.fmm_plan_create(*args)\n"
            "    except f.FmmError:\n"
            "        pass\n") % ROOT
    env = dict(os.environ, FMM_LOG="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stderr.splitlines() if ln.startswith("fmm: ")]
    assert len(lines) == 2, r.stderr
    assert "rejected" in lines[0] and "Brent" in lines[0] and "p=2 R=7 depth=1" in lines[0]
    assert "rejected" in lines[1] and "invalid argument" in lines[1]
    env.pop("FMM_LOG")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0 and "fmm: " not in r.stderr
