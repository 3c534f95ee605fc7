"""Pins for the CPU oracle against facts fixed by the paper and by mathematics.

Nothing here compares the oracle with itself: the checks are the paper's printed
tables and worked examples (Section 2), the classic product it prints as a graph
(Section 3), closed forms (products of basis matrices), exact rational arithmetic,
brute force against an independent library product on integer-valued inputs, and
the paper's principle that integer computations come out exact (abstract).
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest

from golden import algos
from paper_2312_12732_gb300 import inputs

U_DBL = 2.0 ** -53


def all_algos():
    return {
        "paper_strassen": algos.paper_strassen(),
        "strassen1969": algos.strassen1969(),
        "winograd": algos.winograd(),
        "laderman": algos.laderman(),
        "classic_graph": algos.classic_from_graph(),
    }


# ---------------------------------------------------------------- Brent checker


def test_paper_table_as_printed_needs_row_relabel(oracle_mod):
    a, b, ct, labels = algos.paper_strassen_as_printed()
    assert labels == ["C0", "C2", "C1", "C3"]
    # Rows taken in printed order as C0, C1, C2, C3: the equations fail.
    assert oracle_mod.brent_mismatches(2, a, b, ct) == 8
    # Rows placed by their printed labels: exact.
    p, U, V, W = algos.paper_strassen()
    assert oracle_mod.brent_mismatches(p, U, V, W) == 0


@pytest.mark.parametrize("name", list(all_algos()))
def test_brent_accepts_published_algorithms(oracle_mod, name):
    p, U, V, W = all_algos()[name]
    assert oracle_mod.brent_mismatches(p, U, V, W) == 0


def test_product_counts_match_fixture():
    counts = {2: 7, 3: 23}
    for factor, comp, R in algos.product_counts():
        assert int(np.prod(comp)) == factor
        assert int(np.prod([counts[c] for c in comp])) == R


@pytest.mark.parametrize("name", ["paper_strassen", "laderman"])
def test_brent_rejects_every_single_entry_change(oracle_mod, name):
    p, U, V, W = all_algos()[name]
    rng = np.random.default_rng(5)
    for X in (U, V, W):
        for idx in itertools.product(range(X.shape[0]), range(X.shape[1])):
            if name == "laderman" and rng.random() > 0.15:
                continue  # subsample the 3 x 207 entries of Laderman
            old = X[idx]
            X[idx] = old + (1 if old <= 0 else -1)
            assert oracle_mod.brent_mismatches(p, U, V, W) > 0, idx
            X[idx] = old


def test_kronecker_composition_needs_row_major_reindexing(oracle_mod):
    s = algos.paper_strassen()
    p, U, V, W = algos.kron_compose(s, s)
    assert (p, U.shape[1]) == (4, 49)
    assert oracle_mod.brent_mismatches(p, U, V, W) == 0
    p, U, V, W = algos.kron_unpermuted(s, s)
    assert oracle_mod.brent_mismatches(p, U, V, W) == 112


@pytest.mark.parametrize("first,second", [("paper_strassen", "laderman"), ("laderman", "winograd"),
                                          ("laderman", "laderman")])
def test_kronecker_compositions_of_mixed_factors(oracle_mod, first, second):
    table = all_algos()
    p, U, V, W = algos.kron_compose(table[first], table[second])
    assert U.shape[1] == table[first][1].shape[1] * table[second][1].shape[1]
    assert oracle_mod.brent_mismatches(p, U, V, W) == 0


def test_worked_examples_match_relabelled_table():
    p, U, V, W = algos.paper_strassen()
    ex = algos.worked_examples()
    for blk, prods in ex.items():
        assert sorted(np.nonzero(W[blk])[0].tolist()) == sorted(prods)
        for r, (aterms, bterms) in prods.items():
            ua = {int(t.lstrip("+-")[1:]): (-1 if t[0] == "-" else 1) for t in aterms}
            vb = {int(t.lstrip("+-")[1:]): (-1 if t[0] == "-" else 1) for t in bterms}
            assert {i: int(U[i, r]) for i in np.nonzero(U[:, r])[0]} == ua
            assert {j: int(V[j, r]) for j in np.nonzero(V[:, r])[0]} == vb
            assert W[blk, r] == 1


# ---------------------------------------------------------------- classic product


@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (7, 5, 3), (33, 17, 65), (64, 64, 64)])
def test_classic_exact_on_integers_vs_numpy(oracle_mod, M, N, K):
    rng = np.random.default_rng(M * 100 + N)
    A = rng.integers(-16, 17, size=(M, K)).astype(np.float64)
    B = rng.integers(-16, 17, size=(K, N)).astype(np.float64)
    assert np.array_equal(oracle_mod.classic(A, B), A @ B)


def test_classic_within_dot_product_bound_vs_dot2(oracle_mod):
    n = 200
    A, B = inputs.operands(n, "normal", seed=11)
    C = oracle_mod.classic(A, B)
    rows, cols = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    ref = oracle_mod.sample_dot2(A, B, rows.ravel(), cols.ravel()).reshape(n, n)
    gamma = n * U_DBL / (1 - n * U_DBL)
    bound = gamma * (np.abs(A) @ np.abs(B))
    assert np.all(np.abs(C - ref) <= bound)
    assert np.max(np.abs(C - ref)) > 0  # the two orders do differ on real data


# ---------------------------------------------------------------- Dot2


def test_dot2_exact_rational_random(oracle_mod):
    rng = np.random.default_rng(3)
    for K in (1, 2, 17, 500):
        x = rng.standard_normal(K) * 10.0 ** rng.uniform(-5, 5, K)
        y = rng.standard_normal(K)
        exact = sum(Fraction(a) * Fraction(b) for a, b in zip(x.tolist(), y.tolist()))
        got = Fraction(oracle_mod.dot2(x, y))
        # Ogita-Rump-Oishi: |res - exact| <= u |exact| + gamma_{K}^2 sum|x y|
        g = K * U_DBL / (1 - K * U_DBL)
        bound = U_DBL * abs(exact) + Fraction(g * g) * sum(Fraction(abs(a * b)) for a, b in zip(x, y))
        assert abs(got - exact) <= bound


def test_dot2_recovers_cancelled_sum(oracle_mod):
    x = np.array([1e16, 1.0, -1e16])
    y = np.array([1.0, 1.0, 1.0])
    assert oracle_mod.dot2(x, y) == 1.0
    x = np.array([2.0 ** 60, 3.0, -(2.0 ** 60), 2.0 ** -40])
    assert oracle_mod.dot2(x, np.ones(4)) == 3.0 + 2.0 ** -40


# ---------------------------------------------------------------- bilinear evaluator


def _basis(n, i, j):
    E = np.zeros((n, n))
    E[i, j] = 1.0
    return E


@pytest.mark.parametrize("name,depth", [("paper_strassen", 1), ("paper_strassen", 2), ("winograd", 2),
                                        ("strassen1969", 1), ("laderman", 1), ("classic_graph", 2)])
def test_bilinear_exhaustive_basis_pairs(oracle_mod, name, depth):
    p, U, V, W = all_algos()[name]
    n = p ** depth
    for i, j, k, l in itertools.product(range(n), repeat=4):
        C = oracle_mod.bilinear(_basis(n, i, j), _basis(n, k, l), p, U, V, W, depth)
        want = _basis(n, i, l) if j == k else np.zeros((n, n))
        assert np.array_equal(C, want), (i, j, k, l)


def test_bilinear_exhaustive_basis_pairs_444(oracle_mod):
    s = algos.paper_strassen()
    p, U, V, W = algos.kron_compose(s, s)
    for i, j, k, l in itertools.product(range(4), repeat=4):
        C = oracle_mod.bilinear(_basis(4, i, j), _basis(4, k, l), p, U, V, W, 1)
        want = _basis(4, i, l) if j == k else np.zeros((4, 4))
        assert np.array_equal(C, want)


@pytest.mark.parametrize("name", ["paper_strassen", "winograd", "laderman"])
def test_bilinear_brute_force_small_integers(oracle_mod, name):
    p, U, V, W = all_algos()[name]
    rng = np.random.default_rng(1)
    for n in (p, p * p):
        for _ in range(20):
            A = rng.integers(-9, 10, (n, n)).astype(np.float64)
            B = rng.integers(-9, 10, (n, n)).astype(np.float64)
            depth = 1 if n == p else 2
            assert np.array_equal(oracle_mod.bilinear(A, B, p, U, V, W, depth), A @ B)


@pytest.mark.parametrize("name,n,depth", [
    ("paper_strassen", 64, 1), ("paper_strassen", 64, 3), ("paper_strassen", 96, 4),
    ("winograd", 128, 3), ("strassen1969", 48, 2), ("laderman", 81, 2), ("laderman", 54, 1),
    # sizes that need peeling at one or more levels
    ("paper_strassen", 37, 1), ("paper_strassen", 101, 3), ("winograd", 77, 2), ("laderman", 50, 2),
    ("paper_strassen", 3, 2), ("laderman", 2, 1), ("paper_strassen", 1, 3)])
def test_bilinear_bit_exact_on_integer_inputs(oracle_mod, name, n, depth):
    p, U, V, W = all_algos()[name]
    A, B = inputs.operands(n, "integer", seed=n + depth)
    assert np.array_equal(oracle_mod.bilinear(A, B, p, U, V, W, depth), A @ B)


def test_composed_algorithm_equals_two_levels(oracle_mod):
    s = algos.paper_strassen()
    p4, U4, V4, W4 = algos.kron_compose(s, s)
    A, B = inputs.operands(64, "integer", seed=9)
    C1 = oracle_mod.bilinear(A, B, p4, U4, V4, W4, 1)
    C2 = oracle_mod.bilinear(A, B, *s, 2)
    assert np.array_equal(C1, C2) and np.array_equal(C1, A @ B)


def test_planted_mistakes_are_detected(oracle_mod):
    """A sign flip in U, a transposed W (c^t without relabelling), or a swapped V column
    each makes the evaluator disagree with the classic product on integer inputs."""
    p, U, V, W = algos.paper_strassen()
    A, B = inputs.operands(16, "integer", seed=4)
    ref = A @ B
    U2 = U.copy(); U2[2, 0] = -U2[2, 0]
    assert U[2, 0] != 0
    assert not np.array_equal(oracle_mod.bilinear(A, B, p, U2, V, W, 1), ref)
    a, b, ct, _ = algos.paper_strassen_as_printed()
    assert not np.array_equal(oracle_mod.bilinear(A, B, p, a, b, ct, 1), ref)
    V2 = V.copy(); V2[:, [1, 2]] = V2[:, [2, 1]]
    assert not np.array_equal(oracle_mod.bilinear(A, B, p, U, V2, W, 1), ref)


@pytest.mark.parametrize("name,depth,tol", [("paper_strassen", 1, 1e-13), ("paper_strassen", 2, 1e-13),
                                            ("paper_strassen", 3, 1e-12), ("winograd", 3, 1e-12),
                                            ("laderman", 2, 1e-13)])
def test_bilinear_real_inputs_within_normalised_tolerance(oracle_mod, name, depth, tol):
    p, U, V, W = all_algos()[name]
    n = 216 if p == 3 else 256
    A, B = inputs.operands(n, "uniform", seed=21)
    C = oracle_mod.bilinear(A, B, p, U, V, W, depth)
    rows, cols = inputs.sample_indices(n, 2048, seed=5)
    ref = oracle_mod.sample_dot2(A, B, rows, cols)
    err = np.max(np.abs(C[rows, cols] - ref)) / (n * np.abs(A).max() * np.abs(B).max())
    assert err <= tol
    assert err > 0  # fast algorithms do round differently from the exact product


def test_integer_workloads_stay_below_2p53():
    """Entries in [-16, 16]: every intermediate of depth d is bounded by
    16 * 16 * n * (max column nnz of U)^d * (max column nnz of V)^d * (max row l1 of W)^d,
    which stays below 2^53 for the integer workloads (n <= 10007, depth <= 3)."""
    for name in ("paper_strassen", "winograd", "laderman"):
        p, U, V, W = all_algos()[name]
        gu = np.abs(U).sum(0).max()
        gv = np.abs(V).sum(0).max()
        gw = np.abs(W).sum(1).max()
        for depth in (1, 2, 3):
            bound = 256.0 * 10007 * float(gu * gv * gw) ** depth
            assert bound < 2.0 ** 53, (name, depth, bound)


def test_sample_dot2_matches_classic_indices(oracle_mod):
    A = inputs.matrix(30, "integer", seed=1, m=20)
    B = inputs.matrix(20, "integer", seed=2, m=25)
    rows, cols = inputs.sample_indices(25, 100, seed=3)
    rows = rows % 30
    assert np.array_equal(oracle_mod.sample_dot2(A, B, rows, cols), (A @ B)[rows, cols])


@pytest.mark.parametrize("alpha,beta", [(1.0, 0.0), (2.0, -3.0), (-1.0, 1.0), (0.0, 5.0), (3.0, 0.0), (0.0, 0.0)])
def test_scaled_update_exact_on_integers(oracle_mod, alpha, beta):
    """alpha A B + beta C on integer inputs and small integer scalars equals the same
    expression in exact int64 arithmetic (numpy integer matmul), at a peeled size."""
    p, U, V, W = algos.paper_strassen()
    n = 37
    A, B = inputs.operands(n, "integer", seed=5)
    C0 = inputs.matrix(n, "integer", seed=8)
    ref = (int(alpha) * (A.astype(np.int64) @ B.astype(np.int64)) + int(beta) * C0.astype(np.int64))
    got = oracle_mod.scaled(alpha, A, B, beta, C0, p, U, V, W, 2)
    assert np.array_equal(got, ref.astype(np.float64))


def test_scaled_update_does_not_read_what_is_scaled_by_zero(oracle_mod):
    """beta = 0 ignores NaN in C; alpha = 0 ignores NaN in A (BLAS convention)."""
    p, U, V, W = algos.paper_strassen()
    A, B = inputs.operands(8, "integer", seed=6)
    C0 = np.full((8, 8), np.nan)
    assert np.array_equal(oracle_mod.scaled(2.0, A, B, 0.0, C0, p, U, V, W, 1), 2.0 * (A @ B))
    A_nan = A.copy()
    A_nan[3, 4] = np.nan
    C1 = inputs.matrix(8, "integer", seed=9)
    assert np.array_equal(oracle_mod.scaled(0.0, A_nan, B, -2.0, C1, p, U, V, W, 1), -2.0 * C1)
    assert np.array_equal(oracle_mod.scaled(0.0, A_nan, B, 0.0, C0, p, U, V, W, 1), np.zeros((8, 8)))


def test_scaled_update_rounds_each_term_once(oracle_mod):
    """Real scalars: every entry is fl(fl(alpha p) + fl(beta c)), checked against exact
    rational arithmetic on a few entries (error at most one rounding of the sum plus one of
    each product, i.e. within 3 ulps of the exact value scaled by the terms)."""
    rng = np.random.default_rng(11)
    P = rng.standard_normal(64)
    C = rng.standard_normal(64)
    alpha, beta = 0.7, -1.3
    got = oracle_mod.axpby(alpha, P, beta, C)
    for t in range(64):
        exact = Fraction(alpha) * Fraction(P[t]) + Fraction(beta) * Fraction(C[t])
        bound = Fraction(3 * 2.0 ** -53) * (abs(Fraction(alpha) * Fraction(P[t])) + abs(Fraction(beta) * Fraction(C[t])))
        assert abs(Fraction(got[t]) - exact) <= bound
    assert not np.array_equal(oracle_mod.axpby(beta, P, alpha, C), got)  # the roles are not symmetric


# --- rational coefficients (Section 2: the coefficients need not be integers) ---------------

from golden import rational_algos  # noqa: E402

RATIONAL = {"dyadic": rational_algos.strassen_dyadic, "thirds": rational_algos.strassen_thirds,
            "halved": rational_algos.strassen_halved}


@pytest.mark.parametrize("name", list(RATIONAL))
def test_rational_brent_accepts_derived_algorithms_and_needs_the_denominators(oracle_mod, name):
    p, U, V, W, dens = RATIONAL[name]()
    assert oracle_mod.brent_mismatches_rational(p, U, V, W, dens) == 0
    assert oracle_mod.brent_mismatches(p, U, V, W) > 0  # the numerators alone are not an algorithm
    du, dv, dw = dens
    assert oracle_mod.brent_mismatches_rational(p, U, V, W, (du * 2, dv, dw)) > 0


@pytest.mark.parametrize("name", ["dyadic", "thirds"])
def test_rational_brent_rejects_every_single_entry_change(oracle_mod, name):
    p, U, V, W, dens = RATIONAL[name]()
    for M in (U, V, W):
        for idx in zip(*np.nonzero(M)):
            M[idx] += 1
            assert oracle_mod.brent_mismatches_rational(p, U, V, W, dens) > 0
            M[idx] -= 1


def test_rational_brent_with_unit_denominators_is_the_integer_check(oracle_mod):
    for name in ("paper_strassen", "winograd", "laderman"):
        p, U, V, W = all_algos()[name]
        assert oracle_mod.brent_mismatches_rational(p, U, V, W, (1, 1, 1)) == oracle_mod.brent_mismatches(p, U, V, W)
    p, U, V, W = algos.paper_strassen()
    U2 = U.copy(); U2[0, 0] += 1
    assert oracle_mod.brent_mismatches_rational(p, U2, V, W, (1, 1, 1)) == oracle_mod.brent_mismatches(p, U2, V, W) > 0


@pytest.mark.parametrize("depth", [1, 2])
def test_rational_bilinear_exhaustive_basis_pairs_dyadic(oracle_mod, depth):
    """Power-of-two denominators: every basis pair gives the exact elementary product."""
    p, U, V, W, dens = rational_algos.strassen_dyadic()
    n = p ** depth
    for i, j, k, l in itertools.product(range(n), repeat=4):
        C = oracle_mod.bilinear_rational(_basis(n, i, j), _basis(n, k, l), p, U, V, W, dens, depth)
        want = _basis(n, i, l) if j == k else np.zeros((n, n))
        assert np.array_equal(C, want), (i, j, k, l)


def test_rational_bilinear_basis_pairs_thirds_within_rounding(oracle_mod):
    """Denominators 3 and 9: the coefficients are rounded, so basis pairs come out within a few
    ulps of the exact elementary product (and not exactly, which shows the fractions are used)."""
    p, U, V, W, dens = rational_algos.strassen_thirds()
    worst = 0.0
    for i, j, k, l in itertools.product(range(2), repeat=4):
        C = oracle_mod.bilinear_rational(_basis(2, i, j), _basis(2, k, l), p, U, V, W, dens, 1)
        want = _basis(2, i, l) if j == k else np.zeros((2, 2))
        worst = max(worst, float(np.max(np.abs(C - want))))
    assert 0.0 < worst < 64 * 2.0 ** -53


@pytest.mark.parametrize("n,depth", [(16, 1), (37, 2), (64, 3), (101, 2)])
def test_rational_bilinear_bit_exact_on_integers_dyadic(oracle_mod, n, depth):
    p, U, V, W, dens = rational_algos.strassen_dyadic()
    A, B = inputs.operands(n, "integer", seed=n + depth)
    assert np.array_equal(oracle_mod.bilinear_rational(A, B, p, U, V, W, dens, depth), A @ B)
    p, U, V, W, dens = rational_algos.strassen_halved()
    assert np.array_equal(oracle_mod.bilinear_rational(A, B, p, U, V, W, dens, depth), A @ B)


def test_rational_bilinear_with_unit_denominators_equals_integer_bilinear(oracle_mod):
    p, U, V, W = all_algos()["laderman"]
    A, B = inputs.operands(81, "uniform", seed=3)
    assert np.array_equal(oracle_mod.bilinear_rational(A, B, p, U, V, W, (1, 1, 1), 2),
                          oracle_mod.bilinear(A, B, p, U, V, W, 2))


def test_rational_bilinear_thirds_real_inputs_within_tolerance(oracle_mod):
    p, U, V, W, dens = rational_algos.strassen_thirds()
    n = 256
    A, B = inputs.operands(n, "uniform", seed=23)
    rows, cols = inputs.sample_indices(n, 2048, seed=7)
    ref = oracle_mod.sample_dot2(A, B, rows, cols)
    for depth in (1, 2):
        C = oracle_mod.bilinear_rational(A, B, p, U, V, W, dens, depth)
        assert np.max(np.abs(C[rows, cols] - ref)) / (n * np.abs(A).max() * np.abs(B).max()) <= 1e-13


def test_rational_planted_denominator_mistake_is_detected(oracle_mod):
    """Dropping a denominator (den_w = 1 instead of 2) scales the result and breaks exactness."""
    p, U, V, W, (du, dv, dw) = rational_algos.strassen_dyadic()
    A, B = inputs.operands(8, "integer", seed=2)
    assert not np.array_equal(oracle_mod.bilinear_rational(A, B, p, U, V, W, (du, dv, 1), 1), A @ B)
    with pytest.raises(ValueError):
        oracle_mod.bilinear_rational(A, B, p, U, V, W, (0, dv, dw), 1)


# --- double complex (Section 1: single and double complex are among the deployable types) ------

def _cint(n, seed, m=None):
    return inputs.matrix(n, "integer", seed=seed, m=m) + 1j * inputs.matrix(n, "integer", seed=seed + 50, m=m)


@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (7, 5, 3), (33, 17, 65)])
def test_classic_complex_exact_on_integers_vs_numpy(oracle_mod, M, N, K):
    A = _cint(M, 3, m=K)
    B = _cint(K, 4, m=N)
    assert np.array_equal(oracle_mod.classic_complex(A, B), A @ B)


def test_classic_complex_reduces_to_the_real_oracle(oracle_mod):
    """Zero imaginary parts give the real classic product bit for bit (and zero imaginary part);
    a purely imaginary A gives i times it; conjugating both operands conjugates the result."""
    A, B = inputs.operands(40, "uniform", seed=6)
    C = oracle_mod.classic_complex(A + 0j, B + 0j)
    assert np.array_equal(C.real, oracle_mod.classic(A, B)) and not C.imag.any()
    C = oracle_mod.classic_complex(1j * A, B + 0j)
    assert np.array_equal(C.imag, oracle_mod.classic(A, B)) and not C.real.any()
    Z1 = A + 1j * inputs.matrix(40, "normal", seed=7)
    Z2 = B + 1j * inputs.matrix(40, "normal", seed=8)
    assert np.array_equal(oracle_mod.classic_complex(Z1.conj(), Z2.conj()), oracle_mod.classic_complex(Z1, Z2).conj())


def test_classic_complex_within_rounding_of_dot2(oracle_mod):
    """Each part of a complex dot product is a real dot product of length 2K (re: ar br - ai bi,
    im: ar bi + ai br); compared with Dot2 of those vectors, within the dot-product bound."""
    n = 64
    Z1 = inputs.matrix(n, "uniform", seed=11) + 1j * inputs.matrix(n, "uniform", seed=12)
    Z2 = inputs.matrix(n, "uniform", seed=13) + 1j * inputs.matrix(n, "uniform", seed=14)
    C = oracle_mod.classic_complex(Z1, Z2)
    for i, j in [(0, 0), (5, 9), (63, 63), (17, 40)]:
        a, b = Z1[i, :], Z2[:, j]
        re = oracle_mod.dot2(np.concatenate([a.real, -a.imag]), np.concatenate([b.real, b.imag]))
        im = oracle_mod.dot2(np.concatenate([a.real, a.imag]), np.concatenate([b.imag, b.real]))
        bound = 2 * n * 2.0 ** -53 * 2 * n
        assert abs(C[i, j].real - re) <= bound and abs(C[i, j].imag - im) <= bound


@pytest.mark.parametrize("depth", [1, 2])
def test_bilinear_complex_exhaustive_basis_pairs(oracle_mod, depth):
    """(s E_ij)(t E_kl) = s t delta_jk E_il for s, t in {1, i}: every basis pair of both parts."""
    p, U, V, W = algos.paper_strassen()
    n = p ** depth
    for i, j, k, l in itertools.product(range(n), repeat=4):
        for s, t in ((1, 1j), (1j, 1), (1j, 1j)):
            C = oracle_mod.bilinear_complex(s * _basis(n, i, j), t * _basis(n, k, l), p, U, V, W, depth)
            want = (s * t * _basis(n, i, l)) if j == k else np.zeros((n, n), dtype=complex)
            assert np.array_equal(C, want), (i, j, k, l, s, t)


@pytest.mark.parametrize("name,n,depth", [("paper_strassen", 64, 3), ("winograd", 77, 2), ("laderman", 50, 2),
                                          ("paper_strassen", 101, 2)])
def test_bilinear_complex_bit_exact_on_integers(oracle_mod, name, n, depth):
    p, U, V, W = all_algos()[name]
    A, B = _cint(n, n), _cint(n, n + 1)
    assert np.array_equal(oracle_mod.bilinear_complex(A, B, p, U, V, W, depth), A @ B)


def test_bilinear_complex_real_parts_match_the_real_recursion(oracle_mod):
    p, U, V, W = all_algos()["winograd"]
    A, B = inputs.operands(96, "uniform", seed=15)
    C = oracle_mod.bilinear_complex(A + 0j, B + 0j, p, U, V, W, 2)
    assert np.array_equal(C.real, oracle_mod.bilinear(A, B, p, U, V, W, 2)) and not C.imag.any()


def test_bilinear_complex_real_inputs_within_tolerance(oracle_mod):
    p, U, V, W = algos.paper_strassen()
    n = 128
    Z1 = inputs.matrix(n, "uniform", seed=16) + 1j * inputs.matrix(n, "uniform", seed=17)
    Z2 = inputs.matrix(n, "uniform", seed=18) + 1j * inputs.matrix(n, "uniform", seed=19)
    C = oracle_mod.bilinear_complex(Z1, Z2, p, U, V, W, 2)
    ref = oracle_mod.classic_complex(Z1, Z2)
    assert np.max(np.abs(C - ref)) / (n * np.abs(Z1).max() * np.abs(Z2).max()) <= 1e-13


# --- rectangular algorithms <m,k,n;R> (Section 2: factor-6 and factor-12 problems through
#     non-square basic products composed by Kronecker products) ---------------------------------

from golden import rect_algos  # noqa: E402


def _rect_family():
    s = rect_algos.strassen_223()
    return {"classic_232": rect_algos.classic(2, 3, 2), "classic_314": rect_algos.classic(3, 1, 4),
            "strassen_223": s, "transpose_322": rect_algos.transpose(s), "cyclic_232": rect_algos.cyclic(s),
            "cyclic2_322": rect_algos.cyclic(rect_algos.cyclic(s)),
            "compose_466": rect_algos.compose(s, rect_algos.cyclic(s))}


@pytest.mark.parametrize("name", list(_rect_family()))
def test_rect_brent_accepts_constructed_algorithms(oracle_mod, name):
    m, k, n, U, V, W = _rect_family()[name]
    assert oracle_mod.rect_brent_mismatches(m, k, n, U, V, W) == 0


def test_rect_brent_rejects_every_single_entry_change(oracle_mod):
    m, k, n, U, V, W = rect_algos.strassen_223()
    for M in (U, V, W):
        for idx in itertools.product(range(M.shape[0]), range(M.shape[1])):
            M[idx] += 1
            assert oracle_mod.rect_brent_mismatches(m, k, n, U, V, W) > 0
            M[idx] -= 1


def test_rect_brent_on_square_tables_is_the_square_check(oracle_mod):
    for name in ("paper_strassen", "winograd", "laderman"):
        p, U, V, W = all_algos()[name]
        assert oracle_mod.rect_brent_mismatches(p, p, p, U, V, W) == oracle_mod.brent_mismatches(p, U, V, W) == 0
        U2 = U.copy(); U2[1, 2] += 1
        assert oracle_mod.rect_brent_mismatches(p, p, p, U2, V, W) == oracle_mod.brent_mismatches(p, U2, V, W) > 0


def test_rect_symmetries_need_their_grid_transposes(oracle_mod):
    """Swapping U and V without transposing their block grids, or a Kronecker product without the
    row-major re-indexing, is not an algorithm."""
    m, k, n, U, V, W = rect_algos.strassen_223()
    assert oracle_mod.rect_brent_mismatches(n, k, m, V, U, W.copy()) > 0
    s = rect_algos.strassen_223()
    c = rect_algos.cyclic(s)
    plain = (4, 6, 6, np.kron(s[3], c[3]).astype(np.int32), np.kron(s[4], c[4]).astype(np.int32),
             np.kron(s[5], c[5]).astype(np.int32))
    # np.kron of the rows orders the composed block index (a1, b1, a2, b2), not row-major (a1, a2, b1, b2)
    assert oracle_mod.rect_brent_mismatches(*plain) > 0


def test_rect_bilinear_exhaustive_basis_pairs(oracle_mod):
    s = rect_algos.strassen_223()
    for i, j, k, l in itertools.product(range(2), range(2), range(2), range(3)):
        A = np.zeros((2, 2)); A[i, j] = 1.0
        B = np.zeros((2, 3)); B[k, l] = 1.0
        want = np.zeros((2, 3))
        if j == k:
            want[i, l] = 1.0
        assert np.array_equal(oracle_mod.rect_bilinear(A, B, [s]), want), (i, j, k, l)


@pytest.mark.parametrize("M,K,N,levels", [(8, 8, 12, 1), (37, 29, 41, 2), (24, 36, 36, 2), (5, 3, 2, 3)])
def test_rect_bilinear_bit_exact_on_integers(oracle_mod, M, K, N, levels):
    s = rect_algos.strassen_223()
    seq = [s, rect_algos.cyclic(s), rect_algos.cyclic(rect_algos.cyclic(s))][:levels]
    A = inputs.matrix(M, "integer", seed=M, m=K)
    B = inputs.matrix(K, "integer", seed=N, m=N)
    assert np.array_equal(oracle_mod.rect_bilinear(A, B, seq), A @ B)


def test_rect_bilinear_with_square_levels_is_the_square_recursion(oracle_mod):
    p, U, V, W = algos.paper_strassen()
    A, B = inputs.operands(101, "uniform", seed=12)
    sq = (p, p, p, U, V, W)
    assert np.array_equal(oracle_mod.rect_bilinear(A, B, [sq, sq, sq]), oracle_mod.bilinear(A, B, p, U, V, W, 3))


def test_composed_rect_algorithm_equals_nested_levels(oracle_mod):
    """One level of compose(a, b) computes exactly what level a over level b computes (exact on
    integers; within rounding on real inputs, where the summation orders differ)."""
    s = rect_algos.strassen_223()
    c = rect_algos.cyclic(s)
    comp = rect_algos.compose(s, c)
    A = inputs.matrix(40, "integer", seed=3, m=60)
    B = inputs.matrix(60, "integer", seed=4, m=60)
    assert np.array_equal(oracle_mod.rect_bilinear(A, B, [comp]), oracle_mod.rect_bilinear(A, B, [s, c]))
    A = inputs.matrix(40, "uniform", seed=5, m=60)
    B = inputs.matrix(60, "uniform", seed=6, m=60)
    d = oracle_mod.rect_bilinear(A, B, [comp]) - oracle_mod.rect_bilinear(A, B, [s, c])
    assert np.max(np.abs(d)) <= 1e-13 * 60


def test_square_12_from_three_rotations(oracle_mod):
    """<2,2,3;11> (x) <2,3,2;11> (x) <3,2,2;11> is a square <12;1331> that the square recursion runs."""
    m, k, n, U, V, W = rect_algos.strassen_12()
    assert (m, k, n, U.shape[1]) == (12, 12, 12, 1331)
    assert oracle_mod.brent_mismatches(12, U, V, W) == 0
    A, B = inputs.operands(24, "integer", seed=9)
    assert np.array_equal(oracle_mod.bilinear(A, B, 12, U, V, W, 1), A @ B)


def test_rect_bilinear_random_shapes_exact_on_integers(oracle_mod):
    """Seeded random shapes (including ones smaller than a split factor and ones needing peeling in
    every dimension) and random level sequences of <2,2,3;11> rotations: exact on integers."""
    rng = np.random.default_rng(77)
    s = rect_algos.strassen_223()
    rots = [s, rect_algos.cyclic(s), rect_algos.cyclic(rect_algos.cyclic(s)), rect_algos.transpose(s)]
    for _ in range(15):
        M, K, N = (int(x) for x in rng.integers(1, 40, size=3))
        levels = [rots[int(i)] for i in rng.integers(len(rots), size=int(rng.integers(0, 4)))]
        A = rng.integers(-16, 17, size=(M, K)).astype(np.float64)
        B = rng.integers(-16, 17, size=(K, N)).astype(np.float64)
        assert np.array_equal(oracle_mod.rect_bilinear(A, B, levels), A @ B), (M, K, N, len(levels))
