"""Bilinear algorithms with non-integer coefficients, for tests.

Section 2 of the paper allows coefficients of a, b, c that are not integers, as long as the
matrices stay sparse.  No such table is printed, so these are derived here, exactly, from the
paper's Strassen table by the change of basis every algorithm admits: for invertible p x p
matrices X, Y, Z, an algorithm for A B applied to (X A Y^-1)(Y B Z^-1) = X (A B) Z^-1 and
followed by C = X^-1 (.) Z computes A B again, with new tables

    U'[(j,l), r] = sum_{a,b} U[(a,b), r] X[a,j] Yinv[l,b]
    V'[(k,m), r] = sum_{c,d} V[(c,d), r] Y[c,k] Zinv[m,d]
    W'[(e,f), r] = sum_{i,k} Xinv[e,i] W[(i,k), r] Z[k,f]

(blocks indexed row-major, (row, col) -> row * p + col).  Rational X, Y, Z give rational
tables; each is returned as int32 numerators over one positive common denominator per matrix.
The Brent equations of every result are checked by the tests, not assumed.
"""
from __future__ import annotations

from fractions import Fraction
from math import lcm

import numpy as np

from . import algos


def _inv2(M):
    (a, b), (c, d) = M
    det = a * d - b * c
    assert det != 0
    return [[d / det, -b / det], [-c / det, a / det]]


def _frac(M):
    return [[Fraction(x) for x in row] for row in M]


def _common(T):
    """(numerators as int32 array, common denominator) of a table of Fractions."""
    den = 1
    for x in T.flat:
        den = lcm(den, x.denominator)
    num = np.array([[int(x * den) for x in row] for row in T], dtype=np.int64)
    assert np.abs(num).max() < 2 ** 31
    return num.astype(np.int32), den


def sandwich(alg, X, Y, Z):
    """The change of basis above for a 2 x 2 algorithm (p, U, V, W) and 2 x 2 matrices X, Y, Z."""
    p, U, V, W = alg
    assert p == 2
    X, Y, Z = _frac(X), _frac(Y), _frac(Z)
    Xi, Yi, Zi = _inv2(X), _inv2(Y), _inv2(Z)
    R = U.shape[1]
    U2 = np.empty((4, R), dtype=object)
    V2 = np.empty((4, R), dtype=object)
    W2 = np.empty((4, R), dtype=object)
    for r in range(R):
        for j in range(2):
            for l in range(2):
                U2[j * 2 + l, r] = sum(int(U[a * 2 + b, r]) * X[a][j] * Yi[l][b] for a in range(2) for b in range(2))
        for k in range(2):
            for m in range(2):
                V2[k * 2 + m, r] = sum(int(V[c * 2 + d, r]) * Y[c][k] * Zi[m][d] for c in range(2) for d in range(2))
        for e in range(2):
            for f in range(2):
                W2[e * 2 + f, r] = sum(Xi[e][i] * int(W[i * 2 + k, r]) * Z[k][f] for i in range(2) for k in range(2))
    (Un, du), (Vn, dv), (Wn, dw) = _common(U2), _common(V2), _common(W2)
    return p, Un, Vn, Wn, (du, dv, dw)


def strassen_dyadic():
    """Strassen in a basis with power-of-two denominators (1/2, 1/4): every coefficient is exact
    in binary64, so integer inputs still give exact products."""
    return sandwich(algos.paper_strassen(), [[2, 0], [1, 1]], [[1, 1], [0, 2]], [[1, 0], [1, 2]])


def strassen_thirds():
    """Strassen in a basis with denominators 3 and 9: coefficients such as 1/3 are not binary64
    numbers, so results are compared by tolerance only."""
    return sandwich(algos.paper_strassen(), [[3, 0], [1, 1]], [[1, 0], [1, 3]], [[1, 1], [0, 3]])


def strassen_halved():
    """The paper's Strassen with U / 2 and W * 2 (as numerators over den_u = 2)."""
    p, U, V, W = algos.paper_strassen()
    return p, U.copy(), V.copy(), (2 * W).astype(np.int32), (2, 1, 1)
