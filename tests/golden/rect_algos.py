"""Rectangular bilinear algorithms <m,k,n;R> for tests, built from the paper's tables.

Section 2 discusses solving a square problem of factor 6 or 12 through non-square basic products
(2x3x3 with 3x2x3 and so on) composed by Kronecker products. No rectangular table is printed, so
these are constructed here. Each is a tuple (m, k, n, U, V, W): U is (m k) x R over A's m x k block
grid, V is (k n) x R over B's k x n grid, and W is (m n) x R over C's m x n grid, all row-major.
Tests check the Brent equations of every result rather than assuming them.

* classic(m, k, n): one product per (i, j, l), A_ij B_jl -> C_il.
* strassen_223(): <2,2,3;11>, the paper's Strassen on the first two block columns of B and the
  four classic products A_i0 B_02, A_i1 B_12 for the third.
* transpose(alg): <n,k,m> from (A B)^T = B^T A^T.
* cyclic(alg): <k,n,m>. The trilinear form sum A_ab B_bd C_ad is invariant under rotating its three
  factors, so (U, V, W) becomes (V, W^T, U^T), with ^T transposing the block grid.
* compose(a, b): <m1 m2, k1 k2, n1 n2; R1 R2>, where block (i1, i2) of a composed grid is
  row-major (i1 m2 + i2) and product (r1, r2) is r1 R2 + r2, the first factor outermost.
"""
from __future__ import annotations

import numpy as np

from . import algos


def classic(m: int, k: int, n: int):
    R = m * k * n
    U = np.zeros((m * k, R), dtype=np.int32)
    V = np.zeros((k * n, R), dtype=np.int32)
    W = np.zeros((m * n, R), dtype=np.int32)
    r = 0
    for i in range(m):
        for j in range(k):
            for l in range(n):
                U[i * k + j, r] = 1
                V[j * n + l, r] = 1
                W[i * n + l, r] = 1
                r += 1
    return m, k, n, U, V, W


def strassen_223():
    p, Us, Vs, Ws = algos.paper_strassen()
    R = 11
    U = np.zeros((4, R), dtype=np.int32)
    V = np.zeros((6, R), dtype=np.int32)
    W = np.zeros((6, R), dtype=np.int32)
    U[:, :7] = Us
    for j in range(2):
        for l in range(2):
            V[j * 3 + l, :7] = Vs[j * 2 + l]
            W[j * 3 + l, :7] = Ws[j * 2 + l]
    # C_i2 = A_i0 B_02 + A_i1 B_12, products 7 .. 10
    r = 7
    for i in range(2):
        for j in range(2):
            U[i * 2 + j, r] = 1
            V[j * 3 + 2, r] = 1
            W[i * 3 + 2, r] = 1
            r += 1
    return 2, 2, 3, U, V, W


def _grid_t(M, rows, cols):
    """Rows of M indexed over a rows x cols grid, re-indexed over the transposed grid."""
    out = np.empty_like(M)
    for a in range(rows):
        for b in range(cols):
            out[b * rows + a] = M[a * cols + b]
    return out


def transpose(alg):
    m, k, n, U, V, W = alg
    return n, k, m, _grid_t(V, k, n), _grid_t(U, m, k), _grid_t(W, m, n)


def cyclic(alg):
    m, k, n, U, V, W = alg
    return k, n, m, V.copy(), _grid_t(W, m, n), _grid_t(U, m, k)


def _kron_grid(X1, r1, c1, X2, r2, c2):
    R1, R2 = X1.shape[1], X2.shape[1]
    out = np.zeros((r1 * r2 * c1 * c2, R1 * R2), dtype=np.int64)
    for a1 in range(r1):
        for b1 in range(c1):
            for a2 in range(r2):
                for b2 in range(c2):
                    row = (a1 * r2 + a2) * (c1 * c2) + (b1 * c2 + b2)
                    out[row] = np.outer(X1[a1 * c1 + b1], X2[a2 * c2 + b2]).ravel()
    return out.astype(np.int32)


def compose(a, b):
    m1, k1, n1, U1, V1, W1 = a
    m2, k2, n2, U2, V2, W2 = b
    return (m1 * m2, k1 * k2, n1 * n2, _kron_grid(U1, m1, k1, U2, m2, k2), _kron_grid(V1, k1, n1, V2, k2, n2),
            _kron_grid(W1, m1, n1, W2, m2, n2))


def strassen_12():
    """<12,12,12;1331> = <2,2,3;11> (x) <2,3,2;11> (x) <3,2,2;11>, the three rotations of strassen_223."""
    s = strassen_223()
    return compose(compose(s, cyclic(s)), cyclic(cyclic(s)))
