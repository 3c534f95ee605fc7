"""Parsers for the algorithm fixtures in this folder (test helpers, no method arithmetic
beyond reading signed sums of blocks).

Every parser returns (p, U, V, W) with U, V, W integer p^2 x R arrays, row-major
over blocks; W indexes the blocks of C in row-major order.
"""
from __future__ import annotations

import itertools
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def _lines(name):
    with open(os.path.join(HERE, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                yield line


def paper_strassen_as_printed():
    """The a, b, c^t tables exactly as printed (rows of c^t kept in printed order C0, C2, C1, C3)."""
    sec, rows = None, {"a": [], "b": [], "ct": []}
    labels = []
    for line in _lines("strassen_paper_2x2x2_7.txt"):
        if line.startswith("["):
            sec = line.strip("[]")
            continue
        tok = line.split()
        rows[sec].append([int(t) for t in tok[1:]])
        if sec == "ct":
            labels.append(tok[0])
    return np.array(rows["a"]), np.array(rows["b"]), np.array(rows["ct"]), labels


def paper_strassen():
    """The paper's Strassen with c^t relabelled by its printed row labels (C0, C2, C1, C3)."""
    a, b, ct, labels = paper_strassen_as_printed()
    W = np.zeros_like(ct)
    for row, lab in zip(ct, labels):
        W[int(lab[1:])] = row
    return 2, a, b, W


def _parse_products(name, p):
    """Fixtures written as 'mK = <signed aIJ sum> * <signed bIJ sum>' and 'cIJ = <signed mK sum>'."""
    prods, cs = [], {}
    for line in _lines(name):
        lhs, rhs = [s.strip() for s in line.split("=", 1)]
        if lhs.startswith("m"):
            left, right = rhs.split("*")
            prods.append((int(lhs[1:]), left.split(), right.split()))
        else:
            cs[lhs] = rhs.split()
    prods.sort()
    R = len(prods)
    assert [k for k, _, _ in prods] == list(range(1, R + 1))
    U = np.zeros((p * p, R), dtype=np.int64)
    V = np.zeros((p * p, R), dtype=np.int64)
    W = np.zeros((p * p, R), dtype=np.int64)

    def term(t):
        sign = -1 if t.startswith("-") else 1
        body = t.lstrip("+-")
        return sign, body

    for r, (_, left, right) in enumerate(prods):
        for t in left:
            s, body = term(t)
            assert body[0] == "a"
            U[(int(body[1]) - 1) * p + int(body[2]) - 1, r] += s
        for t in right:
            s, body = term(t)
            assert body[0] == "b"
            V[(int(body[1]) - 1) * p + int(body[2]) - 1, r] += s
    for lhs, terms in cs.items():
        l = (int(lhs[1]) - 1) * p + int(lhs[2]) - 1
        for t in terms:
            s, body = term(t)
            W[l, int(body[1:]) - 1] += s
    return p, U, V, W


def laderman():
    return _parse_products("laderman_3x3x3_23.txt", 3)


def winograd():
    return _parse_products("winograd_2x2x2_7.txt", 2)


def strassen1969():
    return _parse_products("strassen1969_2x2x2_7.txt", 2)


def classic_from_graph():
    """<2,2,2;8> from the printed Matrix Flow graph: one product per A-block * B-block term."""
    pat = re.compile(r"CDP\[(\d)\]\s*<<\s*(.*)")
    terms = []
    for line in _lines("classic_2x2x2_8_graph.txt"):
        mo = pat.match(line)
        l = int(mo.group(1))
        for prod in mo.group(2).split("+"):
            ia, ib = re.findall(r"\[(\d)\]", prod)
            terms.append((l, int(ia), int(ib)))
    R = len(terms)
    U = np.zeros((4, R), dtype=np.int64)
    V = np.zeros((4, R), dtype=np.int64)
    W = np.zeros((4, R), dtype=np.int64)
    for r, (l, ia, ib) in enumerate(terms):
        U[ia, r] = V[ib, r] = W[l, r] = 1
    return 2, U, V, W


def worked_examples():
    """{C block: {product: (A-terms, B-terms)}} from the worked-example fixture."""
    out, cur = {}, None
    for line in _lines("worked_examples_strassen_paper.txt"):
        if ":" in line:
            blk, _prods = [s.strip() for s in line.split(":")]
            cur = int(blk[1:])
            out[cur] = {}
        else:
            lhs, rhs = [s.strip() for s in line.split("=", 1)]
            left, right = rhs.split("*")
            out[cur][int(lhs[1:])] = (left.split(), right.split())
    return out


def product_counts():
    rows = []
    for line in _lines("product_counts.txt"):
        f, comp, R = line.split()
        rows.append((int(f), [int(x) for x in comp.split(",")], int(R)))
    return rows


def kron_compose(alg1, alg2):
    """Two-level composition (first factor outermost) with blocks re-indexed row-major
    over the (p1 p2) x (p1 p2) grid: nested block ((i1, j1), (i2, j2)) becomes
    row i1*p2 + i2, column j1*p2 + j2.  Products are numbered r1 * R2 + r2."""
    p1, U1, V1, W1 = alg1
    p2, U2, V2, W2 = alg2
    p = p1 * p2
    out = []
    for X1, X2 in ((U1, U2), (V1, V2), (W1, W2)):
        X = np.zeros((p * p, X1.shape[1] * X2.shape[1]), dtype=np.int64)
        for i1, j1, i2, j2 in itertools.product(range(p1), range(p1), range(p2), range(p2)):
            X[(i1 * p2 + i2) * p + (j1 * p2 + j2)] = np.kron(X1[i1 * p1 + j1], X2[i2 * p2 + j2])
        out.append(X)
    return (p, *out)


def kron_unpermuted(alg1, alg2):
    """Plain Kronecker products of the factor matrices (no block re-indexing)."""
    p1, U1, V1, W1 = alg1
    p2, U2, V2, W2 = alg2
    return (p1 * p2, np.kron(U1, U2), np.kron(V1, V2), np.kron(W1, W2))
