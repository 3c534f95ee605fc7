// Rectangular bilinear algorithms <m,k,n;R> on the host (Section 2: a square
// problem of split factor 6 or 12 can be solved through non-square basic
// products, 2x3x3 with 3x2x3 and so on, composed by Kronecker products).
// A is split into an m x k grid of blocks, B into k x n, C into m x n, each
// indexed row-major; U is (m k) x R, V is (k n) x R, W is (m n) x R.  The GPU
// path multiplies square operands, so a rectangular algorithm reaches it as a
// factor of a square composition (fmm_algo_rect_as_square).
#include "fmm.h"

#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

namespace {

bool rect_ok(const fmm_algo_rect_t *a) {
    return a && a->m >= 1 && a->k >= 1 && a->n >= 1 && a->R >= 1 && a->U && a->V && a->W &&
           (long long)a->m * a->k * a->R < (1LL << 28) && (long long)a->k * a->n * a->R < (1LL << 28) &&
           (long long)a->m * a->n * a->R < (1LL << 28);
}

// Block (a, b) of an r x c grid re-indexed over the transposed c x r grid.
void grid_transpose(const int32_t *X, int rows, int cols, int R, int32_t *out) {
    for (int a = 0; a < rows; ++a)
        for (int b = 0; b < cols; ++b)
            std::memcpy(out + (int64_t)(b * rows + a) * R, X + (int64_t)(a * cols + b) * R, sizeof(int32_t) * R);
}

// Row-major Kronecker product of two coefficient tables over r1 x c1 and
// r2 x c2 block grids: composed block (a1 r2 + a2, b1 c2 + b2), product
// r1 R2 + r2 (the first factor is the outer recursion level).
void kron_grid(const int32_t *X1, int r1, int c1, int R1, const int32_t *X2, int r2, int c2, int R2, int32_t *out) {
    const int64_t R = (int64_t)R1 * R2;
    for (int a1 = 0; a1 < r1; ++a1)
        for (int b1 = 0; b1 < c1; ++b1)
            for (int a2 = 0; a2 < r2; ++a2)
                for (int b2 = 0; b2 < c2; ++b2) {
                    const int64_t row = (int64_t)(a1 * r2 + a2) * (c1 * c2) + (b1 * c2 + b2);
                    const int32_t *x1 = X1 + (int64_t)(a1 * c1 + b1) * R1;
                    const int32_t *x2 = X2 + (int64_t)(a2 * c2 + b2) * R2;
                    for (int s1 = 0; s1 < R1; ++s1)
                        for (int s2 = 0; s2 < R2; ++s2) out[row * R + (int64_t)s1 * R2 + s2] = x1[s1] * x2[s2];
                }
}

// <2,2,3;11>: Strassen on the first two block columns of B and C, and the four
// classic products A_i0 B_02, A_i1 B_12 for the third.
struct Rect223 {
    std::vector<int32_t> U, V, W;
};

const Rect223 &rect_223() {
    static Rect223 t;
    static std::once_flag once;
    std::call_once(once, [] {
        fmm_algo_t s{};
        fmm_algo_builtin("strassen", &s);
        const int R = 11;
        t.U.assign(4 * R, 0);
        t.V.assign(6 * R, 0);
        t.W.assign(6 * R, 0);
        for (int x = 0; x < 4; ++x)
            for (int r = 0; r < 7; ++r) t.U[x * R + r] = s.U[x * 7 + r];
        for (int j = 0; j < 2; ++j)
            for (int l = 0; l < 2; ++l)
                for (int r = 0; r < 7; ++r) {
                    t.V[(j * 3 + l) * R + r] = s.V[(j * 2 + l) * 7 + r];
                    t.W[(j * 3 + l) * R + r] = s.W[(j * 2 + l) * 7 + r];
                }
        int r = 7;
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j, ++r) {
                t.U[(i * 2 + j) * R + r] = 1;
                t.V[(j * 3 + 2) * R + r] = 1;
                t.W[(i * 3 + 2) * R + r] = 1;
            }
    });
    return t;
}

}  // namespace

extern "C" int64_t fmm_algo_rect_brent_mismatches(const fmm_algo_rect_t *a) {
    if (!rect_ok(a)) return -1;
    const int m = a->m, k = a->k, n = a->n, R = a->R;
    // sum_r U[(i,j)] V[(j2,l)] W[(i2,l2)] over the nonzeros of each product,
    // keyed by the triple of block indices; then every triple against
    // delta(j,j2) delta(i,i2) delta(l,l2)
    const int64_t nu = (int64_t)m * k, nv = (int64_t)k * n, nw = (int64_t)m * n;
    std::unordered_map<int64_t, int64_t> acc;
    std::vector<int> iu, iv, iw;
    for (int r = 0; r < R; ++r) {
        iu.clear(); iv.clear(); iw.clear();
        for (int64_t x = 0; x < nu; ++x) if (a->U[x * R + r]) iu.push_back((int)x);
        for (int64_t x = 0; x < nv; ++x) if (a->V[x * R + r]) iv.push_back((int)x);
        for (int64_t x = 0; x < nw; ++x) if (a->W[x * R + r]) iw.push_back((int)x);
        for (int xu : iu)
            for (int xv : iv)
                for (int xw : iw)
                    acc[((int64_t)xu * nv + xv) * nw + xw] +=
                        (int64_t)a->U[(int64_t)xu * R + r] * a->V[(int64_t)xv * R + r] * a->W[(int64_t)xw * R + r];
    }
    int64_t bad = 0, ones_seen = 0;
    for (const auto &kv : acc) {
        const int64_t key = kv.first;
        const int64_t xw = key % nw, xv = (key / nw) % nv, xu = key / (nw * nv);
        const int i = (int)(xu / k), j = (int)(xu % k), j2 = (int)(xv / n), l = (int)(xv % n);
        const int i2 = (int)(xw / n), l2 = (int)(xw % n);
        const bool diag = j == j2 && i == i2 && l == l2;
        if (diag) ++ones_seen;
        if (kv.second != (diag ? 1 : 0)) ++bad;
    }
    // diagonal triples that no product touched sum to 0, not 1
    bad += (int64_t)m * k * n - ones_seen;
    return bad;
}

extern "C" fmm_status_t fmm_algo_rect_builtin(const char *name, fmm_algo_rect_t *out) {
    if (!name || !out) return FMM_ERR_INVALID;
    if (std::string(name) == "strassen_2x2x3") {
        const Rect223 &t = rect_223();
        *out = {2, 2, 3, 11, t.U.data(), t.V.data(), t.W.data()};
        return FMM_OK;
    }
    return FMM_ERR_NOT_FOUND;
}

extern "C" fmm_status_t fmm_algo_rect_classic(int m, int k, int n, int32_t *U, int32_t *V, int32_t *W,
                                              fmm_algo_rect_t *out) {
    if (m < 1 || k < 1 || n < 1 || !U || !V || !W || !out) return FMM_ERR_INVALID;
    if ((long long)m * k * n > (1LL << 20)) return FMM_ERR_UNSUPPORTED;
    const int R = m * k * n;
    std::memset(U, 0, sizeof(int32_t) * (size_t)m * k * R);
    std::memset(V, 0, sizeof(int32_t) * (size_t)k * n * R);
    std::memset(W, 0, sizeof(int32_t) * (size_t)m * n * R);
    int r = 0;
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < k; ++j)
            for (int l = 0; l < n; ++l, ++r) {
                U[(int64_t)(i * k + j) * R + r] = 1;
                V[(int64_t)(j * n + l) * R + r] = 1;
                W[(int64_t)(i * n + l) * R + r] = 1;
            }
    *out = {m, k, n, R, U, V, W};
    return FMM_OK;
}

extern "C" fmm_status_t fmm_algo_rect_transpose(const fmm_algo_rect_t *in, int32_t *U, int32_t *V, int32_t *W,
                                                fmm_algo_rect_t *out) {
    if (!rect_ok(in) || !U || !V || !W || !out) return FMM_ERR_INVALID;
    // (A B)^T = B^T A^T: <n,k,m> with A' = B^T, B' = A^T, C' = C^T
    grid_transpose(in->V, in->k, in->n, in->R, U);
    grid_transpose(in->U, in->m, in->k, in->R, V);
    grid_transpose(in->W, in->m, in->n, in->R, W);
    *out = {in->n, in->k, in->m, in->R, U, V, W};
    return FMM_OK;
}

extern "C" fmm_status_t fmm_algo_rect_cyclic(const fmm_algo_rect_t *in, int32_t *U, int32_t *V, int32_t *W,
                                             fmm_algo_rect_t *out) {
    if (!rect_ok(in) || !U || !V || !W || !out) return FMM_ERR_INVALID;
    // the trilinear form sum A_ab B_bd C_ad is invariant under rotating its
    // factors: <k,n,m> with tables (V, W^T, U^T)
    std::memcpy(U, in->V, sizeof(int32_t) * (size_t)in->k * in->n * in->R);
    grid_transpose(in->W, in->m, in->n, in->R, V);
    grid_transpose(in->U, in->m, in->k, in->R, W);
    *out = {in->k, in->n, in->m, in->R, U, V, W};
    return FMM_OK;
}

extern "C" fmm_status_t fmm_algo_rect_compose(const fmm_algo_rect_t *f, const fmm_algo_rect_t *s, int32_t *U,
                                              int32_t *V, int32_t *W, fmm_algo_rect_t *out) {
    if (!rect_ok(f) || !rect_ok(s) || !U || !V || !W || !out) return FMM_ERR_INVALID;
    const int64_t R = (int64_t)f->R * s->R;
    const int64_t m = (int64_t)f->m * s->m, k = (int64_t)f->k * s->k, n = (int64_t)f->n * s->n;
    if (R >= (1LL << 31) || m * k * R >= (1LL << 30) || k * n * R >= (1LL << 30) || m * n * R >= (1LL << 30))
        return FMM_ERR_UNSUPPORTED;
    kron_grid(f->U, f->m, f->k, f->R, s->U, s->m, s->k, s->R, U);
    kron_grid(f->V, f->k, f->n, f->R, s->V, s->k, s->n, s->R, V);
    kron_grid(f->W, f->m, f->n, f->R, s->W, s->m, s->n, s->R, W);
    *out = {(int)m, (int)k, (int)n, (int)R, U, V, W};
    return FMM_OK;
}

extern "C" fmm_status_t fmm_algo_rect_as_square(const fmm_algo_rect_t *in, fmm_algo_t *out) {
    if (!rect_ok(in) || !out) return FMM_ERR_INVALID;
    if (in->m != in->k || in->k != in->n) return FMM_ERR_UNSUPPORTED;
    *out = {in->m, in->R, in->U, in->V, in->W};
    return FMM_OK;
}
