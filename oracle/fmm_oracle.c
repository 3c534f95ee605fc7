/*
 * fmm_oracle.c -- plain, slow CPU oracle for recursive bilinear fast matrix
 * multiplication (D'Alberto, "Strassen's Matrix Multiplication Algorithm Is
 * Still Faster", arXiv 2312.12732).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path may load,
 * link or call this file; only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header, table or helper with the
 * CUDA library: the algorithm (U, V, W) and the matrices arrive as inputs.
 *
 * Conventions (Section 2 of the paper):
 *   - an n x n matrix split by a factor p is the row-major list of its p*p
 *     blocks A_0 .. A_{p*p-1}; block i covers rows (i / p) * m .. and columns
 *     (i % p) * m .. with m = n / p;
 *   - a bilinear algorithm <p,p,p;R> is three integer p^2 x R row-major
 *     matrices U, V, W.  Product r is P_r = S_r * T_r with
 *     S_r = sum_i U[i][r] A_i and T_r = sum_j V[j][r] B_j, and block l of C is
 *     C_l = sum_r W[l][r] P_r (equation `strassen`).  W indexes the blocks of C
 *     in row-major order; the paper's printed c^t lists them as C0, C2, C1, C3,
 *     i.e. it indexes C transposed, and the tests relabel it before use.
 *
 * Precision: IEEE binary64 throughout.  The file is compiled with
 * -ffp-contract=off so that a*b+c is never fused behind the reader's back; the
 * only fused multiply-adds are the explicit fma() calls of TwoProduct.
 *
 * Parity status: every function below is pinned by CPU tests against
 * closed forms, brute force or exact rational arithmetic (no function here is
 * "parity unpinned").
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Brent equations (Section 2, equation `strassen` read entry-wise).          */
/* ------------------------------------------------------------------------- */

/*
 * Counts the index tuples (i, j, j2, k, i2, k2), each in [0, p), for which
 *     sum_r U[(i,j)][r] * V[(j2,k)][r] * W[(i2,k2)][r]
 *         != delta(j, j2) * delta(i, i2) * delta(k, k2).
 * The algorithm computes C = A B for every A, B exactly when the count is 0.
 * Sums are taken in int64, so the check is exact for any coefficients that
 * fit in int32 and any R below 2^31 / max|coefficient|^3.
 */
int64_t fmm_oracle_brent_mismatches_rational(int p, int R, const int32_t *U, const int32_t *V,
                                             const int32_t *W, int32_t den_u, int32_t den_v, int32_t den_w);

int64_t fmm_oracle_brent_mismatches(int p, int R, const int32_t *U, const int32_t *V,
                                    const int32_t *W) {
    return fmm_oracle_brent_mismatches_rational(p, R, U, V, W, 1, 1, 1);
}

/*
 * Brent equations for rational coefficients U / den_u, V / den_v, W / den_w:
 * multiplied through by den_u den_v den_w they read
 *     sum_r U[(i,j)][r] V[(j2,k)][r] W[(i2,k2)][r]
 *         = den_u den_v den_w delta(j, j2) delta(i, i2) delta(k, k2),
 * an identity of integers, counted here in int64 (exact while R times the
 * largest |U V W| and the denominators' product stay below 2^63; the callers'
 * tables are far below).  Returns -1 for a denominator below 1.
 */
int64_t fmm_oracle_brent_mismatches_rational(int p, int R, const int32_t *U, const int32_t *V,
                                             const int32_t *W, int32_t den_u, int32_t den_v, int32_t den_w) {
    if (den_u < 1 || den_v < 1 || den_w < 1) return -1;
    const int64_t one = (int64_t)den_u * den_v * den_w;
    int64_t bad = 0;
    for (int i = 0; i < p; ++i)
        for (int j = 0; j < p; ++j)
            for (int j2 = 0; j2 < p; ++j2)
                for (int k = 0; k < p; ++k)
                    for (int i2 = 0; i2 < p; ++i2)
                        for (int k2 = 0; k2 < p; ++k2) {
                            const int32_t *u = U + (int64_t)(i * p + j) * R;
                            const int32_t *v = V + (int64_t)(j2 * p + k) * R;
                            const int32_t *w = W + (int64_t)(i2 * p + k2) * R;
                            int64_t s = 0;
                            for (int r = 0; r < R; ++r) s += (int64_t)u[r] * v[r] * w[r];
                            int64_t want = (j == j2 && i == i2 && k == k2) ? one : 0;
                            if (s != want) ++bad;
                        }
    return bad;
}

/* ------------------------------------------------------------------------- */
/* Classic product (Section 2, definition of matrix multiplication).          */
/* ------------------------------------------------------------------------- */

/*
 * C[0:M, 0:N] = A[0:M, 0:K] * B[0:K, 0:N]; all row-major with leading
 * dimensions lda, ldb, ldc.  Every C[i][j] starts at 0.0 and accumulates
 * A[i][k] * B[k][j] in ascending k (loop order i, k, j; each product rounded,
 * then added).  Rows are independent, so the OpenMP split over i does not
 * change any result.
 */
void fmm_oracle_classic(int64_t M, int64_t N, int64_t K, const double *A, int64_t lda,
                        const double *B, int64_t ldb, double *C, int64_t ldc) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < M; ++i) {
        double *c = C + i * ldc;
        for (int64_t j = 0; j < N; ++j) c[j] = 0.0;
        for (int64_t k = 0; k < K; ++k) {
            const double a = A[i * lda + k];
            const double *b = B + k * ldb;
            for (int64_t j = 0; j < N; ++j) c[j] += a * b[j];
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Recursive bilinear evaluation (Section 2, equations `strassen` and         */
/* `eq:recursion`; recursion and composition order in the paragraphs on       */
/* split factors).                                                             */
/* ------------------------------------------------------------------------- */

/* Coefficients are U[i][r] / den_u and so on (Section 2: they need not be
 * integers); integer algorithms have every denominator 1. */
typedef struct {
    int p, R;
    const int32_t *U, *V, *W;
    int32_t den_u, den_v, den_w;
} oracle_alg;

/* The coefficient c / den as a binary64 number (exact when den is a power of
 * two and c is small; otherwise the nearest double), and whether it is +1 or
 * -1, where the oracle adds or subtracts instead of multiplying. */
static double coef_value(int32_t c, int32_t den) { return den == 1 ? (double)c : (double)c / (double)den; }

/* dst[0:m,0:m] (ld m) = sum_i (coef[i][r] / den) * src block i, ascending i. */
static void combine_blocks(int64_t m, int p, int R, const int32_t *coef, int32_t den, int r, const double *src,
                           int64_t ld, double *dst) {
    for (int64_t x = 0; x < m * m; ++x) dst[x] = 0.0;
    for (int i = 0; i < p * p; ++i) {
        const int32_t c = coef[(int64_t)i * R + r];
        if (c == 0) continue;
        const double *blk = src + (int64_t)(i / p) * m * ld + (int64_t)(i % p) * m;
        const double cd = coef_value(c, den);
        for (int64_t y = 0; y < m; ++y)
            for (int64_t x = 0; x < m; ++x) {
                const double a = blk[y * ld + x];
                if (cd == 1.0)
                    dst[y * m + x] += a;
                else if (cd == -1.0)
                    dst[y * m + x] -= a;
                else
                    dst[y * m + x] += cd * a;
            }
    }
}

static int bilinear_rec(int64_t n, const double *A, int64_t lda, const double *B, int64_t ldb,
                        double *C, int64_t ldc, const oracle_alg *alg, int depth) {
    const int p = alg->p, R = alg->R;
    if (depth <= 0 || n < p) {
        fmm_oracle_classic(n, n, n, A, lda, B, ldb, C, ldc);
        return 0;
    }
    /* Peeling rule (the paper only uses sizes that factor exactly): with
     * q = n mod p, the leading n' = n - q rows/columns go through the fast
     * algorithm, and the trailing q rows/columns are fixed up classically:
     *   C[:n',:n'] = fast(A[:n',:n'], B[:n',:n']) + A[:n',n':] B[n':,:n']
     *   C[:n',n':] = A[:n',:] B[:,n':]
     *   C[n':,:]   = A[n':,:] B                                           */
    const int64_t q = n % p, nc = n - q, m = nc / p;
    double *S = (double *)malloc(sizeof(double) * m * m);
    double *T = (double *)malloc(sizeof(double) * m * m);
    double *Pr = (double *)malloc(sizeof(double) * m * m);
    if (!S || !T || !Pr) {
        free(S); free(T); free(Pr);
        return -1;
    }
    for (int64_t y = 0; y < nc; ++y)
        for (int64_t x = 0; x < nc; ++x) C[y * ldc + x] = 0.0;
    int rc = 0;
    for (int r = 0; r < R && rc == 0; ++r) {
        /* S_r = sum_i U[i][r] A_i,  T_r = sum_j V[j][r] B_j */
        combine_blocks(m, p, R, alg->U, alg->den_u, r, A, lda, S);
        combine_blocks(m, p, R, alg->V, alg->den_v, r, B, ldb, T);
        /* P_r = S_r T_r, itself by the same algorithm one level down */
        rc = bilinear_rec(m, S, m, T, m, Pr, m, alg, depth - 1);
        /* C_l += W[l][r] P_r for every l (so each C_l sums in ascending r) */
        for (int l = 0; l < p * p && rc == 0; ++l) {
            const int32_t w = alg->W[(int64_t)l * R + r];
            if (w == 0) continue;
            double *cb = C + (int64_t)(l / p) * m * ldc + (int64_t)(l % p) * m;
            const double wd = coef_value(w, alg->den_w);
            for (int64_t y = 0; y < m; ++y)
                for (int64_t x = 0; x < m; ++x) {
                    const double v = Pr[y * m + x];
                    if (wd == 1.0)
                        cb[y * ldc + x] += v;
                    else if (wd == -1.0)
                        cb[y * ldc + x] -= v;
                    else
                        cb[y * ldc + x] += wd * v;
                }
        }
    }
    free(S); free(T); free(Pr);
    if (rc != 0 || q == 0) return rc;

    double *tmp = (double *)malloc(sizeof(double) * nc * nc);
    if (!tmp) return -1;
    fmm_oracle_classic(nc, nc, q, A + nc, lda, B + nc * ldb, ldb, tmp, nc);
    for (int64_t y = 0; y < nc; ++y)
        for (int64_t x = 0; x < nc; ++x) C[y * ldc + x] += tmp[y * nc + x];
    free(tmp);
    fmm_oracle_classic(nc, q, n, A, lda, B + nc, ldb, C + nc, ldc);
    fmm_oracle_classic(q, n, n, A + nc * lda, lda, B, ldb, C + nc * ldc, ldc);
    return 0;
}

/*
 * C = A * B (n x n, row-major, leading dimensions lda, ldb, ldc) by `depth`
 * levels of the bilinear algorithm (p, R, U, V, W), recursing level by level
 * (never flattened), with classic products at the leaves and for the peeled
 * strips.  Returns 0, or -1 if a temporary could not be allocated.
 */
int fmm_oracle_bilinear(int64_t n, const double *A, int64_t lda, const double *B, int64_t ldb,
                        double *C, int64_t ldc, int p, int R, const int32_t *U, const int32_t *V,
                        const int32_t *W, int depth) {
    oracle_alg alg = {p, R, U, V, W, 1, 1, 1};
    return bilinear_rec(n, A, lda, B, ldb, C, ldc, &alg, depth);
}

/*
 * The same recursion for an algorithm with rational coefficients U / den_u,
 * V / den_v, W / den_w (int32 numerators, positive denominators): every
 * coefficient is applied where it stands, as the binary64 value of its
 * fraction.  Returns 0, -1 if a temporary could not be allocated, -2 for a
 * denominator below 1.
 */
int fmm_oracle_bilinear_rational(int64_t n, const double *A, int64_t lda, const double *B, int64_t ldb,
                                 double *C, int64_t ldc, int p, int R, const int32_t *U, const int32_t *V,
                                 const int32_t *W, int32_t den_u, int32_t den_v, int32_t den_w, int depth) {
    if (den_u < 1 || den_v < 1 || den_w < 1) return -2;
    oracle_alg alg = {p, R, U, V, W, den_u, den_v, den_w};
    return bilinear_rec(n, A, lda, B, ldb, C, ldc, &alg, depth);
}

/* ------------------------------------------------------------------------- */
/* Rectangular algorithms <pm,pk,pn;R> (Section 2 and its discussion of split  */
/* factors: a square problem of factor 6 or 12 can be solved by composing     */
/* non-square basic products, 2x3x3 with 3x2x3 and so on).  A is split into a */
/* pm x pk grid of blocks, B into pk x pn, C into pm x pn, all indexed         */
/* row-major; U is (pm pk) x R, V is (pk pn) x R, W is (pm pn) x R.            */
/* ------------------------------------------------------------------------- */

/*
 * Counts the index tuples (i, j, j2, k, i2, k2) with i, i2 < pm, j, j2 < pk,
 * k, k2 < pn for which sum_r U[(i,j)][r] V[(j2,k)][r] W[(i2,k2)][r] differs
 * from delta(j, j2) delta(i, i2) delta(k, k2); exact in int64.
 */
int64_t fmm_oracle_rect_brent_mismatches(int pm, int pk, int pn, int R, const int32_t *U, const int32_t *V,
                                         const int32_t *W) {
    int64_t bad = 0;
    for (int i = 0; i < pm; ++i)
        for (int j = 0; j < pk; ++j)
            for (int j2 = 0; j2 < pk; ++j2)
                for (int k = 0; k < pn; ++k)
                    for (int i2 = 0; i2 < pm; ++i2)
                        for (int k2 = 0; k2 < pn; ++k2) {
                            const int32_t *u = U + (int64_t)(i * pk + j) * R;
                            const int32_t *v = V + (int64_t)(j2 * pn + k) * R;
                            const int32_t *w = W + (int64_t)(i2 * pn + k2) * R;
                            int64_t sum = 0;
                            for (int r = 0; r < R; ++r) sum += (int64_t)u[r] * v[r] * w[r];
                            const int64_t want = (j == j2 && i == i2 && k == k2) ? 1 : 0;
                            if (sum != want) ++bad;
                        }
    return bad;
}

typedef struct {
    int pm, pk, pn, R;
    const int32_t *U, *V, *W;
} oracle_rect_alg;

/* dst[0:rows,0:cols] (ld cols) = sum_i coef[i][r] * block i of src, ascending i;
 * src is split into a gr x gc grid of rows x cols blocks. */
static void combine_rect(int64_t rows, int64_t cols, int gr, int gc, int R, const int32_t *coef, int r,
                         const double *src, int64_t ld, double *dst) {
    for (int64_t x = 0; x < rows * cols; ++x) dst[x] = 0.0;
    for (int i = 0; i < gr * gc; ++i) {
        const int32_t c = coef[(int64_t)i * R + r];
        if (c == 0) continue;
        const double *blk = src + (int64_t)(i / gc) * rows * ld + (int64_t)(i % gc) * cols;
        const double cd = (double)c;
        for (int64_t y = 0; y < rows; ++y)
            for (int64_t x = 0; x < cols; ++x) {
                const double a = blk[y * ld + x];
                if (c == 1)
                    dst[y * cols + x] += a;
                else if (c == -1)
                    dst[y * cols + x] -= a;
                else
                    dst[y * cols + x] += cd * a;
            }
    }
}

/*
 * C (M x N, ld ldc) = A (M x K) B (K x N) with level l of the recursion using
 * algorithm levels[l] (l = 0 outermost); classic products below the last level
 * or when a dimension is smaller than its split factor.  Peeling per
 * dimension, as in the square recursion: with M', K', N' the largest
 * multiples of pm, pk, pn,
 *   C[:M',:N'] = fast(A[:M',:K'], B[:K',:N']) + A[:M',K':] B[K':,:N'],
 *   C[:M',N':] = A[:M',:] B[:,N':],   C[M':,:] = A[M':,:] B.
 */
static int rect_rec(int64_t M, int64_t K, int64_t N, const double *A, int64_t lda, const double *B, int64_t ldb,
                    double *C, int64_t ldc, const oracle_rect_alg *levels, int nlevels) {
    if (nlevels <= 0 || M < levels[0].pm || K < levels[0].pk || N < levels[0].pn) {
        fmm_oracle_classic(M, N, K, A, lda, B, ldb, C, ldc);
        return 0;
    }
    const oracle_rect_alg *alg = &levels[0];
    const int64_t Mc = M - M % alg->pm, Kc = K - K % alg->pk, Nc = N - N % alg->pn;
    const int64_t bm = Mc / alg->pm, bk = Kc / alg->pk, bn = Nc / alg->pn;
    double *S = (double *)malloc(sizeof(double) * bm * bk);
    double *T = (double *)malloc(sizeof(double) * bk * bn);
    double *Pr = (double *)malloc(sizeof(double) * bm * bn);
    if (!S || !T || !Pr) {
        free(S); free(T); free(Pr);
        return -1;
    }
    for (int64_t y = 0; y < Mc; ++y)
        for (int64_t x = 0; x < Nc; ++x) C[y * ldc + x] = 0.0;
    int rc = 0;
    for (int r = 0; r < alg->R && rc == 0; ++r) {
        combine_rect(bm, bk, alg->pm, alg->pk, alg->R, alg->U, r, A, lda, S);
        combine_rect(bk, bn, alg->pk, alg->pn, alg->R, alg->V, r, B, ldb, T);
        rc = rect_rec(bm, bk, bn, S, bk, T, bn, Pr, bn, levels + 1, nlevels - 1);
        for (int l = 0; l < alg->pm * alg->pn && rc == 0; ++l) {
            const int32_t w = alg->W[(int64_t)l * alg->R + r];
            if (w == 0) continue;
            double *cb = C + (int64_t)(l / alg->pn) * bm * ldc + (int64_t)(l % alg->pn) * bn;
            const double wd = (double)w;
            for (int64_t y = 0; y < bm; ++y)
                for (int64_t x = 0; x < bn; ++x) {
                    const double v = Pr[y * bn + x];
                    if (w == 1)
                        cb[y * ldc + x] += v;
                    else if (w == -1)
                        cb[y * ldc + x] -= v;
                    else
                        cb[y * ldc + x] += wd * v;
                }
        }
    }
    free(S); free(T); free(Pr);
    if (rc != 0) return rc;
    if (K > Kc && Mc > 0 && Nc > 0) {
        double *tmp = (double *)malloc(sizeof(double) * Mc * Nc);
        if (!tmp) return -1;
        fmm_oracle_classic(Mc, Nc, K - Kc, A + Kc, lda, B + Kc * ldb, ldb, tmp, Nc);
        for (int64_t y = 0; y < Mc; ++y)
            for (int64_t x = 0; x < Nc; ++x) C[y * ldc + x] += tmp[y * Nc + x];
        free(tmp);
    }
    if (N > Nc) fmm_oracle_classic(Mc, N - Nc, K, A, lda, B + Nc, ldb, C + Nc, ldc);
    if (M > Mc) fmm_oracle_classic(M - Mc, N, K, A + Mc * lda, lda, B, ldb, C + Mc * ldc, ldc);
    return 0;
}

/* The recursion above; tables[l] = {pm, pk, pn, R} of level l, U/V/W[l] its tables. */
int fmm_oracle_rect_bilinear(int64_t M, int64_t K, int64_t N, const double *A, int64_t lda, const double *B,
                             int64_t ldb, double *C, int64_t ldc, int nlevels, const int32_t *dims,
                             const int32_t *const *U, const int32_t *const *V, const int32_t *const *W) {
    oracle_rect_alg lv[16];
    if (nlevels < 0 || nlevels > 16) return -2;
    for (int l = 0; l < nlevels; ++l) {
        lv[l].pm = dims[4 * l]; lv[l].pk = dims[4 * l + 1]; lv[l].pn = dims[4 * l + 2]; lv[l].R = dims[4 * l + 3];
        lv[l].U = U[l]; lv[l].V = V[l]; lv[l].W = W[l];
        if (lv[l].pm < 1 || lv[l].pk < 1 || lv[l].pn < 1 || lv[l].R < 1) return -2;
    }
    return rect_rec(M, K, N, A, lda, B, ldb, C, ldc, lv, nlevels);
}

/* ------------------------------------------------------------------------- */
/* Double complex (Section 1 lists single and double complex among the types  */
/* the algorithms deploy to).  A complex matrix is stored interleaved: entry  */
/* (i, j) is re at 2 (i ld + j), im right after it, ld counted in complex      */
/* entries.  The bilinear algorithm's coefficients are real, so its pre- and   */
/* post-additions act on the real and imaginary parts alike; only the leaf     */
/* products multiply complex numbers.                                          */
/* ------------------------------------------------------------------------- */

/*
 * C = A B for complex M x K and K x N matrices.  Every C[i][j] starts at 0 and
 * accumulates A[i][k] B[k][j] in ascending k, each product formed as
 * (ac - bd) + (ad + bc) i with every product and difference rounded, then the
 * two parts added to the running sums.
 */
void fmm_oracle_classic_complex(int64_t M, int64_t N, int64_t K, const double *A, int64_t lda, const double *B,
                                int64_t ldb, double *C, int64_t ldc) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < M; ++i) {
        double *c = C + 2 * i * ldc;
        for (int64_t j = 0; j < 2 * N; ++j) c[j] = 0.0;
        for (int64_t k = 0; k < K; ++k) {
            const double ar = A[2 * (i * lda + k)], ai = A[2 * (i * lda + k) + 1];
            const double *b = B + 2 * k * ldb;
            for (int64_t j = 0; j < N; ++j) {
                const double br = b[2 * j], bi = b[2 * j + 1];
                const double x = ar * br, y = ai * bi, u = ar * bi, v = ai * br;
                c[2 * j] += x - y;
                c[2 * j + 1] += u + v;
            }
        }
    }
}

/* dst (m x m complex, ld m) = sum_i coef[i][r] * complex block i of src, ascending i. */
static void combine_blocks_complex(int64_t m, int p, int R, const int32_t *coef, int r, const double *src,
                                   int64_t ld, double *dst) {
    for (int64_t x = 0; x < 2 * m * m; ++x) dst[x] = 0.0;
    for (int i = 0; i < p * p; ++i) {
        const int32_t c = coef[(int64_t)i * R + r];
        if (c == 0) continue;
        const double *blk = src + 2 * ((int64_t)(i / p) * m * ld + (int64_t)(i % p) * m);
        const double cd = (double)c;
        for (int64_t y = 0; y < m; ++y)
            for (int64_t x = 0; x < 2 * m; ++x) {
                const double a = blk[2 * y * ld + x];
                if (c == 1)
                    dst[2 * y * m + x] += a;
                else if (c == -1)
                    dst[2 * y * m + x] -= a;
                else
                    dst[2 * y * m + x] += cd * a;
            }
    }
}

static int bilinear_rec_complex(int64_t n, const double *A, int64_t lda, const double *B, int64_t ldb, double *C,
                                int64_t ldc, const oracle_alg *alg, int depth) {
    const int p = alg->p, R = alg->R;
    if (depth <= 0 || n < p) {
        fmm_oracle_classic_complex(n, n, n, A, lda, B, ldb, C, ldc);
        return 0;
    }
    /* the peeling rule of the real recursion, on complex entries */
    const int64_t q = n % p, nc = n - q, m = nc / p;
    double *S = (double *)malloc(sizeof(double) * 2 * m * m);
    double *T = (double *)malloc(sizeof(double) * 2 * m * m);
    double *Pr = (double *)malloc(sizeof(double) * 2 * m * m);
    if (!S || !T || !Pr) {
        free(S); free(T); free(Pr);
        return -1;
    }
    for (int64_t y = 0; y < nc; ++y)
        for (int64_t x = 0; x < 2 * nc; ++x) C[2 * y * ldc + x] = 0.0;
    int rc = 0;
    for (int r = 0; r < R && rc == 0; ++r) {
        combine_blocks_complex(m, p, R, alg->U, r, A, lda, S);
        combine_blocks_complex(m, p, R, alg->V, r, B, ldb, T);
        rc = bilinear_rec_complex(m, S, m, T, m, Pr, m, alg, depth - 1);
        for (int l = 0; l < p * p && rc == 0; ++l) {
            const int32_t w = alg->W[(int64_t)l * R + r];
            if (w == 0) continue;
            double *cb = C + 2 * ((int64_t)(l / p) * m * ldc + (int64_t)(l % p) * m);
            const double wd = (double)w;
            for (int64_t y = 0; y < m; ++y)
                for (int64_t x = 0; x < 2 * m; ++x) {
                    const double v = Pr[2 * y * m + x];
                    if (w == 1)
                        cb[2 * y * ldc + x] += v;
                    else if (w == -1)
                        cb[2 * y * ldc + x] -= v;
                    else
                        cb[2 * y * ldc + x] += wd * v;
                }
        }
    }
    free(S); free(T); free(Pr);
    if (rc != 0 || q == 0) return rc;

    double *tmp = (double *)malloc(sizeof(double) * 2 * nc * nc);
    if (!tmp) return -1;
    fmm_oracle_classic_complex(nc, nc, q, A + 2 * nc, lda, B + 2 * nc * ldb, ldb, tmp, nc);
    for (int64_t y = 0; y < nc; ++y)
        for (int64_t x = 0; x < 2 * nc; ++x) C[2 * y * ldc + x] += tmp[2 * y * nc + x];
    free(tmp);
    fmm_oracle_classic_complex(nc, q, n, A, lda, B + 2 * nc, ldb, C + 2 * nc, ldc);
    fmm_oracle_classic_complex(q, n, n, A + 2 * nc * lda, lda, B, ldb, C + 2 * nc * ldc, ldc);
    return 0;
}

/* C = A B for complex n x n matrices by `depth` recursive levels of the (integer) algorithm. */
int fmm_oracle_bilinear_complex(int64_t n, const double *A, int64_t lda, const double *B, int64_t ldb, double *C,
                                int64_t ldc, int p, int R, const int32_t *U, const int32_t *V, const int32_t *W,
                                int depth) {
    oracle_alg alg = {p, R, U, V, W, 1, 1, 1};
    return bilinear_rec_complex(n, A, lda, B, ldb, C, ldc, &alg, depth);
}

/* ------------------------------------------------------------------------- */
/* Scaled update (Section 3 states the product as C = alpha A B; beta C is    */
/* the usual BLAS extension of that statement).                               */
/* ------------------------------------------------------------------------- */

/*
 * C[t] = alpha * P[t] + beta * C[t] for t < count, each product rounded, then
 * added.  beta == 0 leaves C unread and alpha == 0 leaves P unread (P may then
 * be NULL), so NaN or infinity there does not reach the result.
 */
void fmm_oracle_axpby(int64_t count, double alpha, const double *P, double beta, double *C) {
    for (int64_t t = 0; t < count; ++t) {
        double x = 0.0;
        if (alpha != 0.0) x = alpha * P[t];
        if (beta != 0.0) {
            double y = beta * C[t];
            x = x + y;
        }
        C[t] = x;
    }
}

/* ------------------------------------------------------------------------- */
/* Compensated dot products for sampled reference entries.                    */
/* Ogita, Rump, Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput.    */
/* 26(6), 2005: TwoSum (Knuth), TwoProduct via FMA, and Dot2 (their Alg. 5.3). */
/* The result is as accurate as if computed in twice the working precision and */
/* then rounded.                                                               */
/* ------------------------------------------------------------------------- */

static inline void two_sum(double a, double b, double *s, double *e) {
    double x = a + b;
    double z = x - a;
    *s = x;
    *e = (a - (x - z)) + (b - z);
}

static inline void two_product(double a, double b, double *p, double *e) {
    double x = a * b;
    *p = x;
    *e = fma(a, b, -x);
}

double fmm_oracle_dot2(int64_t K, const double *x, int64_t incx, const double *y, int64_t incy) {
    if (K <= 0) return 0.0;
    double p, s;
    two_product(x[0], y[0], &p, &s);
    for (int64_t k = 1; k < K; ++k) {
        double h, r, q;
        two_product(x[k * incx], y[k * incy], &h, &r);
        two_sum(p, h, &p, &q);
        s = s + (q + r);
    }
    return p + s;
}

/*
 * out[t] = Dot2(row rows[t] of A, column cols[t] of B) for t < count, where
 * A is M x K (ld lda) and B is K x N (ld ldb).  Indices are not checked.
 */
void fmm_oracle_sample_dot2(int64_t K, const double *A, int64_t lda, const double *B, int64_t ldb,
                            int64_t count, const int64_t *rows, const int64_t *cols, double *out) {
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < count; ++t)
        out[t] = fmm_oracle_dot2(K, A + rows[t] * lda, 1, B + cols[t], ldb);
}

/* ------------------------------------------------------------------------- */
/* Thread count of the OpenMP loops above (timing only; results do not depend */
/* on it: every parallel loop writes disjoint outputs in a fixed order).      */
/* ------------------------------------------------------------------------- */
#ifdef _OPENMP
#include <omp.h>
#endif

void fmm_oracle_set_num_threads(int threads) {
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#else
    (void)threads;
#endif
}
