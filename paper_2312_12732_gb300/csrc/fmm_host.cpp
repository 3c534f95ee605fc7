// Host side of the fast-matrix-multiplication library: built-in algorithms,
// exact Brent check, recursion flattening, tile-task planning, workspace and
// launches.  Public entry points are declared in include/fmm.h.
#include "fmm.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include <sys/mman.h>
#include <unistd.h>

#include "fmm_internal.h"

#include <cudaTypedefs.h>

using fmm::F64Geom;
using fmm::F64Launch;
using fmm::F64Problem;

// ---------------------------------------------------------------------------
// Built-in algorithms.  Each table is p^2 x R row-major over blocks; W indexes
// the blocks of C in row-major order.
// ---------------------------------------------------------------------------
namespace {

// <2,2,2;8>: the classic block product (Section 3, the printed graph
// C0 = A0 B0 + A1 B2, C1 = A0 B1 + A1 B3, C2 = A2 B0 + A3 B2, C3 = A2 B1 + A3 B3).
const int32_t kClassic2U[4 * 8] = {1, 0, 1, 0, 0, 0, 0, 0,  0, 1, 0, 1, 0, 0, 0, 0,
                                   0, 0, 0, 0, 1, 0, 1, 0,  0, 0, 0, 0, 0, 1, 0, 1};
const int32_t kClassic2V[4 * 8] = {1, 0, 0, 0, 1, 0, 0, 0,  0, 0, 1, 0, 0, 0, 1, 0,
                                   0, 1, 0, 0, 0, 1, 0, 0,  0, 0, 0, 1, 0, 0, 0, 1};
const int32_t kClassic2W[4 * 8] = {1, 1, 0, 0, 0, 0, 0, 0,  0, 0, 1, 1, 0, 0, 0, 0,
                                   0, 0, 0, 0, 1, 1, 0, 0,  0, 0, 0, 0, 0, 0, 1, 1};

// Strassen as printed in Section 2 (a, b and c^t of f['2,2,2']); the c^t rows
// are printed with labels C0, C2, C1, C3 and are stored here under those labels.
const int32_t kStrassenU[4 * 7] = {0, 1, 1, 0, 1, 1, 0,   0, 0, -1, 1, 0, 0, 0,
                                   1, 1, 1, 0, 1, 0, 0,   -1, -1, -1, 0, 0, 0, 1};
const int32_t kStrassenV[4 * 7] = {0, 0, 0, 0, 1, 1, 0,   1, 1, 0, 0, 1, 0, 1,
                                   0, 1, 1, 1, 1, 0, 0,   0, 1, 1, 0, 1, 0, 1};
const int32_t kStrassenW[4 * 7] = {0, 0, 0, 1, 0, 1, 0,   -1, 1, -1, -1, 0, 0, 0,
                                   0, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 0, 1};

// Strassen 1969: M1 = (A11+A22)(B11+B22), M2 = (A21+A22)B11, M3 = A11(B12-B22),
// M4 = A22(B21-B11), M5 = (A11+A12)B22, M6 = (A21-A11)(B11+B12),
// M7 = (A12-A22)(B21+B22); C11 = M1+M4-M5+M7, C12 = M3+M5, C21 = M2+M4,
// C22 = M1-M2+M3+M6.
const int32_t kS69U[4 * 7] = {1, 0, 1, 0, 1, -1, 0,  0, 0, 0, 0, 1, 0, 1,
                              0, 1, 0, 0, 0, 1, 0,   1, 1, 0, 1, 0, 0, -1};
const int32_t kS69V[4 * 7] = {1, 1, 0, -1, 0, 1, 0,  0, 0, 1, 0, 0, 1, 0,
                              0, 0, 0, 1, 0, 0, 1,   1, 0, -1, 0, 1, 0, 1};
const int32_t kS69W[4 * 7] = {1, 0, 0, 1, -1, 0, 1,  0, 0, 1, 0, 1, 0, 0,
                              0, 1, 0, 1, 0, 0, 0,   1, -1, 1, 0, 0, 1, 0};

// Strassen-Winograd (15-addition variant) in flat form:
// M1 = A11 B11, M2 = A12 B21, M3 = (A11+A12-A21-A22) B22,
// M4 = A22 (B11-B12-B21+B22), M5 = (A21+A22)(B12-B11),
// M6 = (A21+A22-A11)(B11-B12+B22), M7 = (A11-A21)(B22-B12);
// C11 = M1+M2, C12 = M1+M3+M5+M6, C21 = M1-M4+M6+M7, C22 = M1+M5+M6+M7.
const int32_t kWinoU[4 * 7] = {1, 0, 1, 0, 0, -1, 1,  0, 1, 1, 0, 0, 0, 0,
                               0, 0, -1, 0, 1, 1, -1, 0, 0, -1, 1, 1, 1, 0};
const int32_t kWinoV[4 * 7] = {1, 0, 0, 1, -1, 1, 0,  0, 0, 0, -1, 1, -1, -1,
                               0, 1, 0, -1, 0, 0, 0,  0, 0, 1, 1, 0, 1, 1};
const int32_t kWinoW[4 * 7] = {1, 1, 0, 0, 0, 0, 0,  1, 0, 1, 0, 1, 1, 0,
                               1, 0, 0, -1, 0, 1, 1, 1, 0, 0, 0, 1, 1, 1};

// Laderman <3,3,3;23> (1976), products m1..m23 as columns; built from its
// product list at first use.
struct LinTerm { int sign, i, j; };
struct LadermanProduct { LinTerm a[7]; int na; LinTerm b[7]; int nb; };

std::vector<int32_t> g_lad_u, g_lad_v, g_lad_w;

void build_laderman() {
    if (!g_lad_u.empty()) return;
    // Each product: signed a-terms (1-based row, col), signed b-terms.
    static const LadermanProduct prods[23] = {
        {{{1,1,1},{1,1,2},{1,1,3},{-1,2,1},{-1,2,2},{-1,3,2},{-1,3,3}}, 7, {{1,2,2}}, 1},
        {{{1,1,1},{-1,2,1}}, 2, {{-1,1,2},{1,2,2}}, 2},
        {{{1,2,2}}, 1, {{-1,1,1},{1,1,2},{1,2,1},{-1,2,2},{-1,2,3},{-1,3,1},{1,3,3}}, 7},
        {{{-1,1,1},{1,2,1},{1,2,2}}, 3, {{1,1,1},{-1,1,2},{1,2,2}}, 3},
        {{{1,2,1},{1,2,2}}, 2, {{-1,1,1},{1,1,2}}, 2},
        {{{1,1,1}}, 1, {{1,1,1}}, 1},
        {{{-1,1,1},{1,3,1},{1,3,2}}, 3, {{1,1,1},{-1,1,3},{1,2,3}}, 3},
        {{{-1,1,1},{1,3,1}}, 2, {{1,1,3},{-1,2,3}}, 2},
        {{{1,3,1},{1,3,2}}, 2, {{-1,1,1},{1,1,3}}, 2},
        {{{1,1,1},{1,1,2},{1,1,3},{-1,2,2},{-1,2,3},{-1,3,1},{-1,3,2}}, 7, {{1,2,3}}, 1},
        {{{1,3,2}}, 1, {{-1,1,1},{1,1,3},{1,2,1},{-1,2,2},{-1,2,3},{-1,3,1},{1,3,2}}, 7},
        {{{-1,1,3},{1,3,2},{1,3,3}}, 3, {{1,2,2},{1,3,1},{-1,3,2}}, 3},
        {{{1,1,3},{-1,3,3}}, 2, {{1,2,2},{-1,3,2}}, 2},
        {{{1,1,3}}, 1, {{1,3,1}}, 1},
        {{{1,3,2},{1,3,3}}, 2, {{-1,3,1},{1,3,2}}, 2},
        {{{-1,1,3},{1,2,2},{1,2,3}}, 3, {{1,2,3},{1,3,1},{-1,3,3}}, 3},
        {{{1,1,3},{-1,2,3}}, 2, {{1,2,3},{-1,3,3}}, 2},
        {{{1,2,2},{1,2,3}}, 2, {{-1,3,1},{1,3,3}}, 2},
        {{{1,1,2}}, 1, {{1,2,1}}, 1},
        {{{1,2,3}}, 1, {{1,3,2}}, 1},
        {{{1,2,1}}, 1, {{1,1,3}}, 1},
        {{{1,3,1}}, 1, {{1,1,2}}, 1},
        {{{1,3,3}}, 1, {{1,3,3}}, 1},
    };
    // c_ij as lists of 1-based product numbers, all with coefficient +1.
    static const int cl[9][8] = {
        {6, 14, 19},          {1, 4, 5, 6, 12, 14, 15}, {6, 7, 9, 10, 14, 16, 18},
        {2, 3, 4, 6, 14, 16, 17}, {2, 4, 5, 6, 20},    {14, 16, 17, 18, 21},
        {6, 7, 8, 11, 12, 13, 14}, {12, 13, 14, 15, 22}, {6, 7, 8, 9, 23}};
    const int R = 23;
    g_lad_u.assign(9 * R, 0);
    g_lad_v.assign(9 * R, 0);
    g_lad_w.assign(9 * R, 0);
    for (int r = 0; r < R; ++r) {
        for (int e = 0; e < prods[r].na; ++e) {
            const LinTerm &t = prods[r].a[e];
            g_lad_u[((t.i - 1) * 3 + (t.j - 1)) * R + r] += t.sign;
        }
        for (int e = 0; e < prods[r].nb; ++e) {
            const LinTerm &t = prods[r].b[e];
            g_lad_v[((t.i - 1) * 3 + (t.j - 1)) * R + r] += t.sign;
        }
    }
    for (int l = 0; l < 9; ++l)
        for (int e = 0; e < 8 && cl[l][e] != 0; ++e) g_lad_w[l * R + (cl[l][e] - 1)] += 1;
}

}  // namespace

extern "C" const char *fmm_status_string(fmm_status_t s) {
    switch (s) {
        case FMM_OK: return "ok";
        case FMM_ERR_INVALID: return "invalid argument";
        case FMM_ERR_BRENT: return "algorithm fails the Brent equations";
        case FMM_ERR_UNSUPPORTED: return "unsupported request";
        case FMM_ERR_OOM: return "out of memory";
        case FMM_ERR_CUDA: return "CUDA error";
        case FMM_ERR_TIMEOUT: return "device-side wait timed out";
        case FMM_ERR_NOT_FOUND: return "unknown algorithm name";
        case FMM_ERR_SCRATCH_LIMIT: return "request exceeds the static scratch of fmm_gemm_noalloc";
    }
    return "unknown status";
}

extern "C" fmm_status_t fmm_shard_range(int64_t units, int shard_count, int shard_index, int64_t *begin,
                                        int64_t *end) {
    if (units < 0 || shard_count < 1 || shard_index < 0 || shard_index >= shard_count || !begin || !end)
        return FMM_ERR_INVALID;
    // floor(k units / count) without overflow for any units below 2^62 and count below 2^31
    const auto start = [&](int k) {
        const int64_t q = units / shard_count, r = units % shard_count;
        return q * k + (r * k) / shard_count;
    };
    *begin = start(shard_index);
    *end = start(shard_index + 1);
    return FMM_OK;
}

extern "C" fmm_status_t fmm_algo_builtin(const char *name, fmm_algo_t *out) {
    if (!name || !out) return FMM_ERR_INVALID;
    const std::string s(name);
    if (s == "classic2") { *out = {2, 8, kClassic2U, kClassic2V, kClassic2W}; return FMM_OK; }
    if (s == "strassen") { *out = {2, 7, kStrassenU, kStrassenV, kStrassenW}; return FMM_OK; }
    if (s == "strassen1969") { *out = {2, 7, kS69U, kS69V, kS69W}; return FMM_OK; }
    if (s == "winograd") { *out = {2, 7, kWinoU, kWinoV, kWinoW}; return FMM_OK; }
    if (s == "laderman") {
        build_laderman();
        *out = {3, 23, g_lad_u.data(), g_lad_v.data(), g_lad_w.data()};
        return FMM_OK;
    }
    return FMM_ERR_NOT_FOUND;
}

static bool algo_shape_ok(const fmm_algo_t *a) {
    return a && a->p >= 2 && a->R >= 1 && a->U && a->V && a->W && (long long)a->p * a->p * a->R < (1LL << 28);
}

// Brent equations with right-hand side `one` on the diagonal (1 for integer
// coefficients, the denominators' product for a rational algorithm's numerators).
static int64_t brent_count(const fmm_algo_t *a, int64_t one) {
    const int p = a->p, R = a->R;
    int64_t bad = 0;
    // For each (i,j) of A, (j2,k) of B, (i2,k2) of C: sum_r U V W must equal
    // delta(j,j2) delta(i,i2) delta(k,k2).  Loop over the nonzeros of U and V
    // per product to keep the check fast for large compositions.
    std::vector<int64_t> acc((size_t)p * p * p * p * p * p, 0);
    std::vector<int> unz, vnz, wnz;
    for (int r = 0; r < R; ++r) {
        unz.clear(); vnz.clear(); wnz.clear();
        for (int x = 0; x < p * p; ++x) {
            if (a->U[(int64_t)x * R + r]) unz.push_back(x);
            if (a->V[(int64_t)x * R + r]) vnz.push_back(x);
            if (a->W[(int64_t)x * R + r]) wnz.push_back(x);
        }
        for (int iu : unz)
            for (int iv : vnz)
                for (int iw : wnz) {
                    const int64_t c = (int64_t)a->U[(int64_t)iu * R + r] * a->V[(int64_t)iv * R + r] *
                                      a->W[(int64_t)iw * R + r];
                    acc[((size_t)iu * p * p + iv) * p * p + iw] += c;
                }
    }
    for (int i = 0; i < p; ++i)
        for (int j = 0; j < p; ++j)
            for (int j2 = 0; j2 < p; ++j2)
                for (int k = 0; k < p; ++k)
                    for (int i2 = 0; i2 < p; ++i2)
                        for (int k2 = 0; k2 < p; ++k2) {
                            const int64_t want = (j == j2 && i == i2 && k == k2) ? one : 0;
                            const size_t idx = ((size_t)(i * p + j) * p * p + (j2 * p + k)) * p * p + (i2 * p + k2);
                            if (acc[idx] != want) ++bad;
                        }
    return bad;
}

extern "C" int64_t fmm_algo_brent_mismatches(const fmm_algo_t *a) {
    if (!algo_shape_ok(a)) return -1;
    return brent_count(a, 1);
}

extern "C" int64_t fmm_algo_rational_brent_mismatches(const fmm_algo_rational_t *a) {
    if (!a) return -1;
    const fmm_algo_t num{a->p, a->R, a->U, a->V, a->W};
    if (!algo_shape_ok(&num) || a->den_u < 1 || a->den_v < 1 || a->den_w < 1) return -1;
    // every partial sum stays below 2^62 in magnitude: R * max|U| max|V| max|W| < 2^62
    const size_t cnt = (size_t)a->p * a->p * a->R;
    double mu = 0, mv = 0, mw = 0;
    for (size_t x = 0; x < cnt; ++x) {
        mu = std::max(mu, std::fabs((double)a->U[x]));
        mv = std::max(mv, std::fabs((double)a->V[x]));
        mw = std::max(mw, std::fabs((double)a->W[x]));
    }
    const double lim = 4611686018427387904.0;  // 2^62
    if ((double)a->R * mu * mv * mw >= lim) return -1;
    if ((double)a->den_u * a->den_v * a->den_w >= lim) return -1;
    return brent_count(&num, (int64_t)a->den_u * a->den_v * a->den_w);
}

extern "C" fmm_status_t fmm_algo_from_transposed_c(int p, int R, const int32_t *ct, int32_t *W_out) {
    if (p < 2 || R < 1 || !ct || !W_out) return FMM_ERR_INVALID;
    for (int i = 0; i < p; ++i)
        for (int k = 0; k < p; ++k)
            for (int r = 0; r < R; ++r) W_out[(int64_t)(i * p + k) * R + r] = ct[(int64_t)(k * p + i) * R + r];
    return FMM_OK;
}

extern "C" fmm_status_t fmm_algo_compose(const fmm_algo_t *f, const fmm_algo_t *s, int32_t *U_out,
                                         int32_t *V_out, int32_t *W_out, fmm_algo_t *out) {
    if (!algo_shape_ok(f) || !algo_shape_ok(s) || !U_out || !V_out || !W_out || !out) return FMM_ERR_INVALID;
    const int p1 = f->p, p2 = s->p, R1 = f->R, R2 = s->R, p = p1 * p2;
    const int64_t R = (int64_t)R1 * R2;
    if ((int64_t)p * p * R >= (1LL << 30)) return FMM_ERR_UNSUPPORTED;
    const int32_t *X1[3] = {f->U, f->V, f->W};
    const int32_t *X2[3] = {s->U, s->V, s->W};
    int32_t *XO[3] = {U_out, V_out, W_out};
    for (int w = 0; w < 3; ++w)
        for (int i1 = 0; i1 < p1; ++i1)
            for (int j1 = 0; j1 < p1; ++j1)
                for (int i2 = 0; i2 < p2; ++i2)
                    for (int j2 = 0; j2 < p2; ++j2) {
                        const int64_t row = (int64_t)(i1 * p2 + i2) * p + (j1 * p2 + j2);
                        for (int r1 = 0; r1 < R1; ++r1)
                            for (int r2 = 0; r2 < R2; ++r2)
                                XO[w][row * R + (int64_t)r1 * R2 + r2] =
                                    X1[w][(int64_t)(i1 * p1 + j1) * R1 + r1] * X2[w][(int64_t)(i2 * p2 + j2) * R2 + r2];
                    }
    *out = {p, (int)R, U_out, V_out, W_out};
    return FMM_OK;
}

// ---------------------------------------------------------------------------
// Plans
// ---------------------------------------------------------------------------
namespace {

struct Entry { int blk; int coef; };

// Columns of the flattened coefficient matrix of `levels` recursion levels:
// product (r_0, ..., r_{L-1}) (r_0 outermost) = sum r_l R^(L-1-l); block
// (row, col) on the p^L grid with row = sum i_l p^(L-1-l), col likewise;
// coefficient = prod X[(i_l, j_l)][r_l].
std::vector<std::vector<Entry>> flatten(int p, int R, const int32_t *X, int levels) {
    std::vector<std::vector<Entry>> cols(1, std::vector<Entry>{{0, 1}});
    int P = 1;
    for (int lev = 0; lev < levels; ++lev) {
        std::vector<std::vector<Entry>> next((size_t)cols.size() * R);
        const int Pn = P * p;
        for (size_t c = 0; c < cols.size(); ++c)
            for (int r = 0; r < R; ++r) {
                auto &dst = next[c * R + r];
                for (const Entry &e : cols[c]) {
                    const int row = e.blk / P, col = e.blk % P;
                    for (int x = 0; x < p * p; ++x) {
                        const int32_t v = X[(int64_t)x * R + r];
                        if (!v) continue;
                        const int i = x / p, j = x % p;
                        dst.push_back({(row * p + i) * Pn + (col * p + j), e.coef * v});
                    }
                }
                std::sort(dst.begin(), dst.end(), [](const Entry &a, const Entry &b) { return a.blk < b.blk; });
            }
        cols.swap(next);
        P = Pn;
    }
    return cols;
}

long long ipow(long long b, int e) {
    long long r = 1;
    while (e-- > 0) r *= b;
    return r;
}

}  // namespace

struct fmm_plan {
    int device = 0;
    int64_t n = 0;
    int p = 0, R = 0, depth = 0, mat_levels = 0;
    fmm_dtype_t dtype = FMM_F64;
    int64_t P = 1, P_src = 1, R_total = 1, R_src = 1, nsub = 1, m = 0, n_core = 0, b_src = 0;
    int tiles_m = 0, tiles_n = 0;
    int bn = fmm::kBN;  // leaf tile width of the FP64 kernel
    F64Geom geom{};  // host copy (device pointers inside)
    long long total_tasks = 0;
    double timeout_s = 5.0;
    int poison = 0;
    double wscale = 1.0;  // (den_u den_v den_w)^-depth of a rational algorithm, applied with W
    // product sharding: this plan computes sub-problems [sub_begin, sub_end) of nsub
    int shard_count = 1;
    long long sub_begin = 0, sub_end = 0;
    // double complex (FMM_C128, FMM_C128_3M): the FP64 plan the real parts run on, and its planes
    fmm_plan *inner = nullptr;
    double *d_planes = nullptr;
    // device memory
    void *d_tables = nullptr;     // geometry + CSC tables
    size_t tables_bytes = 0;
    void *d_ws = nullptr;         // counters (zeroed per call) + materialized operands
    size_t counters_bytes = 0;
    size_t ws_bytes = 0;
    unsigned *d_chain = nullptr;
    unsigned long long *d_task_counter = nullptr;
    unsigned long long *d_task_counter2 = nullptr;  // second launch of a call (peel after emulated leaf)
    int *d_error = nullptr;
    double *d_SA = nullptr, *d_SB = nullptr;  // materialized sources (nullptr when fused)
    double *d_TA = nullptr, *d_TB = nullptr;  // intermediate level (materialized depth >= 2)
    // materialization steps, applied in order over all materialized levels:
    // one per level, or the Kronecker factors of a composed level (fewer adds)
    struct MatStep {
        int p = 0, R = 0;
        const int *uptr = nullptr, *vptr = nullptr;
        const int4 *uent = nullptr, *vent = nullptr;
        bool unit_u = false, unit_v = false;  // every coefficient of the step's U (V) is +-1
        bool with_next = false;  // formed in one pass with the next step (both 2 x 2, at most 8 products)
    };
    std::vector<MatStep> mat_steps;
    // emulated leaf (FMM_F64_OZAKI)
    int oz_s = 0, oz_L = 0, oz_kparts = 1;
    int64_t oz_Mp = 0;
    unsigned char *d_sla = nullptr, *d_slb = nullptr;  // slices
    int *d_mxa = nullptr, *d_mxb = nullptr;            // exponents (zeroed per call with the counters)
    const F64Geom *d_geom_peel = nullptr;              // FP64 peel-only geometry
    int oz_engine = 2;                                  // 2 = tcgen05 CTA pairs, 1 = tcgen05, 0 = mma.sync
    CUtensorMap oz_map_a{}, oz_map_b{}, oz_map_bh{};    // TMA maps over the slices (h: 64-row boxes)
    double *d_pout = nullptr;                           // [R][m][m] leaf products of the tcgen05 engines
    const int *d_wl_ptr = nullptr;                      // per C block: products (r, coefficient) in ascending r
    const int2 *d_wl_ent = nullptr;
    double flops_lowp = 0;
    // FMM_F64 plans whose leaf products are stored and summed level by level in separate passes:
    // the passes (tables set at creation; buffers, C, alpha and beta per call), the product and
    // intermediate buffers, the leaf launch's geometry (border and core tasks, products stored)
    // and the rank-q launch's (after the passes)
    bool post_levels = false;
    bool oz_levels = false;  // FMM_F64_OZAKI: its stored products summed by the same passes
    std::vector<fmm::LevelPass> level_passes;
    double *d_pbuf = nullptr, *d_xbuf = nullptr;
    const F64Geom *d_geom_leaf = nullptr, *d_geom_rq = nullptr;
    long long leaf_tasks = 0, rq_tasks = 0;
    // host-buffer path: device copies of the operands, a stream for B's copy and its events
    double *d_hostA = nullptr, *d_hostB = nullptr, *d_hostC = nullptr;
    cudaStream_t host_copy_stream = nullptr;
    cudaEvent_t host_ev[2] = {nullptr, nullptr};
    // set only inside fmm_gemm_host: the event B's copy records; the pre-additions of B wait for it
    cudaEvent_t b_ready = nullptr;
    // optional timing events: [0] call start, [1] leaf start, [2] leaf end,
    // [3] after counter reset + materialization, [4] call end, [5] after the
    // separate post-additions of the emulated leaf
    cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    bool timed_once = false;
    // statistics
    double flops_leaf = 0, flops_exec = 0;
    long long total_products_hint = 0;
    int grid = 0;
    int sms = 0;
};

namespace {

fmm_status_t cuda_status(cudaError_t e) { return e == cudaSuccess ? FMM_OK : FMM_ERR_CUDA; }

// Every allocation the library makes for plans, the host-buffer path and the
// autotuner goes through these three functions, which keep a count of what is
// live and can be told to fail the k-th next request (fmm_debug_fail_allocation),
// so that each error path can be tested without exhausting a device.
std::atomic<long long> g_live_allocs{0};
std::atomic<long long> g_fail_countdown{-1};

bool inject_failure() {
    long long k = g_fail_countdown.load();
    while (k >= 0) {
        if (g_fail_countdown.compare_exchange_weak(k, k - 1)) return k == 0;
    }
    return false;
}

cudaError_t dev_alloc(void **p, size_t bytes) {
    *p = nullptr;
    if (inject_failure()) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) ++g_live_allocs;
    else cudaGetLastError();
    return e;
}
template <class T>
cudaError_t dev_alloc(T **p, size_t bytes) {
    void *q = nullptr;
    const cudaError_t e = dev_alloc(&q, bytes);
    *p = static_cast<T *>(q);
    return e;
}
void dev_free(void *p) {
    if (!p) return;
    cudaFree(p);
    --g_live_allocs;
}
// Page-locked host memory (fmm_host_alloc).  A request of at least one
// transparent huge page is mapped at a huge-page boundary, rounded up to whole
// huge pages, advised to use them and registered with the driver; anything
// else, or a registration the driver refuses, comes from cudaHostAlloc.  The
// registry maps each returned address to how it was obtained.
struct HostBlock {
    size_t len;       // bytes mapped and registered (0: cudaHostAlloc memory)
};
std::mutex g_host_mu;
std::unordered_map<void *, HostBlock> g_host_blocks;

size_t huge_page_bytes() {
    static const size_t hp = [] {
        unsigned long long v = 0;
        if (FILE *f = std::fopen("/sys/kernel/mm/transparent_hugepage/hpage_pmd_size", "r")) {
            if (std::fscanf(f, "%llu", &v) != 1) v = 0;
            std::fclose(f);
        }
        const long page = sysconf(_SC_PAGESIZE);
        // a usable size is a power of two above the base page
        if (page <= 0 || v <= (unsigned long long)page || (v & (v - 1)) != 0) v = 0;
        return (size_t)v;
    }();
    return hp;
}

void *huge_page_registered(size_t bytes, size_t *len_out) {
    const size_t hp = huge_page_bytes();
    if (hp == 0 || bytes < hp || bytes > SIZE_MAX / 2 - hp) return nullptr;
    const size_t len = (bytes + hp - 1) / hp * hp;
    void *raw = mmap(nullptr, len + hp, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
    if (raw == MAP_FAILED) return nullptr;
    const uintptr_t r = (uintptr_t)raw, a = (r + hp - 1) / hp * hp;
    const size_t head = a - r, tail = hp - head;
    if (head) munmap(raw, head);
    if (tail) munmap(reinterpret_cast<void *>(a + len), tail);
    void *q = reinterpret_cast<void *>(a);
    madvise(q, len, MADV_HUGEPAGE);  // advice only: without huge pages the buffer still works
    if (cudaHostRegister(q, len, cudaHostRegisterPortable) != cudaSuccess) {
        cudaGetLastError();
        munmap(q, len);
        return nullptr;
    }
    *len_out = len;
    return q;
}

cudaError_t pinned_alloc(void **p, size_t bytes) {
    *p = nullptr;
    if (inject_failure()) return cudaErrorMemoryAllocation;
    size_t len = 0;
    void *q = huge_page_registered(bytes, &len);
    if (!q) {
        const cudaError_t e = cudaHostAlloc(&q, bytes ? bytes : 1, cudaHostAllocPortable);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return e;
        }
        len = 0;
    }
    {
        std::lock_guard<std::mutex> lk(g_host_mu);
        g_host_blocks[q] = HostBlock{len};
    }
    ++g_live_allocs;
    *p = q;
    return cudaSuccess;
}
bool pinned_free(void *p) {
    HostBlock b{};
    {
        std::lock_guard<std::mutex> lk(g_host_mu);
        auto it = g_host_blocks.find(p);
        if (it == g_host_blocks.end()) return false;
        b = it->second;
        g_host_blocks.erase(it);
    }
    if (b.len) {
        cudaHostUnregister(p);
        munmap(p, b.len);
    } else {
        cudaFreeHost(p);
    }
    cudaGetLastError();
    --g_live_allocs;
    return true;
}
// Host objects of the library (plans, batch graphs, launch descriptors).
template <class T>
T *host_new() {
    if (inject_failure()) return nullptr;
    T *x = new (std::nothrow) T();
    if (x) ++g_live_allocs;
    return x;
}
template <class T>
void host_delete(T *x) {
    if (!x) return;
    delete x;
    --g_live_allocs;
}

// cuTensorMapEncodeTiled from the CUDA driver library, without linking libcuda.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
        else
            cudaGetLastError();
    }
    return fn;
}

// 2-D uint8 map over `rows` x `kp` bytes (row pitch kp), 128 x 128 boxes, 128B swizzle.
// TMA map over slices stored as rows x kp bytes; boxes of 128 K-bytes by box_rows rows.
bool make_slice_map(CUtensorMap *map, void *base, unsigned long long rows, unsigned long long kp,
                    unsigned box_rows = 128) {
    auto enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t dims[2] = {kp, rows};
    const cuuint64_t strides[1] = {kp};
    const cuuint32_t box[2] = {128, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

void free_plan_memory(fmm_plan *pl) {
    if (pl->inner) {
        free_plan_memory(pl->inner);
        host_delete(pl->inner);
        pl->inner = nullptr;
    }
    dev_free(pl->d_planes);
    pl->d_planes = nullptr;
    for (auto &e : pl->ev)
        if (e) { cudaEventDestroy(e); e = nullptr; }
    dev_free(pl->d_tables);
    dev_free(pl->d_ws);
    dev_free(pl->d_hostA);
    dev_free(pl->d_hostB);
    dev_free(pl->d_hostC);
    for (auto &e : pl->host_ev)
        if (e) { cudaEventDestroy(e); e = nullptr; }
    if (pl->host_copy_stream) cudaStreamDestroy(pl->host_copy_stream);
    pl->host_copy_stream = nullptr;
    pl->d_tables = pl->d_ws = nullptr;
    pl->d_hostA = pl->d_hostB = pl->d_hostC = nullptr;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Default number of materialized levels.  On GB300 the FP64 pipe is the
// scarce resource (about 1 TFLOP/s) while HBM bandwidth and capacity are
// plentiful: a pre-addition fused into operand staging is recomputed once per
// output tile column (m / kBN times), a materialized one once, and forming
// the levels one at a time shares each level's sums across all products below
// it.  So every level whose operands combine more than one block on average
// is materialized; algorithms whose columns are single blocks stay fused.
// One recursion level's U and V, possibly a Kronecker factor of them.
struct LevelFactor {
    int p = 0, R = 0;
    std::vector<int32_t> U, V;
};

// X (p^2 x R, row-major blocks, indexed as fmm_algo_compose builds products:
// block (i1 p2 + i2, j1 p2 + j2), product r1 R2 + r2) as X1 (p1^2 x R1)
// Kronecker X2 (p2^2 x R2) with integer entries.  The factors are read off a
// +-1 entry and the product is then checked entry by entry.
bool kron_split(const std::vector<int32_t> &X, int p, int R, int p1, int R1, std::vector<int32_t> &X1,
                std::vector<int32_t> &X2) {
    const int p2 = p / p1, R2 = R / R1;
    auto at = [&](int i1, int j1, int i2, int j2, int r1, int r2) {
        return X[((size_t)(i1 * p2 + i2) * p + (j1 * p2 + j2)) * R + (size_t)r1 * R2 + r2];
    };
    int a0 = -1, b0 = -1, c0 = -1, d0 = -1, v0 = 0;
    for (int a = 0; a < p1 * p1 && v0 == 0; ++a)
        for (int b = 0; b < p2 * p2 && v0 == 0; ++b)
            for (int c = 0; c < R1 && v0 == 0; ++c)
                for (int d = 0; d < R2 && v0 == 0; ++d) {
                    const int v = at(a / p1, a % p1, b / p2, b % p2, c, d);
                    if (v == 1 || v == -1) { a0 = a; b0 = b; c0 = c; d0 = d; v0 = v; }
                }
    if (v0 == 0) return false;
    X1.assign((size_t)p1 * p1 * R1, 0);
    X2.assign((size_t)p2 * p2 * R2, 0);
    for (int a = 0; a < p1 * p1; ++a)
        for (int c = 0; c < R1; ++c) X1[(size_t)a * R1 + c] = at(a / p1, a % p1, b0 / p2, b0 % p2, c, d0) * v0;
    for (int b = 0; b < p2 * p2; ++b)
        for (int d = 0; d < R2; ++d) X2[(size_t)b * R2 + d] = at(a0 / p1, a0 % p1, b / p2, b % p2, c0, d);
    for (int a = 0; a < p1 * p1; ++a)
        for (int b = 0; b < p2 * p2; ++b)
            for (int c = 0; c < R1; ++c)
                for (int d = 0; d < R2; ++d)
                    if ((int64_t)X1[(size_t)a * R1 + c] * X2[(size_t)b * R2 + d] !=
                        (int64_t)at(a / p1, a % p1, b / p2, b % p2, c, d))
                        return false;
    return true;
}

// FP64 adds of forming one level by the steps `seq`, per element of its input.
double steps_cost(const std::vector<LevelFactor> &seq) {
    double cost = 0, cnt = 1, area = 1;
    for (const LevelFactor &f : seq) {
        long long nu = 0, nv = 0;
        for (int32_t x : f.U) nu += x != 0;
        for (int32_t x : f.V) nv += x != 0;
        area /= (double)f.p * f.p;
        cost += cnt * (double)(nu - f.R + nv - f.R) * area;
        cnt *= f.R;
    }
    return cost;
}

// Cheapest sequence of materialization steps for one level: the level itself,
// or (recursively) Kronecker factors of its U and V with equal shapes.
std::vector<LevelFactor> decompose_level(const LevelFactor &f) {
    std::vector<LevelFactor> best{f};
    double best_cost = steps_cost(best);
    for (int p1 = 2; p1 < f.p; ++p1) {
        if (f.p % p1) continue;
        for (int R1 = 2; R1 < f.R; ++R1) {
            if (f.R % R1) continue;
            LevelFactor a, b;
            a.p = p1; a.R = R1; b.p = f.p / p1; b.R = f.R / R1;
            if (!kron_split(f.U, f.p, f.R, p1, R1, a.U, b.U) || !kron_split(f.V, f.p, f.R, p1, R1, a.V, b.V)) continue;
            std::vector<LevelFactor> seq = decompose_level(a);
            for (const LevelFactor &x : decompose_level(b)) seq.push_back(x);
            const double c = steps_cost(seq);
            if (c < best_cost) { best_cost = c; best = seq; }
        }
    }
    return best;
}

// W of one recursion level, or a Kronecker factor of it (the post-additions).
struct WFactor {
    int p = 0, R = 0;
    std::vector<int32_t> W;
};

// FP64 operations of summing one level's products into its blocks by the
// factors `seq`, innermost first, per position of a leaf block: factor k
// runs once per (product of the outer factors, block of the inner ones).
double w_steps_cost(const std::vector<WFactor> &seq) {
    double cost = 0;
    for (size_t k = 0; k < seq.size(); ++k) {
        double groups = 1;
        for (size_t j = 0; j < k; ++j) groups *= seq[j].R;
        for (size_t j = k + 1; j < seq.size(); ++j) groups *= (double)seq[j].p * seq[j].p;
        long long nnz = 0;
        for (int32_t x : seq[k].W) nnz += x != 0;
        cost += groups * (double)nnz;
    }
    return cost;
}

// Cheapest sequence of Kronecker factors of one level's W (the level itself
// when it has none), outermost first.
std::vector<WFactor> decompose_w(const WFactor &f) {
    std::vector<WFactor> best{f};
    double best_cost = w_steps_cost(best);
    for (int p1 = 2; p1 < f.p; ++p1) {
        if (f.p % p1) continue;
        for (int R1 = 2; R1 < f.R; ++R1) {
            if (f.R % R1) continue;
            WFactor a, b;
            a.p = p1; a.R = R1; b.p = f.p / p1; b.R = f.R / R1;
            if (!kron_split(f.W, f.p, f.R, p1, R1, a.W, b.W)) continue;
            std::vector<WFactor> seq = decompose_w(a);
            for (const WFactor &x : decompose_w(b)) seq.push_back(x);
            const double c = w_steps_cost(seq);
            if (c < best_cost) { best_cost = c; best = seq; }
        }
    }
    return best;
}

int default_materialized_levels(int p, int R, const fmm_algo_t *a, int depth) {
    if (depth < 1) return 0;
    long long nnz_u = 0, nnz_v = 0;
    for (int64_t x = 0; x < (int64_t)p * p * R; ++x) {
        nnz_u += a->U[x] != 0;
        nnz_v += a->V[x] != 0;
    }
    const double avg = 0.5 * (double)(nnz_u + nnz_v) / R;  // sources per operand per level
    return avg > 1.5 ? depth : 0;
}

// Leaf tile width.  Both widths run the same 64 x 32 warp tiles; the 64-column
// tile fits two CTAs per SM so that one CTA's prologue and epilogue overlap
// the other's MMAs, and it halves the ragged-tile waste for small leaves.
int default_tile_n(long long m, long long products) {
    (void)products;
    (void)m;
    const char *env = std::getenv("FMM_TILE_N");
    if (env && std::string(env) == "128") return 128;
    if (env && std::string(env) == "64") return 64;
    return 64;
}

}  // namespace

namespace {

// Plan creation for integer tables; `den` is the product of a rational
// algorithm's denominators (1 for an integer algorithm, whose Brent equations
// are checked here; a rational algorithm's are checked by the caller).
fmm_status_t plan_create(fmm_plan_t **out, int64_t n, const fmm_algo_t *algo, int depth, fmm_dtype_t dtype,
                         const fmm_plan_options_t *opts, int64_t den) {
    if (!out) return FMM_ERR_INVALID;
    *out = nullptr;
    if (n < 1 || depth < 0 || depth > 8 || !algo_shape_ok(algo) || den < 1) return FMM_ERR_INVALID;
    if (n > (1LL << 31) / 2) return FMM_ERR_UNSUPPORTED;
    if (opts && opts->shard_count > 1 && dtype != FMM_F64) return FMM_ERR_UNSUPPORTED;
    if (dtype == FMM_F32) {
        // an emulated-FP64 plan with fewer slices (6 by default: 30 bits for 24-bit operands) and
        // three binary64 planes for A, B and C
        fmm_plan_options_t o2{};
        if (opts) o2 = *opts;
        if (!o2.ozaki_slices) o2.ozaki_slices = 6;
        fmm_plan_t *inner = nullptr;
        fmm_status_t st = plan_create(&inner, n, algo, depth, FMM_F64_OZAKI, &o2, den);
        if (st != FMM_OK) return st;
        fmm_plan *pl = host_new<fmm_plan>();
        if (!pl) {
            fmm_plan_destroy(inner);
            return FMM_ERR_OOM;
        }
        pl->inner = inner;
        pl->device = inner->device;
        pl->n = n; pl->p = inner->p; pl->R = inner->R; pl->depth = depth; pl->dtype = dtype;
        pl->wscale = inner->wscale;
        pl->ws_bytes = 3 * (size_t)n * (size_t)n * sizeof(double);
        if (dev_alloc(&pl->d_planes, pl->ws_bytes) != cudaSuccess) {
            fmm_plan_destroy(pl);
            return FMM_ERR_OOM;
        }
        if (opts && opts->record_kernel_time)
            for (int e : {0, 1, 2})
                if (cudaEventCreate(&pl->ev[e]) != cudaSuccess) {
                    cudaGetLastError();
                    fmm_plan_destroy(pl);
                    return FMM_ERR_CUDA;
                }
        *out = pl;
        return FMM_OK;
    }
    if (dtype == FMM_C128 || dtype == FMM_C128_3M) {
        // a real plan for the parts, and the planes: 4M splits A, B and C (6 planes),
        // 3M splits A and B with their part sums and keeps three products (9 planes)
        fmm_plan_t *inner = nullptr;
        fmm_status_t st = plan_create(&inner, n, algo, depth, FMM_F64, opts, den);
        if (st != FMM_OK) return st;
        fmm_plan *pl = host_new<fmm_plan>();
        if (!pl) {
            fmm_plan_destroy(inner);
            return FMM_ERR_OOM;
        }
        pl->inner = inner;
        pl->device = inner->device;
        pl->n = n; pl->p = inner->p; pl->R = inner->R; pl->depth = depth; pl->dtype = dtype;
        pl->wscale = inner->wscale;
        const size_t planes = dtype == FMM_C128 ? 6 : 9;
        pl->ws_bytes = planes * (size_t)n * (size_t)n * sizeof(double);
        if (dev_alloc(&pl->d_planes, pl->ws_bytes) != cudaSuccess) {
            fmm_plan_destroy(pl);
            return FMM_ERR_OOM;
        }
        if (opts && opts->record_kernel_time)
            for (int e : {0, 1, 2})
                if (cudaEventCreate(&pl->ev[e]) != cudaSuccess) {
                    cudaGetLastError();
                    fmm_plan_destroy(pl);
                    return FMM_ERR_CUDA;
                }
        *out = pl;
        return FMM_OK;
    }
    if (dtype != FMM_F64 && dtype != FMM_F64_OZAKI) return FMM_ERR_UNSUPPORTED;
    if (den == 1 && fmm_algo_brent_mismatches(algo) != 0) return FMM_ERR_BRENT;
    const int shards = opts && opts->shard_count > 1 ? opts->shard_count : 1;
    if (opts && (opts->shard_count < 0 || opts->shard_index < 0 || opts->shard_index >= shards))
        return FMM_ERR_INVALID;
    // the scale (den^depth)^-1, rounded once; den^depth must be an exact double
    double den_d = 1.0;
    for (int l = 0; l < depth; ++l) {
        den_d *= (double)den;
        if (den_d > 9007199254740992.0) return FMM_ERR_UNSUPPORTED;
    }
    const int p = algo->p, R = algo->R;
    const long long P = ipow(p, depth);
    const long long Rt = ipow(R, depth);
    if (P > n) return FMM_ERR_INVALID;  // leaf size would be < 1
    if (Rt > (1LL << 24)) return FMM_ERR_UNSUPPORTED;

    int mat = 0;
    fmm_plan_options_t o{};
    if (opts) o = *opts;
    if (o.schedule == FMM_SCHED_FUSED) mat = 0;
    else if (o.schedule == FMM_SCHED_HYBRID) mat = o.materialize_levels;
    else mat = default_materialized_levels(p, R, algo, depth);
    if (mat < 0 || mat > depth) return FMM_ERR_INVALID;
    int oz_s = 0;
    if (dtype == FMM_F64_OZAKI) {
        // S_r and T_r must exist in FP64 before they are sliced: materialize all levels.
        if (o.schedule != FMM_SCHED_AUTO && mat != depth) return FMM_ERR_UNSUPPORTED;
        mat = depth;
        oz_s = o.ozaki_slices ? o.ozaki_slices : 12;
        if (oz_s < 2 || oz_s > fmm::kOzMaxSlices) return FMM_ERR_INVALID;
        if (n / P > (1LL << 30) / 128) return FMM_ERR_UNSUPPORTED;
    }

    fmm_plan *pl = host_new<fmm_plan>();
    if (!pl) return FMM_ERR_OOM;
    cudaGetDevice(&pl->device);
    pl->n = n; pl->p = p; pl->R = R; pl->depth = depth; pl->dtype = dtype; pl->mat_levels = mat;
    pl->wscale = 1.0 / den_d;
    pl->P = P; pl->R_total = Rt;
    pl->m = n / P;
    pl->n_core = P * pl->m;
    pl->P_src = ipow(p, depth - mat);
    pl->R_src = ipow(R, depth - mat);
    pl->nsub = ipow(R, mat);
    pl->b_src = pl->P_src * pl->m;
    // the shard's range of sub-problems (all of them unless sharded)
    pl->shard_count = shards;
    if (shards > (long long)pl->nsub) {
        host_delete(pl);
        return FMM_ERR_UNSUPPORTED;
    }
    {
        int64_t b = 0, e = 0;
        fmm_shard_range((int64_t)pl->nsub, shards, shards > 1 ? opts->shard_index : 0, &b, &e);
        pl->sub_begin = b;
        pl->sub_end = e;
    }
    const long long prod_lo = pl->sub_begin * pl->R_src, prod_hi = pl->sub_end * pl->R_src;
    const bool with_peel = pl->sub_begin == 0;
    pl->tiles_m = (int)((pl->m + fmm::kBM - 1) / fmm::kBM);
    if (dtype == FMM_F64_OZAKI) {
        pl->bn = fmm::kBN;  // the slice GEMM and its counters use 128 x 128 tiles
    } else if (o.tile_n) {
        if (o.tile_n != 64 && o.tile_n != 128) { host_delete(pl); return FMM_ERR_INVALID; }
        pl->bn = o.tile_n;
    } else {
        pl->bn = default_tile_n(pl->m, pl->total_products_hint = Rt);
    }
    pl->tiles_n = (int)((pl->m + pl->bn - 1) / pl->bn);
    if (o.wait_timeout_s > 0) pl->timeout_s = o.wait_timeout_s;
    pl->poison = o.debug_poison_chain;

    // Coefficient tables: bottom levels for the fused operands, all levels for W.
    auto ucols = flatten(p, R, algo->U, depth - mat);
    auto vcols = flatten(p, R, algo->V, depth - mat);
    auto wcols = flatten(p, R, algo->W, depth);
    // Materialization: each level formed by its cheapest sequence of Kronecker
    // factors (the level itself when it has none); product and block order
    // match the flattened algorithm because composition nests the same way.
    std::vector<LevelFactor> steps;
    if (mat > 0) {
        LevelFactor lvl;
        lvl.p = p; lvl.R = R;
        lvl.U.assign(algo->U, algo->U + (size_t)p * p * R);
        lvl.V.assign(algo->V, algo->V + (size_t)p * p * R);
        steps = decompose_level(lvl);
    }
    size_t maxc = 0;
    for (auto &c : ucols) maxc = std::max(maxc, c.size());
    for (auto &c : vcols) maxc = std::max(maxc, c.size());
    for (auto &c : wcols) maxc = std::max(maxc, c.size());
    if (maxc > (size_t)fmm::kMaxTerms) { host_delete(pl); return FMM_ERR_UNSUPPORTED; }

    auto csc2 = [](const std::vector<std::vector<Entry>> &cols, std::vector<int> &ptr, std::vector<int2> &ent) {
        ptr.assign(cols.size() + 1, 0);
        for (size_t c = 0; c < cols.size(); ++c) {
            ptr[c + 1] = ptr[c] + (int)cols[c].size();
            for (const Entry &e : cols[c]) ent.push_back(make_int2(e.blk, e.coef));
        }
    };
    std::vector<int> u_ptr, v_ptr, w_ptr, w_row((size_t)P * P, 0);
    std::vector<int2> u_ent, v_ent;
    std::vector<int4> w_ent;
    csc2(ucols, u_ptr, u_ent);
    csc2(vcols, v_ptr, v_ent);
    // per materialization step: CSC over its products of {block row, block col, coefficient as the two
    // words of a double}, and whether every coefficient of the step is +-1
    std::vector<std::vector<int>> st_uptr(steps.size()), st_vptr(steps.size());
    std::vector<std::vector<int4>> st_uent(steps.size()), st_vent(steps.size());
    std::vector<char> st_unit_u(steps.size(), 1), st_unit_v(steps.size(), 1);
    auto mat_entry = [](int blk, int p, int c) {
        const double d = (double)c;
        unsigned long long bits = 0;
        std::memcpy(&bits, &d, sizeof bits);
        return make_int4(blk / p, blk % p, (int)(unsigned)(bits & 0xffffffffULL), (int)(unsigned)(bits >> 32));
    };
    for (size_t k = 0; k < steps.size(); ++k) {
        const LevelFactor &f = steps[k];
        std::vector<int2> tmp;
        csc2(flatten(f.p, f.R, f.U.data(), 1), st_uptr[k], tmp);
        for (const int2 &e : tmp) {
            st_uent[k].push_back(mat_entry(e.x, f.p, e.y));
            if (e.y != 1 && e.y != -1) st_unit_u[k] = 0;
        }
        tmp.clear();
        csc2(flatten(f.p, f.R, f.V.data(), 1), st_vptr[k], tmp);
        for (const int2 &e : tmp) {
            st_vent[k].push_back(mat_entry(e.x, f.p, e.y));
            if (e.y != 1 && e.y != -1) st_unit_v[k] = 0;
        }
    }
    // W entries of every product; the ordering positions (and each C block's count of contributions)
    // cover only the shard's products, the others are never read
    w_ptr.assign(wcols.size() + 1, 0);
    for (size_t c = 0; c < wcols.size(); ++c) {
        w_ptr[c + 1] = w_ptr[c] + (int)wcols[c].size();
        const bool mine = (long long)c >= prod_lo && (long long)c < prod_hi;
        for (const Entry &e : wcols[c]) w_ent.push_back(make_int4(e.blk, e.coef, mine ? w_row[e.blk]++ : 0, 0));
    }
    // the same nonzeros by C block, products in ascending order (separate post-additions)
    std::vector<int> wl_ptr((size_t)P * P + 1, 0);
    std::vector<int2> wl_ent(w_ent.size());
    for (size_t l = 0; l < (size_t)P * P; ++l) wl_ptr[l + 1] = wl_ptr[l] + w_row[l];
    for (size_t c = 0; c < wcols.size(); ++c) {
        if ((long long)c < prod_lo || (long long)c >= prod_hi) continue;
        for (int k = w_ptr[c]; k < w_ptr[c + 1]; ++k) {
            const int4 &e = w_ent[k];
            wl_ent[wl_ptr[e.x] + e.z] = make_int2((int)c, e.y);
        }
    }

    const char *post_env = std::getenv("FMM_OZAKI_POSTADD");
    const bool oz_flat = post_env && std::string(post_env) == "flat";

    // Stored leaf products, summed level by level (FMM_F64, and FMM_F64_OZAKI from depth 2): W's
    // Kronecker factors over all levels, outermost first; passes from the innermost factor up, two 2 x 2
    // factors of at most 8 products at a time, else one.  FMM_F64: option, then FMM_F64_POSTADD (fused /
    // levels), then the planner's choice; FMM_F64_OZAKI: always, unless FMM_OZAKI_POSTADD=flat.
    int post_mode = o.post_additions;
    if (post_mode < 0 || post_mode > 2) { host_delete(pl); return FMM_ERR_INVALID; }
    if (post_mode == 0)
        if (const char *pe = std::getenv("FMM_F64_POSTADD")) {
            if (std::string(pe) == "fused") post_mode = 1;
            if (std::string(pe) == "levels") post_mode = 2;
        }
    std::vector<WFactor> wseq;
    if ((dtype == FMM_F64 && depth >= 1) || (dtype == FMM_F64_OZAKI && depth >= 2 && !oz_flat)) {
        WFactor lvl;
        lvl.p = p; lvl.R = R;
        lvl.W.assign(algo->W, algo->W + (size_t)p * p * R);
        const std::vector<WFactor> wf = decompose_w(lvl);
        for (int lev = 0; lev < depth; ++lev)
            for (const WFactor &f : wf) wseq.push_back(f);
    }
    bool levels_ok = !wseq.empty() && shards == 1 && !o.debug_poison_chain;
    for (const WFactor &f : wseq) {
        if (f.p * f.p > fmm::kLevelMaxQ) levels_ok = false;
        for (int q = 0; q < f.p * f.p; ++q) {
            bool any = false;
            for (int r = 0; r < f.R; ++r) any = any || f.W[(size_t)q * f.R + r] != 0;
            if (!any) levels_ok = false;
        }
    }
    if (dtype == FMM_F64 && post_mode == 2 && !levels_ok && depth >= 1) {
        host_delete(pl);
        return FMM_ERR_UNSUPPORTED;
    }
    if (dtype == FMM_F64 && post_mode == 0 && levels_ok) {
        // The planner stores the products when the fused epilogue's adds, (nnz(W flattened) - P^2) m^2,
        // reach 0.4 % of the leaf's 2 R^depth m^3 flops, and the product buffers take at most a quarter
        // of the free device memory.  Measured at n = 1024 .. 8192 (Strassen depth 1-7, <4,4,4;49>,
        // Winograd, Laderman): above that ratio the stored form was faster, by 1.1 % (n = 4096, depth 3,
        // ratio 0.0095) up to 3.8x (n = 8192, depth 7); below it the two were within 0.7 % of each
        // other, except Laderman at n = 1024 (ratio 0.0054), 4.5 % slower stored.
        long long nnz_flat = 0;
        for (const auto &c : wcols) nnz_flat += (long long)c.size();
        const double ratio = (double)(nnz_flat - P * P) / ((double)Rt * (double)pl->m);
        const double extra = 1.5 * (double)Rt * (double)pl->m * (double)pl->m * sizeof(double);
        size_t free_b = 0, total_b = 0;
        const bool room = cudaMemGetInfo(&free_b, &total_b) == cudaSuccess && extra <= 0.25 * (double)free_b;
        if (!room) cudaGetLastError();
        post_mode = ratio >= 0.008 && room ? 2 : 1;
    }
    const bool post_levels = dtype == FMM_F64 && levels_ok && post_mode == 2;
    const bool oz_levels = dtype == FMM_F64_OZAKI && levels_ok;
    const bool build_levels = post_levels || oz_levels;
    struct PassTables {
        std::vector<int> bptr, aptr;
        std::vector<int4> bent, aent;
    };
    std::vector<fmm::LevelPass> lpasses;
    std::vector<PassTables> ltables;
    std::vector<int2> c_blk;
    double post_fma = 0;  // FP64 operations of the passes, per position of a leaf block
    if (build_levels) {
        auto words = [](int c, int &lo, int &hi) {
            const double d = (double)c;
            unsigned long long bits = 0;
            std::memcpy(&bits, &d, sizeof bits);
            lo = (int)(unsigned)(bits & 0xffffffffULL);
            hi = (int)(unsigned)(bits >> 32);
        };
        // columns r of f's W: {q, coefficient, flags: 1 first term of row q, 2 coefficient +-1}
        auto by_columns = [&](const WFactor &f, std::vector<int> &ptr, std::vector<int4> &ent) {
            const int Q = f.p * f.p;
            std::vector<int> first(Q, -1);
            for (int q = 0; q < Q; ++q)
                for (int r = 0; r < f.R && first[q] < 0; ++r)
                    if (f.W[(size_t)q * f.R + r]) first[q] = r;
            ptr.assign((size_t)f.R + 1, 0);
            for (int r = 0; r < f.R; ++r) {
                for (int q = 0; q < Q; ++q) {
                    const int c = f.W[(size_t)q * f.R + r];
                    if (!c) continue;
                    int lo = 0, hi = 0;
                    words(c, lo, hi);
                    ent.push_back(make_int4(q, lo, hi, (first[q] == r ? 1 : 0) | (c == 1 || c == -1 ? 2 : 0)));
                }
                ptr[r + 1] = (int)ent.size();
            }
        };
        long long np = 1, ns = 1;
        for (const WFactor &f : wseq) np *= f.R;
        for (int k = (int)wseq.size() - 1; k >= 0;) {
            fmm::LevelPass a{};
            PassTables t;
            const WFactor &fb = wseq[k];
            long long nnz_b = 0;
            for (int32_t x : fb.W) nnz_b += x != 0;
            if (k >= 1 && fb.p == 2 && wseq[k - 1].p == 2 && fb.R <= 8 && wseq[k - 1].R <= 8) {
                const WFactor &fa = wseq[k - 1];
                long long nnz_a = 0;
                for (int32_t x : fa.W) nnz_a += x != 0;
                np /= (long long)fa.R * fb.R;
                a.ra = fa.R; a.qa = 4; a.rb = fb.R; a.qb = 4;
                a.unit_b = 1;
                t.bptr.assign(5, 0);
                for (int q = 0; q < 4; ++q) {
                    for (int r = 0; r < fb.R; ++r) {
                        const int c = fb.W[(size_t)q * fb.R + r];
                        if (!c) continue;
                        int lo = 0, hi = 0;
                        words(c, lo, hi);
                        t.bent.push_back(make_int4(r, lo, hi, 0));
                        if (c != 1 && c != -1) a.unit_b = 0;
                    }
                    t.bptr[q + 1] = (int)t.bent.size();
                }
                by_columns(fa, t.aptr, t.aent);
                post_fma += (double)np * ns * (double)(fa.R * (nnz_b - 4) + 4 * (nnz_a - 4));
                k -= 2;
            } else {
                np /= fb.R;
                a.ra = 1; a.qa = 1; a.rb = fb.R; a.qb = fb.p * fb.p;
                by_columns(fb, t.bptr, t.bent);
                post_fma += (double)np * ns * (double)(nnz_b - a.qb);
                k -= 1;
            }
            a.np = (int)np;
            a.ns = (int)ns;
            ns *= (long long)a.qa * a.qb;
            a.m = pl->m;
            a.mm = pl->m * pl->m;
            a.last = k < 0;
            lpasses.push_back(a);
            ltables.push_back(std::move(t));
        }
        // C block (row, column) of output o of the last pass: digits q_k = i_k p_k + j_k, innermost last
        c_blk.resize((size_t)P * P);
        for (long long o2 = 0; o2 < P * P; ++o2) {
            long long rem = o2, row = 0, col = 0, mult = 1;
            for (int k = (int)wseq.size() - 1; k >= 0; --k) {
                const int pk = wseq[k].p;
                const long long q = rem % (pk * pk);
                rem /= pk * pk;
                row += (q / pk) * mult;
                col += (q % pk) * mult;
                mult *= pk;
            }
            c_blk[(size_t)o2] = make_int2((int)row, (int)col);
        }
    }

    // Task counts.
    const long long tiles = (long long)pl->tiles_m * pl->tiles_n;
    const long long q = n - pl->n_core;
    F64Geom &g = pl->geom;
    g.n = n; g.m = pl->m; g.n_core = pl->n_core;
    g.P = (int)P; g.P_src = (int)pl->P_src; g.R_src = (int)pl->R_src; g.nsub = (int)pl->nsub;
    g.tiles_m = pl->tiles_m; g.tiles_n = pl->tiles_n;
    g.bn = pl->bn;
    g.ld_src_a = mat > 0 ? pl->b_src : n;
    g.ld_src_b = g.ld_src_a;
    g.sub_stride_a = mat > 0 ? pl->b_src * pl->b_src : 0;
    g.sub_stride_b = g.sub_stride_a;
    g.sub_begin = (int)pl->sub_begin;
    g.tasks_core = tiles * (prod_hi - prod_lo);
    if (q > 0 && with_peel) {
        g.rb_tm = (int)((pl->n_core + fmm::kBM - 1) / fmm::kBM);
        g.rb_tn = (int)((q + pl->bn - 1) / pl->bn);
        g.bb_tm = (int)((q + fmm::kBM - 1) / fmm::kBM);
        g.bb_tn = (int)((n + pl->bn - 1) / pl->bn);
        g.tasks_right = (long long)g.rb_tm * g.rb_tn;
        g.tasks_bottom = (long long)g.bb_tm * g.bb_tn;
        g.tasks_rankq = (long long)P * P * tiles;
    }
    pl->total_tasks = g.tasks_core + g.tasks_right + g.tasks_bottom + g.tasks_rankq;

    // Flop accounting (executed, as scheduled; multiply-add = 2 flops).
    const double md = (double)pl->m;
    pl->flops_leaf = 2.0 * (double)(prod_hi - prod_lo) * md * md * md;
    double adds = 0;
    {
        long long nnz_u = (long long)u_ent.size(), nnz_v = (long long)v_ent.size();
        const double fused_factor_a = (double)pl->tiles_n;  // S slab rebuilt per tile column
        const double fused_factor_b = (double)pl->tiles_m;
        adds += (double)pl->nsub * ((double)(nnz_u - pl->R_src) * md * md * fused_factor_a +
                                    (double)(nnz_v - pl->R_src) * md * md * fused_factor_b);
        for (int lev = 1; lev <= mat; ++lev) {
            const double bl = (double)(pl->n_core / ipow(p, lev - 1));  // input side of the level
            adds += (double)ipow(R, lev - 1) * steps_cost(steps) * bl * bl;
        }
        long long w_nnz = 0, blocks_hit = 0;  // the shard's post-additions: all but each block's first term
        for (int c : w_row) {
            w_nnz += c;
            blocks_hit += c > 0;
        }
        adds += build_levels ? post_fma * md * md : (double)(w_nnz - blocks_hit) * md * md;
    }
    const double qd = with_peel ? (double)q : 0.0, ncd = (double)pl->n_core, nd = (double)n;
    const double peel = 2.0 * (ncd * qd * nd + qd * nd * nd + ncd * ncd * qd);
    pl->flops_exec = (dtype == FMM_F64_OZAKI ? 0.0 : pl->flops_leaf) + adds + peel;

    // Device tables.
    size_t off = 0;
    auto reserve = [&](size_t bytes) { size_t o2 = align_up(off, 256); off = o2 + bytes; return o2; };
    const size_t o_geom = reserve(sizeof(F64Geom));
    const size_t o_geom_peel = reserve(sizeof(F64Geom));
    const size_t o_uptr = reserve(u_ptr.size() * sizeof(int));
    const size_t o_uent = reserve(std::max<size_t>(1, u_ent.size()) * sizeof(int2));
    const size_t o_vptr = reserve(v_ptr.size() * sizeof(int));
    const size_t o_vent = reserve(std::max<size_t>(1, v_ent.size()) * sizeof(int2));
    const size_t o_wptr = reserve(w_ptr.size() * sizeof(int));
    const size_t o_went = reserve(std::max<size_t>(1, w_ent.size()) * sizeof(int4));
    const size_t o_wrow = reserve(w_row.size() * sizeof(int));
    const size_t o_wlptr = reserve(wl_ptr.size() * sizeof(int));
    const size_t o_wlent = reserve(std::max<size_t>(1, wl_ent.size()) * sizeof(int2));
    const size_t o_geom_leaf = reserve(sizeof(F64Geom));
    const size_t o_geom_rq = reserve(sizeof(F64Geom));
    const size_t o_cblk = reserve(std::max<size_t>(1, c_blk.size()) * sizeof(int2));
    std::vector<size_t> o_lp(4 * lpasses.size());
    for (size_t k = 0; k < lpasses.size(); ++k) {
        const PassTables &t = ltables[k];
        o_lp[4 * k] = reserve(t.bptr.size() * sizeof(int));
        o_lp[4 * k + 1] = reserve(std::max<size_t>(1, t.bent.size()) * sizeof(int4));
        o_lp[4 * k + 2] = reserve(std::max<size_t>(1, t.aptr.size()) * sizeof(int));
        o_lp[4 * k + 3] = reserve(std::max<size_t>(1, t.aent.size()) * sizeof(int4));
    }
    std::vector<size_t> o_st(4 * steps.size());
    for (size_t k = 0; k < steps.size(); ++k) {
        o_st[4 * k] = reserve(st_uptr[k].size() * sizeof(int));
        o_st[4 * k + 1] = reserve(std::max<size_t>(1, st_uent[k].size()) * sizeof(int4));
        o_st[4 * k + 2] = reserve(st_vptr[k].size() * sizeof(int));
        o_st[4 * k + 3] = reserve(std::max<size_t>(1, st_vent[k].size()) * sizeof(int4));
    }
    pl->tables_bytes = off;
    if (dev_alloc(&pl->d_tables, pl->tables_bytes) != cudaSuccess) {
        host_delete(pl);
        return FMM_ERR_OOM;
    }
    char *base = (char *)pl->d_tables;
    g.u_ptr = (const int *)(base + o_uptr);
    g.u_ent = (const int2 *)(base + o_uent);
    g.v_ptr = (const int *)(base + o_vptr);
    g.v_ent = (const int2 *)(base + o_vent);
    g.w_ptr = (const int *)(base + o_wptr);
    g.w_ent = (const int4 *)(base + o_went);
    g.w_row_nnz = (const int *)(base + o_wrow);
    pl->d_wl_ptr = (const int *)(base + o_wlptr);
    pl->d_wl_ent = (const int2 *)(base + o_wlent);
    std::vector<char> host(pl->tables_bytes, 0);
    auto put = [&](size_t o2, const void *src, size_t bytes) { if (bytes) std::memcpy(host.data() + o2, src, bytes); };
    put(o_uptr, u_ptr.data(), u_ptr.size() * sizeof(int));
    put(o_uent, u_ent.data(), u_ent.size() * sizeof(int2));
    put(o_vptr, v_ptr.data(), v_ptr.size() * sizeof(int));
    put(o_vent, v_ent.data(), v_ent.size() * sizeof(int2));
    put(o_wptr, w_ptr.data(), w_ptr.size() * sizeof(int));
    put(o_went, w_ent.data(), w_ent.size() * sizeof(int4));
    put(o_wrow, w_row.data(), w_row.size() * sizeof(int));
    put(o_wlptr, wl_ptr.data(), wl_ptr.size() * sizeof(int));
    put(o_wlent, wl_ent.data(), wl_ent.size() * sizeof(int2));
    for (size_t k = 0; k < steps.size(); ++k) {
        put(o_st[4 * k], st_uptr[k].data(), st_uptr[k].size() * sizeof(int));
        put(o_st[4 * k + 1], st_uent[k].data(), st_uent[k].size() * sizeof(int4));
        put(o_st[4 * k + 2], st_vptr[k].data(), st_vptr[k].size() * sizeof(int));
        put(o_st[4 * k + 3], st_vent[k].data(), st_vent[k].size() * sizeof(int4));
    }
    for (int lev = 0; lev < mat; ++lev)
        for (size_t k = 0; k < steps.size(); ++k) {
            fmm_plan::MatStep ms;
            ms.p = steps[k].p;
            ms.R = steps[k].R;
            ms.uptr = (const int *)(base + o_st[4 * k]);
            ms.uent = (const int4 *)(base + o_st[4 * k + 1]);
            ms.vptr = (const int *)(base + o_st[4 * k + 2]);
            ms.vent = (const int4 *)(base + o_st[4 * k + 3]);
            ms.unit_u = st_unit_u[k] != 0;
            ms.unit_v = st_unit_v[k] != 0;
            pl->mat_steps.push_back(ms);
        }
    for (size_t k = 0; k + 1 < pl->mat_steps.size(); ++k) {
        fmm_plan::MatStep &a = pl->mat_steps[k], &b = pl->mat_steps[k + 1];
        if (a.p == 2 && b.p == 2 && a.R <= 8 && b.R <= 8 && !(k > 0 && pl->mat_steps[k - 1].with_next)) a.with_next = true;
    }
    put(o_cblk, c_blk.data(), c_blk.size() * sizeof(int2));
    for (size_t k = 0; k < lpasses.size(); ++k) {
        const PassTables &t = ltables[k];
        put(o_lp[4 * k], t.bptr.data(), t.bptr.size() * sizeof(int));
        put(o_lp[4 * k + 1], t.bent.data(), t.bent.size() * sizeof(int4));
        put(o_lp[4 * k + 2], t.aptr.data(), t.aptr.size() * sizeof(int));
        put(o_lp[4 * k + 3], t.aent.data(), t.aent.size() * sizeof(int4));
        fmm::LevelPass &a = lpasses[k];
        a.b_ptr = (const int *)(base + o_lp[4 * k]);
        a.b_ent = (const int4 *)(base + o_lp[4 * k + 1]);
        a.a_ptr = t.aptr.empty() ? nullptr : (const int *)(base + o_lp[4 * k + 2]);
        a.a_ent = t.aent.empty() ? nullptr : (const int4 *)(base + o_lp[4 * k + 3]);
        a.c_blk = (const int2 *)(base + o_cblk);
    }
    pl->post_levels = post_levels;
    pl->oz_levels = oz_levels;
    pl->level_passes = lpasses;
    pl->d_geom_leaf = (const F64Geom *)(base + o_geom_leaf);
    pl->d_geom_rq = (const F64Geom *)(base + o_geom_rq);
    put(o_geom, &g, sizeof(F64Geom));
    {
        F64Geom gp = g;  // the peel tasks alone, run after the emulated leaf products and their post-additions
        gp.tasks_core = 0;
        gp.rankq_free = 1;
        put(o_geom_peel, &gp, sizeof(F64Geom));
        pl->d_geom_peel = (const F64Geom *)(base + o_geom_peel);
    }
    if (cudaMemcpy(pl->d_tables, host.data(), pl->tables_bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        free_plan_memory(pl);
        host_delete(pl);
        return FMM_ERR_CUDA;
    }

    // Workspace: [error int][pad][task counter u64][second task counter u64]
    // [pad][chain counters] then the materialized operands.
    const size_t chain_count = (size_t)P * P * (size_t)tiles;
    pl->counters_bytes = align_up(32 + chain_count * sizeof(unsigned), 256);
    size_t o_mx = 0;
    if (dtype == FMM_F64_OZAKI) {
        pl->oz_s = oz_s;
        pl->oz_Mp = (pl->m + 127) / 128 * 128;
        o_mx = pl->counters_bytes;
        pl->counters_bytes = align_up(o_mx + 2 * (size_t)Rt * (size_t)pl->oz_Mp * sizeof(int), 256);
        // int64 recombination stays below 2^62: L >= log2(1.1 Kp 256) + 5 (s - 1) - 62
        const double lg = std::log2(1.1 * (double)pl->oz_Mp * 256.0) + fmm::kOzDigitBits * (oz_s - 1) - 62.0;
        pl->oz_L = lg > 0 ? (int)std::ceil(lg) : 0;
        const double mp = (double)pl->oz_Mp;
        pl->flops_lowp = 2.0 * (double)Rt * (oz_s * (oz_s + 1) / 2) * mp * mp * mp;
    }
    size_t ws = pl->counters_bytes;
    size_t o_sa = 0, o_sb = 0, o_ta = 0, o_tb = 0;
    if (mat > 0) {
        // passes (a step, or two fused steps) alternate between the final buffer and one
        // temporary, ending in the final buffer
        size_t fin_bytes = 0, tmp_bytes = 0;
        {
            std::vector<size_t> outs;
            double cnt = 1, side = (double)pl->n_core;
            for (size_t k = 0; k < pl->mat_steps.size(); ++k) {
                const fmm_plan::MatStep &st = pl->mat_steps[k];
                cnt *= st.R;
                side /= st.p;
                if (!st.with_next) outs.push_back((size_t)(cnt * side * side) * sizeof(double));
            }
            const size_t G = outs.size();
            for (size_t g = 1; g <= G; ++g) {
                if ((G - g) % 2 == 0) fin_bytes = std::max(fin_bytes, outs[g - 1]);
                else tmp_bytes = std::max(tmp_bytes, outs[g - 1]);
            }
        }
        o_sa = ws; ws = align_up(ws + fin_bytes, 256);
        o_sb = ws; ws = align_up(ws + fin_bytes, 256);
        if (tmp_bytes > 0) {
            o_ta = ws; ws = align_up(ws + tmp_bytes, 256);
            o_tb = ws; ws = align_up(ws + tmp_bytes, 256);
        }
    }
    size_t o_sla = 0, o_slb = 0, o_pout = 0, slice_bytes = 0;
    if (dtype == FMM_F64_OZAKI) {
        slice_bytes = (size_t)Rt * (size_t)oz_s * (size_t)pl->oz_Mp * (size_t)pl->oz_Mp;
        o_sla = ws; ws = align_up(ws + slice_bytes, 256);
        o_slb = ws; ws = align_up(ws + slice_bytes, 256);
        o_pout = ws; ws = align_up(ws + (size_t)Rt * (size_t)pl->m * (size_t)pl->m * sizeof(double), 256);
    }
    size_t o_pbuf = 0, o_xbuf = 0;
    if (build_levels) {
        // pass k reads pass k-1's output (pass 0: the products) and writes the intermediate
        // buffer (even k) or the product buffer (odd k); the last pass writes C
        const size_t blk = (size_t)pl->m * (size_t)pl->m * sizeof(double);
        size_t xblocks = 0;
        for (size_t k = 0; k + 1 < lpasses.size(); k += 2) {
            const fmm::LevelPass &a = lpasses[k];
            xblocks = std::max(xblocks, (size_t)a.np * a.qa * a.qb * a.ns);
        }
        if (post_levels) { o_pbuf = ws; ws = align_up(ws + (size_t)Rt * blk, 256); }  // the emulated leaf's: d_pout
        if (xblocks) { o_xbuf = ws; ws = align_up(ws + xblocks * blk, 256); }
    }
    pl->ws_bytes = ws;
    if (dev_alloc(&pl->d_ws, ws) != cudaSuccess) {
        free_plan_memory(pl);
        host_delete(pl);
        return FMM_ERR_OOM;
    }
    char *wsb = (char *)pl->d_ws;
    pl->d_error = (int *)wsb;
    pl->d_task_counter = (unsigned long long *)(wsb + 8);
    pl->d_task_counter2 = (unsigned long long *)(wsb + 16);
    pl->d_chain = (unsigned *)(wsb + 32);
    if (mat > 0) {
        pl->d_SA = (double *)(wsb + o_sa);
        pl->d_SB = (double *)(wsb + o_sb);
        if (o_ta) {
            pl->d_TA = (double *)(wsb + o_ta);
            pl->d_TB = (double *)(wsb + o_tb);
        }
    }
    pl->d_xbuf = o_xbuf ? (double *)(wsb + o_xbuf) : nullptr;
    if (post_levels) {
        pl->d_pbuf = (double *)(wsb + o_pbuf);
        F64Geom gl = g;  // border and core tasks, products stored
        gl.pout = pl->d_pbuf;
        gl.tasks_rankq = 0;
        F64Geom gq = g;  // the rank-q tasks alone, after the passes
        gq.tasks_core = gq.tasks_right = gq.tasks_bottom = 0;
        gq.rankq_free = 1;
        pl->leaf_tasks = gl.tasks_core + gl.tasks_right + gl.tasks_bottom;
        pl->rq_tasks = gq.tasks_rankq;
        if (cudaMemcpy((void *)pl->d_geom_leaf, &gl, sizeof gl, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy((void *)pl->d_geom_rq, &gq, sizeof gq, cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            free_plan_memory(pl);
            host_delete(pl);
            return FMM_ERR_CUDA;
        }
    }
    if (dtype == FMM_F64_OZAKI) {
        pl->d_mxa = (int *)(wsb + o_mx);
        pl->d_mxb = pl->d_mxa + (size_t)Rt * pl->oz_Mp;
        pl->d_sla = (unsigned char *)(wsb + o_sla);
        pl->d_slb = (unsigned char *)(wsb + o_slb);
        pl->d_pout = (double *)(wsb + o_pout);
        pl->d_pbuf = pl->d_pout;  // the passes read the products from here
        // engine: CTA pairs (one pair per cluster) by default; FMM_OZAKI_ENGINE=tc1 (one CTA per
        // tile) or mma_sync
        const char *eng = std::getenv("FMM_OZAKI_ENGINE");
        const std::string es = eng ? eng : "";
        pl->oz_engine = es == "mma_sync" ? 0 : (es == "tc1" ? 1 : 2);
        // K pieces of the CTA-pair slice GEMM, about 1024 of K each, at most four.  Measured leaf times
        // for one / two / four pieces: K = 1024 2.51 / 2.66 / 3.10 ms (n = 4096, Strassen depth 2),
        // K = 2048 19.08 / 18.81 / 19.62 ms (n = 8192, depth 2; DRAM reads 57 % lower with two),
        // K = 4096 24.13 / 23.34 / 23.07 ms (n = 8192, depth 1)
        pl->oz_kparts = (int)std::max<int64_t>(1, std::min<int64_t>(4, pl->oz_Mp / 1024));
        if (const char *kp = std::getenv("FMM_OZAKI_KPARTS")) pl->oz_kparts = std::max(1, std::min(8, std::atoi(kp)));
        if (pl->oz_engine == 2 && fmm::ozaki_tc_max_pairs() < 1) pl->oz_engine = 1;
        const unsigned long long srows = (unsigned long long)Rt * oz_s * pl->oz_Mp;
        if (pl->oz_engine >= 1 && (!make_slice_map(&pl->oz_map_a, pl->d_sla, srows, pl->oz_Mp) ||
                                   !make_slice_map(&pl->oz_map_b, pl->d_slb, srows, pl->oz_Mp) ||
                                   !make_slice_map(&pl->oz_map_bh, pl->d_slb, srows, pl->oz_Mp, 64))) {
            free_plan_memory(pl);
            host_delete(pl);
            return FMM_ERR_CUDA;
        }
        // padding rows/columns of the slices are never written by the kernels
        if (cudaMemset(pl->d_sla, 0, slice_bytes) != cudaSuccess || cudaMemset(pl->d_slb, 0, slice_bytes) != cudaSuccess) {
            cudaGetLastError();
            free_plan_memory(pl);
            host_delete(pl);
            return FMM_ERR_CUDA;
        }
    }
    if (cudaMemset(pl->d_ws, 0, pl->counters_bytes) != cudaSuccess) {
        cudaGetLastError();
        free_plan_memory(pl);
        host_delete(pl);
        return FMM_ERR_CUDA;
    }

    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, pl->device);
    const int per_sm = dtype == FMM_F64_OZAKI ? fmm::ozaki_ctas_per_sm() : fmm::f64_kernel_ctas_per_sm(pl->bn);
    if (per_sm <= 0 || fmm::f64_kernel_ctas_per_sm(pl->bn) <= 0) {
        cudaGetLastError();
        free_plan_memory(pl);
        host_delete(pl);
        return FMM_ERR_CUDA;
    }
    pl->grid = (int)std::min<long long>(pl->total_tasks, (long long)sms * per_sm);
    if (pl->grid < 1) pl->grid = 1;
    pl->sms = sms;
    if (o.record_kernel_time) {
        for (auto &e : pl->ev)
            if (cudaEventCreate(&e) != cudaSuccess) {
                cudaGetLastError();
                free_plan_memory(pl);
                host_delete(pl);
                return FMM_ERR_CUDA;
            }
    }
    *out = pl;
    return FMM_OK;
}

}  // namespace

namespace {

// FMM_LOG: 0 (default) silent; 1 one line per plan created or rejected; 2 also one line per multiplication
// enqueued.  Read on every use, so a process can change it between calls.
int log_level() {
    const char *e = std::getenv("FMM_LOG");
    return e ? std::atoi(e) : 0;
}

const char *dtype_name(fmm_dtype_t d) {
    switch (d) {
        case FMM_F64: return "f64";
        case FMM_F64_OZAKI: return "f64_ozaki";
        case FMM_C128: return "c128";
        case FMM_C128_3M: return "c128_3m";
        case FMM_F32: return "f32";
    }
    return "?";
}

fmm_status_t log_plan(const char *what, fmm_status_t st, const fmm_plan_t *pl, int64_t n, const fmm_algo_t *algo,
                      int depth, fmm_dtype_t dtype) {
    if (log_level() < 1) return st;
    if (st != FMM_OK) {
        std::fprintf(stderr, "fmm: %s rejected n=%lld p=%d R=%d depth=%d dtype=%s: %s\n", what, (long long)n,
                     algo ? algo->p : 0, algo ? algo->R : 0, depth, dtype_name(dtype), fmm_status_string(st));
        return st;
    }
    fmm_plan_info_t in{};
    fmm_plan_get_info(pl, &in);
    std::fprintf(stderr,
                 "fmm: %s n=%lld p=%d R=%d depth=%d dtype=%s leaf=%lld products=%lld..%lld materialized=%d "
                 "passes=%d tile_n=%d tasks=%lld slices=%d workspace=%.1f MB\n",
                 what, (long long)n, in.p, algo->R, depth, dtype_name(dtype), (long long)in.m,
                 (long long)in.product_begin, (long long)in.product_end, in.materialized_levels,
                 in.materialize_passes, in.tile_n, (long long)in.tasks, in.ozaki_slices,
                 (double)in.workspace_bytes / 1048576.0);
    return st;
}

}  // namespace

extern "C" fmm_status_t fmm_plan_create_ex(fmm_plan_t **out, int64_t n, const fmm_algo_t *algo, int depth,
                                           fmm_dtype_t dtype, const fmm_plan_options_t *opts) {
    const fmm_status_t st = plan_create(out, n, algo, depth, dtype, opts, 1);
    return log_plan("fmm_plan_create", st, st == FMM_OK ? *out : nullptr, n, algo, depth, dtype);
}

extern "C" fmm_status_t fmm_plan_create(fmm_plan_t **out, int64_t n, const fmm_algo_t *algo, int depth,
                                        fmm_dtype_t dtype) {
    return fmm_plan_create_ex(out, n, algo, depth, dtype, nullptr);
}

extern "C" fmm_status_t fmm_plan_create_rational(fmm_plan_t **out, int64_t n, const fmm_algo_rational_t *algo,
                                                 int depth, fmm_dtype_t dtype, const fmm_plan_options_t *opts) {
    if (!out) return FMM_ERR_INVALID;
    *out = nullptr;
    const int64_t bad = fmm_algo_rational_brent_mismatches(algo);
    if (bad != 0) {
        const fmm_algo_t shape{algo ? algo->p : 0, algo ? algo->R : 0, nullptr, nullptr, nullptr};
        return log_plan("fmm_plan_create_rational", bad < 0 ? FMM_ERR_INVALID : FMM_ERR_BRENT, nullptr, n, &shape,
                        depth, dtype);
    }
    const fmm_algo_t num{algo->p, algo->R, algo->U, algo->V, algo->W};
    const fmm_status_t st =
        plan_create(out, n, &num, depth, dtype, opts, (int64_t)algo->den_u * algo->den_v * algo->den_w);
    return log_plan("fmm_plan_create_rational", st, st == FMM_OK ? *out : nullptr, n, &num, depth, dtype);
}

namespace {

const F64Geom *dev_geom(const fmm_plan *pl) { return (const F64Geom *)pl->d_tables; }

// Enqueues the counter reset and the materialization pass of one plan.
fmm_status_t prepare(const fmm_plan *pl, const double *A, const double *B, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(pl->d_ws, 0, pl->counters_bytes, st);
    if (e != cudaSuccess) return FMM_ERR_CUDA;
    if (pl->poison) {
        e = cudaMemsetAsync(pl->d_chain, 0xFF, sizeof(unsigned), st);
        if (e != cudaSuccess) return FMM_ERR_CUDA;
    }
    // Pass g (one step, or two steps fused) reads pass g-1's output (pass 0 =
    // the n_core x n_core corner of the operand, ld n) and writes R times as
    // many matrices of side 1/p per step; the last pass lands in d_SA / d_SB,
    // earlier ones alternate with d_TA / d_TB.
    const int K = (int)pl->mat_steps.size();
    int G = 0;
    for (int k = 0; k < K; ++k) G += pl->mat_steps[k].with_next ? 0 : 1;
    for (int side = 0; side < 2; ++side) {
        // the host-buffer path copies B on its own stream while A's passes run
        if (side == 1 && pl->b_ready && cudaStreamWaitEvent(st, pl->b_ready, 0) != cudaSuccess) return FMM_ERR_CUDA;
        const double *src = side == 0 ? A : B;
        double *fin = side == 0 ? pl->d_SA : pl->d_SB;
        double *tmp = side == 0 ? pl->d_TA : pl->d_TB;
        long long ld_in = pl->n, b_in = pl->n_core, n_in = 1;
        int g = 0;
        for (int k = 0; k < K; ++k) {
            const fmm_plan::MatStep &ms = pl->mat_steps[k];
            ++g;
            double *dst = ((G - g) % 2 == 0) ? fin : tmp;
            const long long in_stride = (g == 1) ? 0 : b_in * b_in;
            if (ms.with_next) {
                const fmm_plan::MatStep &m2 = pl->mat_steps[k + 1];
                const long long b_out = b_in / 4;
                const bool unit = side == 0 ? ms.unit_u && m2.unit_u : ms.unit_v && m2.unit_v;
                e = fmm::launch_materialize_two_steps(src, ld_in, in_stride, (int)n_in, b_out, ms.R,
                                                      side == 0 ? ms.uptr : ms.vptr, side == 0 ? ms.uent : ms.vent,
                                                      m2.R, side == 0 ? m2.uptr : m2.vptr,
                                                      side == 0 ? m2.uent : m2.vent, unit, dst, st);
                n_in *= (long long)ms.R * m2.R;
                b_in = b_out;
                ++k;
            } else {
                const long long b_out = b_in / ms.p;
                e = fmm::launch_materialize_level(src, ld_in, in_stride, (int)n_in, b_out, ms.p, ms.R,
                                                  side == 0 ? ms.uptr : ms.vptr, side == 0 ? ms.uent : ms.vent,
                                                  side == 0 ? ms.unit_u : ms.unit_v, dst, st);
                n_in *= ms.R;
                b_in = b_out;
            }
            if (e != cudaSuccess) return FMM_ERR_CUDA;
            src = dst;
            ld_in = b_in;
        }
    }
    return FMM_OK;
}

F64Problem problem_of(const fmm_plan *pl, const double *A, const double *B, double *C, long long begin,
                      double alpha = 1.0, double beta = 0.0) {
    F64Problem pr{};
    pr.g = dev_geom(pl);
    pr.A = A; pr.B = B; pr.C = C;
    pr.alpha = alpha * pl->wscale;
    pr.alpha_peel = alpha;
    pr.beta = beta;
    pr.SA = pl->mat_levels > 0 ? pl->d_SA : A;
    pr.SB = pl->mat_levels > 0 ? pl->d_SB : B;
    pr.chain = pl->d_chain;
    pr.task_begin = begin;
    return pr;
}

}  // namespace

namespace {

// The post-addition passes of a plan with stored leaf products, from its
// product buffer into C (C = alpha sum + beta C in the last pass).
fmm_status_t run_level_passes(const fmm_plan *pl, double *C, double alpha, double beta, cudaStream_t st) {
    const size_t npass = pl->level_passes.size();
    for (size_t k = 0; k < npass; ++k) {
        fmm::LevelPass a = pl->level_passes[k];
        a.in = k == 0 ? pl->d_pbuf : (k % 2 == 1 ? pl->d_xbuf : pl->d_pbuf);
        a.out = a.last ? C : (k % 2 == 0 ? pl->d_xbuf : pl->d_pbuf);
        a.ldc = pl->n;
        a.alpha = a.last ? alpha * pl->wscale : 1.0;
        a.beta = a.last ? beta : 0.0;
        if (fmm::launch_level_pass(a, st) != cudaSuccess) return FMM_ERR_CUDA;
    }
    return FMM_OK;
}

// Emulated leaf: FP64 pre-additions, exponents and slices of every S_r / T_r,
// the slice GEMM with fused post-additions, then the FP64 peel tasks.
fmm_status_t gemm_ozaki(const fmm_plan *pl, const double *A, const double *B, double *C, double alpha, double beta,
                        cudaStream_t st) {
    const long long m = pl->m;
    const int nmat = (int)pl->R_total;
    const double *S = pl->depth > 0 ? pl->d_SA : A;
    const double *T = pl->depth > 0 ? pl->d_SB : B;
    const long long ld = pl->depth > 0 ? m : pl->n;
    const long long stride = pl->depth > 0 ? m * m : 0;
    const int Mp = (int)pl->oz_Mp;
    if (fmm::launch_ozaki_slices(S, ld, stride, nmat, (int)m, (int)m, true, pl->d_mxa, Mp, pl->oz_s, Mp, Mp,
                                 pl->d_sla, st) != cudaSuccess ||
        fmm::launch_ozaki_slices(T, ld, stride, nmat, (int)m, (int)m, false, pl->d_mxb, Mp, pl->oz_s, Mp, Mp,
                                 pl->d_slb, st) != cudaSuccess)
        return FMM_ERR_CUDA;
    if (pl->ev[1] && cudaEventRecord(pl->ev[1], st) != cudaSuccess) return FMM_ERR_CUDA;
    fmm::OzParams P{};
    P.sa = pl->d_sla;
    P.sb = pl->d_slb;
    P.mxa = pl->d_mxa;
    P.mxb = pl->d_mxb;
    P.C = C;
    P.ldc = pl->n;
    P.pout = pl->d_pout;
    P.m = m;
    P.Mp = Mp;
    P.Kp = Mp;
    P.s = pl->oz_s;
    P.L = pl->oz_L;
    P.kparts = pl->oz_kparts;
    P.tiles_m = pl->tiles_m;
    P.tiles_n = pl->tiles_n;
    P.R = nmat;
    P.P = (int)pl->P;
    P.w_ptr = pl->geom.w_ptr;
    P.w_ent = pl->geom.w_ent;
    P.chain = pl->d_chain;
    P.tasks = (long long)nmat * pl->tiles_m * pl->tiles_n;
    P.task_counter = pl->d_task_counter;
    P.error = pl->d_error;
    P.timeout_ns = (long long)(pl->timeout_s * 1e9);
    P.alpha = alpha * pl->wscale;
    P.beta = beta;
    if (pl->oz_engine == 2) {
        // a task covers a pair of tile rows and two tile columns; the last row or column of a
        // task may be padding.  One CTA per SM, one pair per cluster.
        P.tasks = (long long)nmat * ((pl->tiles_m + 1) / 2) * ((pl->tiles_n + 1) / 2);
        const long long pairs = std::min<long long>(2 * P.tasks, (long long)fmm::ozaki_tc_max_pairs());
        const int ctas = (int)(2 * pairs);
        if (fmm::launch_ozaki_tc_pair(pl->oz_map_a, pl->oz_map_bh, P, ctas < 2 ? 2 : ctas, st) != cudaSuccess)
            return FMM_ERR_CUDA;
    } else if (pl->oz_engine == 1) {
        const int grid = (int)std::min<long long>(P.tasks, (long long)pl->sms);
        if (fmm::launch_ozaki_tc(pl->oz_map_a, pl->oz_map_b, P, grid < 1 ? 1 : grid, st) != cudaSuccess)
            return FMM_ERR_CUDA;
    } else {
        const int grid = (int)std::min<long long>(P.tasks, (long long)pl->sms * fmm::ozaki_ctas_per_sm());
        if (fmm::launch_ozaki_gemm(P, grid < 1 ? 1 : grid, st) != cudaSuccess) return FMM_ERR_CUDA;
    }
    if (pl->ev[2] && cudaEventRecord(pl->ev[2], st) != cudaSuccess) return FMM_ERR_CUDA;
    if (pl->oz_engine >= 1) {
        if (pl->oz_levels) {
            if (run_level_passes(pl, C, alpha, beta, st) != FMM_OK) return FMM_ERR_CUDA;
        } else if (fmm::launch_ozaki_postadd(pl->d_pout, m, (int)pl->P, pl->d_wl_ptr, pl->d_wl_ent, C, pl->n,
                                             alpha * pl->wscale, beta, st) != cudaSuccess) {
            return FMM_ERR_CUDA;
        }
    }
    if (pl->ev[5] && cudaEventRecord(pl->ev[5], st) != cudaSuccess) return FMM_ERR_CUDA;
    const long long peel = pl->geom.tasks_right + pl->geom.tasks_bottom + pl->geom.tasks_rankq;
    if (peel > 0) {
        F64Launch<1> L{};
        L.nprobs = 1;
        L.total_tasks = peel;
        L.task_counter = pl->d_task_counter2;
        L.error = pl->d_error;
        L.timeout_ns = (long long)(pl->timeout_s * 1e9);
        L.probs[0].g = pl->d_geom_peel;
        L.probs[0].A = A;
        L.probs[0].B = B;
        L.probs[0].SA = A;
        L.probs[0].SB = B;
        L.probs[0].C = C;
        L.probs[0].chain = pl->d_chain;
        L.probs[0].task_begin = 0;
        L.probs[0].alpha = alpha * pl->wscale;  // core tasks: none in this launch
        L.probs[0].alpha_peel = alpha;
        L.probs[0].beta = beta;
        const int g2 = (int)std::min<long long>(peel, (long long)pl->sms * fmm::f64_kernel_ctas_per_sm(pl->bn));
        if (fmm::launch_f64_single(L, g2 < 1 ? 1 : g2, st, pl->bn) != cudaSuccess) return FMM_ERR_CUDA;
    }
    return FMM_OK;
}

// Tasks of a plan in the (first) leaf launch of a call.
long long launch_tasks(const fmm_plan *pl) { return pl->post_levels ? pl->leaf_tasks : pl->total_tasks; }

// Stored leaf products: the leaf launch (border tasks, then every core task
// storing its P_r tile), the level-by-level post-addition passes into C, then
// the rank-q fix-ups of a non-divisible n, which add into C's core blocks.
fmm_status_t gemm_levels(const fmm_plan *pl, const double *A, const double *B, double *C, double alpha, double beta,
                         cudaStream_t st) {
    F64Launch<1> L{};
    L.nprobs = 1;
    L.total_tasks = pl->leaf_tasks;
    L.task_counter = pl->d_task_counter;
    L.error = pl->d_error;
    L.timeout_ns = (long long)(pl->timeout_s * 1e9);
    L.probs[0] = problem_of(pl, A, B, C, 0, alpha, beta);
    L.probs[0].g = pl->d_geom_leaf;
    const int per_sm = fmm::f64_kernel_ctas_per_sm(pl->bn);
    const int grid = (int)std::max<long long>(1, std::min<long long>(pl->leaf_tasks, (long long)pl->sms * per_sm));
    if (pl->leaf_tasks > 0 && fmm::launch_f64_single(L, grid, st, pl->bn) != cudaSuccess) return FMM_ERR_CUDA;
    if (pl->ev[2] && cudaEventRecord(pl->ev[2], st) != cudaSuccess) return FMM_ERR_CUDA;
    if (run_level_passes(pl, C, alpha, beta, st) != FMM_OK) return FMM_ERR_CUDA;
    if (pl->ev[5] && cudaEventRecord(pl->ev[5], st) != cudaSuccess) return FMM_ERR_CUDA;
    if (pl->rq_tasks > 0) {
        F64Launch<1> Q{};
        Q.nprobs = 1;
        Q.total_tasks = pl->rq_tasks;
        Q.task_counter = pl->d_task_counter2;
        Q.error = pl->d_error;
        Q.timeout_ns = L.timeout_ns;
        Q.probs[0] = L.probs[0];
        Q.probs[0].g = pl->d_geom_rq;
        const int g2 = (int)std::max<long long>(1, std::min<long long>(pl->rq_tasks, (long long)pl->sms * per_sm));
        if (fmm::launch_f64_single(Q, g2, st, pl->bn) != cudaSuccess) return FMM_ERR_CUDA;
    }
    if (pl->ev[4] && cudaEventRecord(pl->ev[4], st) != cudaSuccess) return FMM_ERR_CUDA;
    if (pl->ev[2]) const_cast<fmm_plan *>(pl)->timed_once = true;
    return FMM_OK;
}

// Double complex through real fast products on split planes (FMM_C128: four,
// FMM_C128_3M: three; see fmm_dtype_t).  The 4M form accumulates its second
// product of each part with beta = 1, so every part is one ordered sum.
fmm_status_t gemm_complex(const fmm_plan *pl, double alpha, const double *A, const double *B, double beta, double *C,
                          cudaStream_t st) {
    const long long N = pl->n * pl->n;
    double *P = pl->d_planes;
    const fmm_plan *in = pl->inner;
    if (pl->ev[0] && (cudaEventRecord(pl->ev[0], st) != cudaSuccess || cudaEventRecord(pl->ev[1], st) != cudaSuccess))
        return FMM_ERR_CUDA;
    fmm_status_t s = FMM_OK;
    if (pl->dtype == FMM_C128) {
        double *Ar = P, *Ai = P + N, *Br = P + 2 * N, *Bi = P + 3 * N, *Cr = P + 4 * N, *Ci = P + 5 * N;
        if (fmm::launch_split_complex(A, N, Ar, Ai, nullptr, st) != cudaSuccess ||
            fmm::launch_split_complex(B, N, Br, Bi, nullptr, st) != cudaSuccess ||
            (beta != 0.0 && fmm::launch_split_complex(C, N, Cr, Ci, nullptr, st) != cudaSuccess))
            return FMM_ERR_CUDA;
        if ((s = fmm_gemm_ex(in, alpha, Ar, Br, beta, Cr, st)) != FMM_OK) return s;
        if ((s = fmm_gemm_ex(in, -alpha, Ai, Bi, 1.0, Cr, st)) != FMM_OK) return s;
        if ((s = fmm_gemm_ex(in, alpha, Ar, Bi, beta, Ci, st)) != FMM_OK) return s;
        if ((s = fmm_gemm_ex(in, alpha, Ai, Br, 1.0, Ci, st)) != FMM_OK) return s;
        if (fmm::launch_join_complex(Cr, Ci, C, N, st) != cudaSuccess) return FMM_ERR_CUDA;
    } else {
        double *Ar = P, *Ai = P + N, *As = P + 2 * N, *Br = P + 3 * N, *Bi = P + 4 * N, *Bs = P + 5 * N;
        double *T1 = P + 6 * N, *T2 = P + 7 * N, *T3 = P + 8 * N;
        if (fmm::launch_split_complex(A, N, Ar, Ai, As, st) != cudaSuccess ||
            fmm::launch_split_complex(B, N, Br, Bi, Bs, st) != cudaSuccess)
            return FMM_ERR_CUDA;
        if ((s = fmm_gemm(in, Ar, Br, T1, st)) != FMM_OK) return s;
        if ((s = fmm_gemm(in, Ai, Bi, T2, st)) != FMM_OK) return s;
        if ((s = fmm_gemm(in, As, Bs, T3, st)) != FMM_OK) return s;
        if (fmm::launch_gauss_join(T1, T2, T3, C, N, alpha, beta, st) != cudaSuccess) return FMM_ERR_CUDA;
    }
    if (pl->ev[0]) {
        if (cudaEventRecord(pl->ev[2], st) != cudaSuccess) return FMM_ERR_CUDA;
        const_cast<fmm_plan *>(pl)->timed_once = true;
    }
    return FMM_OK;
}

}  // namespace

extern "C" fmm_status_t fmm_gemm(const fmm_plan_t *pl, const double *A, const double *B, double *C, void *stream) {
    return fmm_gemm_ex(pl, 1.0, A, B, 0.0, C, stream);
}

extern "C" fmm_status_t fmm_gemm_ex(const fmm_plan_t *pl, double alpha, const double *A, const double *B, double beta,
                                    double *C, void *stream) {
    if (!pl || !A || !B || !C || !std::isfinite(alpha) || !std::isfinite(beta)) return FMM_ERR_INVALID;
    if (pl->dtype == FMM_F32) return FMM_ERR_INVALID;  // binary32 operands go through fmm_gemm_f32_ex
    cudaStream_t st = (cudaStream_t)stream;
    const long long doubles = pl->n * pl->n * (pl->inner ? 2 : 1);
    if (pl->inner && ((((uintptr_t)A) | ((uintptr_t)B) | ((uintptr_t)C)) & 15) != 0) return FMM_ERR_INVALID;
    if (pl->shard_count > 1 && beta != 0.0) return FMM_ERR_UNSUPPORTED;
    if (log_level() >= 2)
        std::fprintf(stderr, "fmm: gemm n=%lld depth=%d dtype=%s alpha=%g beta=%g stream=%p\n", (long long)pl->n,
                     pl->depth, dtype_name(pl->dtype), alpha, beta, stream);
    if (alpha == 0.0) return cuda_status(fmm::launch_scale_c(C, doubles, beta, st));  // A, B unread
    if (pl->inner) return gemm_complex(pl, alpha, A, B, beta, C, st);
    if (pl->ev[0] && cudaEventRecord(pl->ev[0], st) != cudaSuccess) return FMM_ERR_CUDA;
    // a shard writes only the C blocks its products reach: the rest of its partial C is zero
    if (pl->shard_count > 1 && cudaMemsetAsync(C, 0, (size_t)doubles * sizeof(double), st) != cudaSuccess)
        return FMM_ERR_CUDA;
    fmm_status_t s = prepare(pl, A, B, st);
    if (s != FMM_OK) return s;
    if (pl->ev[3] && cudaEventRecord(pl->ev[3], st) != cudaSuccess) return FMM_ERR_CUDA;
    if (pl->dtype == FMM_F64_OZAKI) {
        s = gemm_ozaki(pl, A, B, C, alpha, beta, st);
        if (s == FMM_OK && pl->ev[4] && cudaEventRecord(pl->ev[4], st) != cudaSuccess) return FMM_ERR_CUDA;
        if (s == FMM_OK && pl->ev[2]) const_cast<fmm_plan *>(pl)->timed_once = true;
        return s;
    }
    if (pl->ev[1] && cudaEventRecord(pl->ev[1], st) != cudaSuccess) return FMM_ERR_CUDA;
    if (pl->post_levels) return gemm_levels(pl, A, B, C, alpha, beta, st);
    F64Launch<1> L{};
    L.nprobs = 1;
    L.total_tasks = pl->total_tasks;
    L.task_counter = pl->d_task_counter;
    L.error = pl->d_error;
    L.timeout_ns = (long long)(pl->timeout_s * 1e9);
    L.probs[0] = problem_of(pl, A, B, C, 0, alpha, beta);
    fmm_status_t ls = cuda_status(fmm::launch_f64_single(L, pl->grid, st, pl->bn));
    if (ls != FMM_OK) return ls;
    if (pl->ev[2]) {
        if (cudaEventRecord(pl->ev[2], st) != cudaSuccess) return FMM_ERR_CUDA;
        if (cudaEventRecord(pl->ev[5], st) != cudaSuccess) return FMM_ERR_CUDA;
        if (cudaEventRecord(pl->ev[4], st) != cudaSuccess) return FMM_ERR_CUDA;
        const_cast<fmm_plan *>(pl)->timed_once = true;
    }
    return FMM_OK;
}

extern "C" fmm_status_t fmm_gemm_f32_ex(const fmm_plan_t *pl, float alpha, const float *A, const float *B,
                                        float beta, float *C, void *stream) {
    if (!pl || !A || !B || !C || pl->dtype != FMM_F32 || !std::isfinite(alpha) || !std::isfinite(beta))
        return FMM_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    const long long N = pl->n * pl->n;
    if (alpha == 0.0f) return cuda_status(fmm::launch_scale_f32(C, N, beta, st));  // A, B unread
    double *Ad = pl->d_planes, *Bd = pl->d_planes + N, *Cd = pl->d_planes + 2 * N;
    if (pl->ev[0] && (cudaEventRecord(pl->ev[0], st) != cudaSuccess || cudaEventRecord(pl->ev[1], st) != cudaSuccess))
        return FMM_ERR_CUDA;
    if (fmm::launch_f32_to_f64(A, N, Ad, st) != cudaSuccess || fmm::launch_f32_to_f64(B, N, Bd, st) != cudaSuccess ||
        (beta != 0.0f && fmm::launch_f32_to_f64(C, N, Cd, st) != cudaSuccess))
        return FMM_ERR_CUDA;
    // binary32 scalars widen exactly; the product is formed in binary64 and rounded once
    fmm_status_t s = fmm_gemm_ex(pl->inner, (double)alpha, Ad, Bd, (double)beta, Cd, st);
    if (s != FMM_OK) return s;
    if (fmm::launch_f64_to_f32(Cd, N, C, st) != cudaSuccess) return FMM_ERR_CUDA;
    if (pl->ev[0]) {
        if (cudaEventRecord(pl->ev[2], st) != cudaSuccess) return FMM_ERR_CUDA;
        const_cast<fmm_plan *>(pl)->timed_once = true;
    }
    return FMM_OK;
}

extern "C" fmm_status_t fmm_plan_last_phase_ms(const fmm_plan_t *pl, float *phases, int count) {
    if (!pl || !phases || count < 1 || !pl->ev[0] || !pl->timed_once || pl->inner) return FMM_ERR_INVALID;
    if (cudaEventSynchronize(pl->ev[4]) != cudaSuccess) return FMM_ERR_CUDA;
    // [0] counter reset + materialization, [1] slicing (emulated leaf), [2] leaf kernel, [3] peel tasks,
    // [4] separate post-additions (emulated leaf)
    const cudaEvent_t from[5] = {pl->ev[0], pl->ev[3], pl->ev[1], pl->ev[5], pl->ev[2]};
    const cudaEvent_t to[5] = {pl->ev[3], pl->ev[1], pl->ev[2], pl->ev[4], pl->ev[5]};
    for (int i = 0; i < count && i < 5; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, from[i], to[i]) != cudaSuccess) return FMM_ERR_CUDA;
        phases[i] = ms;
    }
    return FMM_OK;
}

extern "C" fmm_status_t fmm_plan_last_kernel_ms(const fmm_plan_t *pl, float *leaf_ms, float *total_ms) {
    if (!pl || !pl->ev[0] || !pl->timed_once) return FMM_ERR_INVALID;
    if (cudaEventSynchronize(pl->ev[2]) != cudaSuccess) return FMM_ERR_CUDA;
    float a = 0, b = 0;
    if (cudaEventElapsedTime(&a, pl->ev[1], pl->ev[2]) != cudaSuccess) return FMM_ERR_CUDA;
    if (cudaEventElapsedTime(&b, pl->ev[0], pl->ev[2]) != cudaSuccess) return FMM_ERR_CUDA;
    if (leaf_ms) *leaf_ms = a;
    if (total_ms) *total_ms = b;
    return FMM_OK;
}

extern "C" fmm_status_t fmm_gemm_host(fmm_plan_t *pl, const double *hA, const double *hB, double *hC, void *stream) {
    if (!pl || !hA || !hB || !hC) return FMM_ERR_INVALID;
    const size_t elem = pl->dtype == FMM_F32 ? sizeof(float) : sizeof(double) * (pl->inner ? 2 : 1);
    const size_t bytes = (size_t)pl->n * (size_t)pl->n * elem;
    if (!pl->d_hostA) {
        if (dev_alloc(&pl->d_hostA, bytes) != cudaSuccess || dev_alloc(&pl->d_hostB, bytes) != cudaSuccess ||
            dev_alloc(&pl->d_hostC, bytes) != cudaSuccess) {
            dev_free(pl->d_hostA);
            dev_free(pl->d_hostB);
            dev_free(pl->d_hostC);
            pl->d_hostA = pl->d_hostB = pl->d_hostC = nullptr;
            return FMM_ERR_OOM;
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    const bool overlap = pl->dtype == FMM_F64 || pl->dtype == FMM_F64_OZAKI;
    if (overlap && !pl->host_copy_stream) {
        if (cudaStreamCreateWithFlags(&pl->host_copy_stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&pl->host_ev[0], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&pl->host_ev[1], cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return FMM_ERR_CUDA;
        }
    }
    fmm_status_t s = FMM_OK;
    if (overlap) {
        // A on the call's stream; B on the plan's copy stream once the work already queued on `stream`
        // is done, so that (for page-locked sources, whose copies return at once) A's pre-addition
        // passes run while B is still in flight; B's own passes wait for its copy
        cudaStream_t cs = pl->host_copy_stream;
        if (cudaEventRecord(pl->host_ev[0], st) != cudaSuccess || cudaStreamWaitEvent(cs, pl->host_ev[0], 0) != cudaSuccess ||
            cudaMemcpyAsync(pl->d_hostA, hA, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(pl->d_hostB, hB, bytes, cudaMemcpyHostToDevice, cs) != cudaSuccess ||
            cudaEventRecord(pl->host_ev[1], cs) != cudaSuccess)
            return FMM_ERR_CUDA;
        pl->b_ready = pl->host_ev[1];
        s = fmm_gemm(pl, pl->d_hostA, pl->d_hostB, pl->d_hostC, stream);
        pl->b_ready = nullptr;
        // a launch that failed before B's passes leaves the copy unwaited: order it before C's copy
        if (s != FMM_OK) {
            cudaStreamWaitEvent(st, pl->host_ev[1], 0);
            cudaStreamSynchronize(st);
            return s;
        }
    } else {
        if (cudaMemcpyAsync(pl->d_hostA, hA, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) return FMM_ERR_CUDA;
        if (cudaMemcpyAsync(pl->d_hostB, hB, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) return FMM_ERR_CUDA;
        s = pl->dtype == FMM_F32
                ? fmm_gemm_f32_ex(pl, 1.0f, reinterpret_cast<const float *>(pl->d_hostA),
                                  reinterpret_cast<const float *>(pl->d_hostB), 0.0f,
                                  reinterpret_cast<float *>(pl->d_hostC), stream)
                : fmm_gemm(pl, pl->d_hostA, pl->d_hostB, pl->d_hostC, stream);
        if (s != FMM_OK) return s;
    }
    if (cudaMemcpyAsync(hC, pl->d_hostC, bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess) return FMM_ERR_CUDA;
    return cuda_status(cudaStreamSynchronize(st));
}

extern "C" fmm_status_t fmm_gemm_batched(fmm_plan_t *const *plans, const double *const *A, const double *const *B,
                                         double *const *C, int count, void *stream) {
    return fmm_gemm_batched_ex(plans, nullptr, A, B, nullptr, C, count, stream);
}

extern "C" fmm_status_t fmm_gemm_batched_ex(fmm_plan_t *const *plans, const double *alpha, const double *const *A,
                                            const double *const *B, const double *beta, double *const *C, int count,
                                            void *stream) {
    if (count < 0 || (count > 0 && (!plans || !A || !B || !C))) return FMM_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    for (int i = 0; i < count; ++i) {
        if (!plans[i] || !A[i] || !B[i] || !C[i] || plans[i]->dtype != FMM_F64 || plans[i]->shard_count > 1)
            return FMM_ERR_INVALID;
        if ((alpha && !std::isfinite(alpha[i])) || (beta && !std::isfinite(beta[i]))) return FMM_ERR_INVALID;
        for (int j = 0; j < i; ++j)
            if (plans[j] == plans[i]) return FMM_ERR_INVALID;  // a plan's counters serve one product
    }
    const auto al = [&](int i) { return alpha ? alpha[i] : 1.0; };
    const auto be = [&](int i) { return beta ? beta[i] : 0.0; };
    // problems with alpha = 0 only scale C (A and B unread); they join no launch
    for (int i = 0; i < count; ++i)
        if (al(i) == 0.0 && fmm::launch_scale_c(C[i], plans[i]->n * plans[i]->n, be(i), st) != cudaSuccess)
            return FMM_ERR_CUDA;
    // one grouped launch per tile width present in the batch
    for (int bn : {128, 64}) {
        std::vector<int> sel;
        for (int i = 0; i < count; ++i)
            if (plans[i]->bn == bn && al(i) != 0.0) sel.push_back(i);
        for (size_t c0 = 0; c0 < sel.size(); c0 += fmm::kMaxBatchPerLaunch) {
            const int cnt = (int)std::min<size_t>(sel.size() - c0, fmm::kMaxBatchPerLaunch);
            F64Launch<fmm::kMaxBatchPerLaunch> *L = host_new<F64Launch<fmm::kMaxBatchPerLaunch>>();
            if (!L) return FMM_ERR_OOM;
            long long begin = 0;
            for (int k = 0; k < cnt; ++k) {
                const int i = sel[c0 + k];
                const fmm_plan *pl = plans[i];
                fmm_status_t s = prepare(pl, A[i], B[i], st);
                if (s != FMM_OK) { host_delete(L); return s; }
                L->probs[k] = problem_of(pl, A[i], B[i], C[i], begin, al(i), be(i));
                if (pl->post_levels) L->probs[k].g = pl->d_geom_leaf;  // border and core tasks, P_r stored
                begin += launch_tasks(pl);
            }
            const fmm_plan *lead = plans[sel[c0]];
            L->nprobs = cnt;
            L->total_tasks = begin;
            L->task_counter = lead->d_task_counter;
            L->error = lead->d_error;
            L->timeout_ns = (long long)(lead->timeout_s * 1e9);
            if (cnt > 1) {
                // interleaved order: problems by task count, descending, round-robin
                std::vector<int> idx(cnt);
                for (int k = 0; k < cnt; ++k) idx[k] = k;
                std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) {
                    return launch_tasks(plans[sel[c0 + x]]) > launch_tasks(plans[sel[c0 + y]]);
                });
                std::vector<long long> c(cnt + 1, 0);
                for (int j = 0; j < cnt; ++j) {
                    c[j] = launch_tasks(plans[sel[c0 + idx[j]]]);
                    L->order[j] = (short)idx[j];
                }
                long long G = 0;
                for (int q = cnt; q >= 1; --q) {  // segment with q active problems
                    L->seg_start[q - 1] = G;
                    L->seg_round[q - 1] = (int)c[q];
                    G += (long long)q * (c[q - 1] - c[q]);
                }
                L->interleave = 1;
            }
            int sms = 0;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, lead->device);
            int grid = (int)std::min<long long>(begin, (long long)sms * fmm::f64_kernel_ctas_per_sm(bn));
            if (grid < 1) grid = 1;
            cudaError_t e = fmm::launch_f64_batch(*L, grid, st, bn);
            host_delete(L);
            if (e != cudaSuccess) return FMM_ERR_CUDA;
        }
    }
    // plans with stored leaf products: their post-addition passes, then one grouped launch per tile
    // width of their rank-q fix-ups
    for (int i = 0; i < count; ++i)
        if (plans[i]->post_levels && al(i) != 0.0 && run_level_passes(plans[i], C[i], al(i), be(i), st) != FMM_OK)
            return FMM_ERR_CUDA;
    for (int bn : {128, 64}) {
        std::vector<int> sel;
        for (int i = 0; i < count; ++i)
            if (plans[i]->bn == bn && al(i) != 0.0 && plans[i]->post_levels && plans[i]->rq_tasks > 0)
                sel.push_back(i);
        for (size_t c0 = 0; c0 < sel.size(); c0 += fmm::kMaxBatchPerLaunch) {
            const int cnt = (int)std::min<size_t>(sel.size() - c0, fmm::kMaxBatchPerLaunch);
            F64Launch<fmm::kMaxBatchPerLaunch> *L = host_new<F64Launch<fmm::kMaxBatchPerLaunch>>();
            if (!L) return FMM_ERR_OOM;
            long long begin = 0;
            for (int k = 0; k < cnt; ++k) {
                const int i = sel[c0 + k];
                L->probs[k] = problem_of(plans[i], A[i], B[i], C[i], begin, al(i), be(i));
                L->probs[k].g = plans[i]->d_geom_rq;
                begin += plans[i]->rq_tasks;
            }
            const fmm_plan *lead = plans[sel[c0]];
            L->nprobs = cnt;
            L->total_tasks = begin;
            L->task_counter = lead->d_task_counter2;
            L->error = lead->d_error;
            L->timeout_ns = (long long)(lead->timeout_s * 1e9);
            int sms = 0;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, lead->device);
            const int grid = (int)std::max<long long>(
                1, std::min<long long>(begin, (long long)sms * fmm::f64_kernel_ctas_per_sm(bn)));
            cudaError_t e = fmm::launch_f64_batch(*L, grid, st, bn);
            host_delete(L);
            if (e != cudaSuccess) return FMM_ERR_CUDA;
        }
    }
    return FMM_OK;
}

struct fmm_batch_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

extern "C" fmm_status_t fmm_batch_graph_create(fmm_batch_graph_t **out, fmm_plan_t *const *plans,
                                               const double *const *A, const double *const *B, double *const *C,
                                               int count) {
    if (!out || count < 1) return FMM_ERR_INVALID;
    *out = nullptr;
    // kernel attributes are set outside the capture
    if (fmm::f64_kernel_ctas_per_sm(128) <= 0 || fmm::f64_kernel_ctas_per_sm(64) <= 0) return FMM_ERR_CUDA;
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return FMM_ERR_CUDA;
    fmm_batch_graph *g = host_new<fmm_batch_graph>();
    if (!g) {
        cudaStreamDestroy(cs);
        return FMM_ERR_OOM;
    }
    fmm_status_t st = FMM_OK;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        st = FMM_ERR_CUDA;
    } else {
        st = fmm_gemm_batched(plans, A, B, C, count, (void *)cs);
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(cs, &graph);
        if (st == FMM_OK && e != cudaSuccess) st = FMM_ERR_CUDA;
        g->graph = graph;
        if (st == FMM_OK && cudaGraphInstantiate(&g->exec, graph, 0) != cudaSuccess) st = FMM_ERR_CUDA;
    }
    cudaStreamDestroy(cs);
    if (st != FMM_OK) {
        cudaGetLastError();
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->graph) cudaGraphDestroy(g->graph);
        host_delete(g);
        return st;
    }
    *out = g;
    return FMM_OK;
}

extern "C" fmm_status_t fmm_batch_graph_launch(const fmm_batch_graph_t *g, void *stream) {
    if (!g || !g->exec) return FMM_ERR_INVALID;
    return cuda_status(cudaGraphLaunch(g->exec, (cudaStream_t)stream));
}

extern "C" void fmm_batch_graph_destroy(fmm_batch_graph_t *g) {
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    host_delete(g);
}

namespace {

__global__ void fill_kernel(double *x, long long count, unsigned long long seed) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        unsigned long long z = seed + (unsigned long long)(i + 1) * 0x9E3779B97F4A7C15ULL;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        z ^= z >> 31;
        x[i] = (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
    }
}

}  // namespace

extern "C" fmm_status_t fmm_autotune(int64_t n, const fmm_algo_t *const *algos, int nalgos, int max_depth,
                                     int64_t min_leaf, int reps, void *stream, fmm_tune_result_t *best) {
    if (n < 1 || !algos || nalgos < 1 || max_depth < 0 || !best || min_leaf < 1) return FMM_ERR_INVALID;
    if (reps < 1) reps = 5;
    if (reps > 64) reps = 64;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)n * (size_t)n * sizeof(double);
    double *A = nullptr, *B = nullptr, *C = nullptr;
    if (dev_alloc(&A, bytes) != cudaSuccess || dev_alloc(&B, bytes) != cudaSuccess ||
        dev_alloc(&C, bytes) != cudaSuccess) {
        dev_free(A);
        dev_free(B);
        dev_free(C);
        return FMM_ERR_OOM;
    }
    fill_kernel<<<256, 256, 0, st>>>(A, (long long)n * n, 11);
    fill_kernel<<<256, 256, 0, st>>>(B, (long long)n * n, 12);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // the candidate list: (algorithm, depth, tile width, schedule); depth 0 once
    struct Cand { int ai, depth, tile; fmm_schedule_t sched; };
    std::vector<Cand> cands;
    const fmm_algo_t *first = nullptr;
    for (int ai = 0; ai < nalgos && !first; ++ai)
        if (algos[ai]) first = algos[ai];
    // FMM_FORCE_DEPTH=d keeps only the candidates of depth d (still searching algorithm, tile and schedule)
    const char *fd = std::getenv("FMM_FORCE_DEPTH");
    const int force = fd && *fd ? std::atoi(fd) : -1;
    if (force <= 0)
        for (int tile : {64, 128}) cands.push_back({0, 0, tile, FMM_SCHED_AUTO});
    for (int ai = 0; ai < nalgos && force != 0; ++ai) {
        if (!algo_shape_ok(algos[ai])) continue;
        for (int d = force > 0 ? force : 1; d <= (force > 0 ? force : max_depth); ++d) {
            long long P = 1;
            for (int k = 0; k < d; ++k) P *= algos[ai]->p;
            if (n / P < min_leaf) break;
            const bool both = d == 1 && default_materialized_levels(algos[ai]->p, algos[ai]->R, algos[ai], 1) > 0;
            for (int tile : {64, 128}) {
                cands.push_back({ai, d, tile, FMM_SCHED_AUTO});
                if (both) cands.push_back({ai, d, tile, FMM_SCHED_FUSED});
            }
        }
    }
    fmm_status_t result = FMM_ERR_INVALID;
    best->ms = 1e30;
    best->depth0_ms = 1e30;
    best->candidates = 0;
    for (const Cand &c : cands) {
        const fmm_algo_t *al = c.depth == 0 ? first : algos[c.ai];
        if (!al) continue;
        fmm_plan_options_t o{};
        o.schedule = c.sched;
        o.tile_n = c.tile;
        fmm_plan_t *pl = nullptr;
        const fmm_status_t cs = fmm_plan_create_ex(&pl, n, al, c.depth, FMM_F64, &o);
        if (cs == FMM_ERR_OOM) {
            result = FMM_ERR_OOM;
            break;
        }
        if (cs != FMM_OK) continue;
        std::vector<float> runs;
        bool ok = fmm_gemm(pl, A, B, C, st) == FMM_OK;  // warm-up
        for (int rep = 0; rep < reps && ok; ++rep) {
            float ms = 0.f;
            cudaEventRecord(e0, st);
            ok = fmm_gemm(pl, A, B, C, st) == FMM_OK;
            cudaEventRecord(e1, st);
            if (!(ok && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)) {
                ok = false;
                break;
            }
            runs.push_back(ms);
            if (rep == 0 && best->ms < 1e29 && ms > 1.5 * best->ms) break;  // clearly slower: pruned
        }
        ok = ok && fmm_sync_status(pl, stream) == FMM_OK;
        fmm_plan_destroy(pl);
        if (!ok || runs.empty()) continue;
        std::sort(runs.begin(), runs.end());
        const double med = runs[runs.size() / 2];
        ++best->candidates;
        if (c.depth == 0 && med < best->depth0_ms) best->depth0_ms = med;
        if (med < best->ms) {
            best->ms = med;
            best->algo_index = c.ai;
            best->depth = c.depth;
            best->tile_n = c.tile;
            best->schedule = c.sched;
            result = FMM_OK;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dev_free(A);
    dev_free(B);
    dev_free(C);
    if (cudaGetLastError() != cudaSuccess) return FMM_ERR_CUDA;
    return result;
}

extern "C" fmm_status_t fmm_sync_status(const fmm_plan_t *pl, void *stream) {
    if (!pl) return FMM_ERR_INVALID;
    if (pl->inner) return fmm_sync_status(pl->inner, stream);
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaStreamSynchronize(st) != cudaSuccess) return FMM_ERR_CUDA;
    int err = 0;
    if (cudaMemcpy(&err, pl->d_error, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return FMM_ERR_CUDA;
    if (err != fmm::kDevOk) {
        const int zero = 0;
        cudaMemcpy(pl->d_error, &zero, sizeof(int), cudaMemcpyHostToDevice);
        return FMM_ERR_TIMEOUT;
    }
    return FMM_OK;
}

extern "C" fmm_status_t fmm_plan_get_info(const fmm_plan_t *pl, fmm_plan_info_t *info) {
    if (!pl || !info) return FMM_ERR_INVALID;
    if (pl->inner) {
        // a complex plan: its real plan's figures times the number of real products, plus the
        // part sums and joins (4M: one add per element of each part; 3M: 2 n^2 sums, 3 n^2 joins)
        fmm_status_t s = fmm_plan_get_info(pl->inner, info);
        if (s != FMM_OK) return s;
        if (pl->dtype == FMM_F32) {  // one emulated product; the widening and rounding add no flops
            info->workspace_bytes += pl->ws_bytes;
            return FMM_OK;
        }
        const double k = pl->dtype == FMM_C128 ? 4.0 : 3.0;
        const double n2 = (double)pl->n * (double)pl->n;
        info->flops_leaf *= k;
        info->flops_executed = k * info->flops_executed + (pl->dtype == FMM_C128 ? 2.0 : 5.0) * n2;
        info->tasks = (int64_t)k * info->tasks;
        info->workspace_bytes += pl->ws_bytes;
        return FMM_OK;
    }
    info->n = pl->n;
    info->p = pl->p;
    info->depth = pl->depth;
    info->P = pl->P;
    info->R_total = pl->R_total;
    info->m = pl->m;
    info->n_core = pl->n_core;
    info->tasks = pl->total_tasks;
    info->materialized_levels = pl->mat_levels;
    info->flops_leaf = pl->flops_leaf;
    info->flops_executed = pl->flops_exec;
    info->workspace_bytes = pl->ws_bytes;
    info->ozaki_slices = pl->oz_s;
    info->tile_n = pl->bn;
    info->flops_lowp = pl->flops_lowp;
    info->coef_scale = pl->wscale;
    info->product_begin = pl->sub_begin * pl->R_src;
    info->product_end = pl->sub_end * pl->R_src;
    info->post_passes = pl->post_levels || pl->oz_levels ? (int)pl->level_passes.size() : 0;
    info->materialize_passes = 0;
    for (const fmm_plan::MatStep &ms : pl->mat_steps) info->materialize_passes += ms.with_next ? 0 : 1;
    return FMM_OK;
}

extern "C" fmm_status_t fmm_measure_fp64_peak(void *stream, double *dmma, double *dfma) {
    return cuda_status(fmm::measure_fp64_peaks((cudaStream_t)stream, dmma, dfma));
}

extern "C" fmm_status_t fmm_measure_e4m3_peak(void *stream, double *tflops) {
    return cuda_status(fmm::measure_e4m3_peak((cudaStream_t)stream, tflops));
}

extern "C" size_t fmm_plan_workspace_bytes(const fmm_plan_t *pl) {
    return pl ? pl->ws_bytes + (pl->inner ? pl->inner->ws_bytes : 0) : 0;
}

extern "C" void fmm_plan_destroy(fmm_plan_t *pl) {
    if (!pl) return;
    free_plan_memory(pl);
    host_delete(pl);
}

extern "C" void fmm_debug_fail_allocation(int64_t k) { g_fail_countdown.store(k < 0 ? -1 : (long long)k); }

extern "C" int64_t fmm_debug_live_allocations(void) { return (int64_t)g_live_allocs.load(); }

extern "C" fmm_status_t fmm_host_alloc(void **out, size_t bytes) {
    if (!out) return FMM_ERR_INVALID;
    *out = nullptr;
    return pinned_alloc(out, bytes) == cudaSuccess ? FMM_OK : FMM_ERR_OOM;
}

extern "C" fmm_status_t fmm_host_free(void *p) {
    if (!p) return FMM_OK;
    return pinned_free(p) ? FMM_OK : FMM_ERR_INVALID;
}

extern "C" int64_t fmm_host_huge_page_bytes(void) { return (int64_t)huge_page_bytes(); }
