// FP64 leaf kernel of the fast-matrix-multiplication library (sm_103a).
//
// One persistent kernel serves the classic product (depth 0), every flattened
// bilinear algorithm, peeled sizes and grouped batches.  CTAs fetch tile tasks
// from a global counter in increasing order.  A core task computes one
// 128 x 128 (or 128 x 64) tile of a leaf product P_r = S_r T_r (Section 2, equation
// `strassen`):
//   * operand staging forms the S_r / T_r slab on the fly from the source
//     blocks named by column r of U and V (pre-additions fused into the
//     global -> register -> shared-memory staging; S_r and T_r never reach
//     HBM);
//   * the product runs on the FP64 tensor-core path, mma.sync m16n8k4 (DMMA),
//     with accumulators in registers;
//   * the epilogue applies C_l (+)= W[l][r] P_r for every nonzero of column r
//     of W (post-additions fused into the epilogue).  Contributions to one
//     (C block, tile) are applied in ascending r, ordered by a per-tile
//     counter, so results are deterministic; the first contributor stores
//     (adding beta C when beta != 0), the others read-modify-write.  With
//     alpha != 1 every coefficient is scaled by alpha (C = alpha A B + beta C,
//     the BLAS form of Section 3's C = alpha A B).
// Every wait points at a task with a lower index, tasks are handed out in
// increasing order and only to running CTAs, so the lowest unfinished task can
// always proceed: no co-residency assumption is needed.  Each wait is also
// bounded in time; on expiry the kernel records kDevTimeout and drains.
#include <cuda_runtime.h>

#include "fmm_device.cuh"
#include "fmm_internal.h"

namespace fmm {
namespace {

// Tile configurations (template parameter BNT): BM = 128 rows by BNT = 128
// or 64 columns, NT = 2 * BNT threads (2 x BNT/32 warps, 4 x 4 m16 x n8
// sub-tiles each, interleaved over the tile).
// The 128-column tile runs one CTA per SM; the 64-column tile fits two, so
// one CTA's prologue and epilogue overlap the other's MMAs.
constexpr int BM = kBM, BK = kBK;
// Shared-memory row pitches (in doubles) chosen so that the m16n8k4 fragment
// reads are free of bank conflicts: A rows 20 doubles apart (8 banks of
// 4 bytes mod 32), B rows BNT + 4 apart (8 banks mod 32 for BNT = 64, 128).
constexpr int A_LD = BK + 4;

// Coefficients stay integers on the device: tests on them run on the integer
// pipe, and only coefficients other than +-1 are ever converted to FP64.
struct Src {
    const double *ptr;  // element (0, 0) of this source's part of the tile
    int coef;
    int pad;
};
struct Dst {
    double *ptr;        // element (0, 0) of the destination tile
    unsigned *chain;    // ordering counter, or nullptr for a single writer
    int coef;
    int pos;            // number of contributions that must precede this one
};

template <int BNT>
struct Smem {
    double a[2][BM * A_LD];
    double b[2][BK * (BNT + 4)];
    Src srcA[kMaxTerms];
    Src srcB[kMaxTerms];
    Dst dst[kMaxTerms];
    long long lda, ldb, ldc;
    long long task;
    double alpha, beta;  // C = alpha A B + beta C of the task's problem
    int nA, nB, nD;
    int rows, cols, K;
    int ok;
    int pick;
    unsigned char done[kMaxTerms];  // destinations of the current task already applied
};

using dev::chain_wait;
using dev::global_ns;
using dev::ld_volatile;
using dev::neg;

__device__ __forceinline__ long long lmin(long long a, long long b) { return a < b ? a : b; }

__device__ __forceinline__ void dmma_16x8x4(double (&d)[4], const double (&a)[2], double b) {
    asm volatile(
        "mma.sync.aligned.m16n8k4.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};"
        : "+d"(d[0]), "+d"(d[1]), "+d"(d[2]), "+d"(d[3])
        : "d"(a[0]), "d"(a[1]), "d"(b));
}

// Decodes task `local` of problem `pr` into the shared source / destination
// lists.  All threads run the index arithmetic; list entries are filled in
// parallel.
template <int BNT>
__device__ void setup_task(Smem<BNT> &S, const F64Problem &pr, const F64Geom &g, long long local) {
    constexpr int BN = BNT, NT = 2 * BNT;
    const int tid = threadIdx.x;
    const long long n = g.n, m = g.m, nc = g.n_core;
    const long long q = n - nc;
    // Task order: the border products first (K = n, the longest tasks, and independent of all others),
    // then the core products, then the rank-q updates, which wait for the core contributions to their
    // C block.  Started last, the border products left a tail of a few long tasks on few SMs.
    const long long border = g.tasks_right + g.tasks_bottom;
    if (local >= border && local - border < g.tasks_core) {
        local -= border;
        const int tiles = g.tiles_m * g.tiles_n;
        const long long per_sub = (long long)tiles * g.R_src;
        const int sub = g.sub_begin + (int)(local / per_sub);
        const long long rem = local - (long long)(sub - g.sub_begin) * per_sub;
        const int t = (int)(rem / g.R_src);
        const int r = (int)(rem - (long long)t * g.R_src);
        const int ti = t / g.tiles_n, tj = t - ti * g.tiles_n;
        const int rglob = sub * g.R_src + r;
        const double *SA = pr.SA + (long long)sub * g.sub_stride_a;
        const double *SB = pr.SB + (long long)sub * g.sub_stride_b;
        const int ua = g.u_ptr[r], nA = g.u_ptr[r + 1] - ua;
        const int vb = g.v_ptr[r], nB = g.v_ptr[r + 1] - vb;
        const int wc = g.w_ptr[rglob];
        // stored products: one destination, P_r itself (coefficient 1, alpha 1, beta 0)
        const int nD = g.pout != nullptr ? 1 : g.w_ptr[rglob + 1] - wc;
        for (int e = tid; e < nA; e += NT) {
            const int2 en = g.u_ent[ua + e];
            const long long br = en.x / g.P_src, bc = en.x % g.P_src;
            S.srcA[e].ptr = SA + (br * m + (long long)ti * BM) * g.ld_src_a + bc * m;
            S.srcA[e].coef = en.y;
        }
        for (int e = tid; e < nB; e += NT) {
            const int2 en = g.v_ent[vb + e];
            const long long br = en.x / g.P_src, bc = en.x % g.P_src;
            S.srcB[e].ptr = SB + (br * m) * g.ld_src_b + bc * m + (long long)tj * BN;
            S.srcB[e].coef = en.y;
        }
        if (g.pout != nullptr) {
            if (tid == 0) {
                S.dst[0].ptr = g.pout + (long long)rglob * (m * m) + (long long)ti * BM * m + (long long)tj * BN;
                S.dst[0].chain = nullptr;
                S.dst[0].coef = 1;
                S.dst[0].pos = 0;
                S.done[0] = 0;
                S.nA = nA; S.nB = nB; S.nD = 1;
                S.lda = g.ld_src_a; S.ldb = g.ld_src_b; S.ldc = m;
                S.rows = (int)lmin(BM, m - (long long)ti * BM);
                S.cols = (int)lmin(BN, m - (long long)tj * BN);
                S.K = (int)m;
                S.alpha = 1.0; S.beta = 0.0;
            }
            return;
        }
        for (int e = tid; e < nD; e += NT) {
            const int4 en = g.w_ent[wc + e];
            const long long br = en.x / g.P, bc = en.x % g.P;
            S.dst[e].ptr = pr.C + (br * m + (long long)ti * BM) * n + bc * m + (long long)tj * BN;
            S.dst[e].chain = pr.chain + (long long)en.x * tiles + t;
            S.dst[e].coef = en.y;
            S.dst[e].pos = en.z;
            S.done[e] = 0;
        }
        if (tid == 0) {
            S.nA = nA; S.nB = nB; S.nD = nD;
            S.lda = g.ld_src_a; S.ldb = g.ld_src_b; S.ldc = n;
            S.rows = (int)lmin(BM, m - (long long)ti * BM);
            S.cols = (int)lmin(BN, m - (long long)tj * BN);
            S.K = (int)m;
            S.alpha = pr.alpha; S.beta = pr.beta;
        }
        return;
    }
    if (local >= border) local -= g.tasks_core;
    if (tid != 0) return;
    S.alpha = pr.alpha_peel; S.beta = pr.beta;
    S.nA = S.nB = S.nD = 1;
    S.lda = n; S.ldb = n; S.ldc = n;
    S.srcA[0].coef = S.srcB[0].coef = 1;
    S.dst[0].coef = 1;
    S.done[0] = 0;
    if (local < g.tasks_right) {  // C[0:nc, nc:n] = A[0:nc, :] B[:, nc:n]
        const int bi = (int)(local / g.rb_tn), bj = (int)(local % g.rb_tn);
        S.srcA[0].ptr = pr.A + (long long)bi * BM * n;
        S.srcB[0].ptr = pr.B + nc + (long long)bj * BN;
        S.dst[0].ptr = pr.C + (long long)bi * BM * n + nc + (long long)bj * BN;
        S.dst[0].chain = nullptr; S.dst[0].pos = 0;
        S.rows = (int)lmin(BM, nc - (long long)bi * BM);
        S.cols = (int)lmin(BN, q - (long long)bj * BN);
        S.K = (int)n;
        return;
    }
    local -= g.tasks_right;
    if (local < g.tasks_bottom) {  // C[nc:n, :] = A[nc:n, :] B
        const int bi = (int)(local / g.bb_tn), bj = (int)(local % g.bb_tn);
        S.srcA[0].ptr = pr.A + (nc + (long long)bi * BM) * n;
        S.srcB[0].ptr = pr.B + (long long)bj * BN;
        S.dst[0].ptr = pr.C + (nc + (long long)bi * BM) * n + (long long)bj * BN;
        S.dst[0].chain = nullptr; S.dst[0].pos = 0;
        S.rows = (int)lmin(BM, q - (long long)bi * BM);
        S.cols = (int)lmin(BN, n - (long long)bj * BN);
        S.K = (int)n;
        return;
    }
    local -= g.tasks_bottom;
    {  // C[:nc, :nc] += A[:nc, nc:n] B[nc:n, :nc], tile t of block l, after every core contribution
        const int tiles = g.tiles_m * g.tiles_n;
        const int l = (int)(local / tiles), t = (int)(local % tiles);
        const int ti = t / g.tiles_n, tj = t - ti * g.tiles_n;
        const long long row0 = (long long)(l / g.P) * m + (long long)ti * BM;
        const long long col0 = (long long)(l % g.P) * m + (long long)tj * BN;
        S.srcA[0].ptr = pr.A + row0 * n + nc;
        S.srcB[0].ptr = pr.B + nc * n + col0;
        S.dst[0].ptr = pr.C + row0 * n + col0;
        S.dst[0].chain = g.rankq_free ? nullptr : pr.chain + (long long)l * tiles + t;
        S.dst[0].pos = g.w_row_nnz[l];  // > 0: added into C, after the core contributions
        S.rows = (int)lmin(BM, m - (long long)ti * BM);
        S.cols = (int)lmin(BN, m - (long long)tj * BN);
        S.K = (int)q;
    }
}

// Accumulates one source's 8 values into r[] with the coefficient's sign
// resolved once per source (uniform across the CTA, so no divergence).
template <int N>
__device__ __forceinline__ void accumulate(double (&r)[N], const double (&v)[N], int c, bool first) {
    if (first) {
        if (c == 1) {
#pragma unroll
            for (int j = 0; j < N; ++j) r[j] = v[j];
        } else if (c == -1) {
#pragma unroll
            for (int j = 0; j < N; ++j) r[j] = neg(v[j]);
        } else {
            const double cd = (double)c;
#pragma unroll
            for (int j = 0; j < N; ++j) r[j] = cd * v[j];
        }
    } else {
        if (c == 1) {
#pragma unroll
            for (int j = 0; j < N; ++j) r[j] += v[j];
        } else if (c == -1) {
#pragma unroll
            for (int j = 0; j < N; ++j) r[j] -= v[j];
        } else {
            const double cd = (double)c;
#pragma unroll
            for (int j = 0; j < N; ++j) r[j] = fma(cd, v[j], r[j]);
        }
    }
}

// Loads the K slab [kk, kk + BK) of both operands, combining the sources.
// A: thread column c = tid % 16, rows r0 + (NT/16) j; B: column tid % BNT,
// rows r0 + 2 j.
template <int BNT>
__device__ __forceinline__ void load_slab(const Smem<BNT> &S, int kk, double (&ra)[1024 / BNT],
                                          double (&rb)[8]) {
    constexpr int NT = 2 * BNT, AP = 2048 / NT, RS = NT / 16;
    const int tid = threadIdx.x;
    {
        const int c = tid & 15, r0 = tid >> 4;
        const bool kval = kk + c < S.K;
        const long long lda = S.lda;
        for (int e = 0; e < S.nA; ++e) {
            const double *p = S.srcA[e].ptr + kk + c;
            double v[AP];
#pragma unroll
            for (int j = 0; j < AP; ++j) {
                const int row = r0 + RS * j;
                v[j] = (kval && row < S.rows) ? __ldg(p + row * lda) : 0.0;
            }
            accumulate<AP>(ra, v, S.srcA[e].coef, e == 0);
        }
        if (S.nA == 0) {
#pragma unroll
            for (int j = 0; j < AP; ++j) ra[j] = 0.0;
        }
    }
    {
        const int c = tid & (BNT - 1), r0 = tid / BNT;
        const bool cval = c < S.cols;
        const long long ldb = S.ldb;
        for (int e = 0; e < S.nB; ++e) {
            const double *p = S.srcB[e].ptr + (long long)kk * ldb + c;
            double v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int row = r0 + 2 * j;
                v[j] = (cval && kk + row < S.K) ? __ldg(p + row * ldb) : 0.0;
            }
            accumulate<8>(rb, v, S.srcB[e].coef, e == 0);
        }
        if (S.nB == 0) {
#pragma unroll
            for (int j = 0; j < 8; ++j) rb[j] = 0.0;
        }
    }
}

template <int BNT>
__device__ __forceinline__ void store_slab(Smem<BNT> &S, int buf, const double (&ra)[1024 / BNT],
                                           const double (&rb)[8]) {
    constexpr int NT = 2 * BNT, AP = 2048 / NT, RS = NT / 16;
    const int tid = threadIdx.x;
    {
        const int c = tid & 15, r0 = tid >> 4;
#pragma unroll
        for (int j = 0; j < AP; ++j) S.a[buf][(r0 + RS * j) * A_LD + c] = ra[j];
    }
    {
        const int c = tid & (BNT - 1), r0 = tid / BNT;
#pragma unroll
        for (int j = 0; j < 8; ++j) S.b[buf][(r0 + 2 * j) * (BNT + 4) + c] = rb[j];
    }
}

// Warp tiling: the 128 x BNT tile is split into m16 x n8 sub-tiles, and warp
// (wm, wn) of the 2 x BNT/32 warps takes sub-tile rows i = 0..3 at 16 (2 i + wm)
// and columns j = 0..3 at 8 (BNT/32 j + wn), interleaved rather than as one
// 64 x 32 block, so that the valid part of a ragged tile (a leaf side that is
// not a multiple of the tile) is spread over all warps: the task takes as long
// as its busiest warp.
template <int BNT>
__device__ __forceinline__ int sub_row(int wm, int i) { return 16 * (2 * i + wm); }
template <int BNT>
__device__ __forceinline__ int sub_col(int wn, int j) { return 8 * ((BNT / 32) * j + wn); }

// One K slab of MMAs.  m16 x n8 sub-tiles that lie entirely outside the
// valid rows / columns of a ragged tile are skipped (row_ok / col_ok are
// uniform across the warp): the FP64 pipe is shared by the SM's warps, so the
// skipped work shortens the task instead of being computed on zeros.
template <int BNT>
__device__ __forceinline__ void mma_slab(const Smem<BNT> &S, int buf, double (&acc)[4][4][4], unsigned row_ok,
                                         unsigned col_ok) {
    constexpr int B_LD = BNT + 4;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int wm = warp & 1, wn = warp >> 1;  // 2 x BNT/32 warps, 4 x 4 interleaved sub-tiles each
    const double *As = S.a[buf];
    const double *Bs = S.b[buf];
#pragma unroll
    for (int kq = 0; kq < BK / 4; ++kq) {
        double af[4][2], bf[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int row = sub_row<BNT>(wm, i) + g;
            af[i][0] = As[row * A_LD + kq * 4 + t];
            af[i][1] = As[(row + 8) * A_LD + kq * 4 + t];
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) bf[j] = Bs[(kq * 4 + t) * B_LD + sub_col<BNT>(wn, j) + g];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (((row_ok >> i) & (col_ok >> j)) & 1u) dmma_16x8x4(acc[i][j], af[i], bf[j]);
    }
}

// Index of a destination of the current task that is not applied yet and
// whose ordering counter has reached its position (or -1 after a timeout or
// another CTA's error).  Destinations are applied in whatever order they
// become ready; each (C block, tile) still sees its contributions in
// ascending product order.  Called by one thread.
template <int BNT>
__device__ int pick_ready(const Smem<BNT> &S, int *error, long long timeout_ns) {
    const unsigned long long t0 = global_ns();
    unsigned sleep = 32;
    while (true) {
        for (int d = 0; d < S.nD; ++d) {
            if (S.done[d]) continue;
            const Dst &dst = S.dst[d];
            if (dst.chain == nullptr || dst.pos == 0 || dev::ld_acquire(dst.chain) == (unsigned)dst.pos) return d;
        }
        if (ld_volatile(error) != kDevOk) return -1;
        if ((long long)(global_ns() - t0) > timeout_ns) {
            atomicCAS(error, kDevOk, kDevTimeout);
            return -1;
        }
        __nanosleep(sleep);
        if (sleep < 256) sleep <<= 1;
    }
}

template <int MAXP, int BNT>
__global__ void __launch_bounds__(2 * BNT, 128 / BNT) fmm_f64_kernel(const __grid_constant__ F64Launch<MAXP> L) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<BNT> &S = *reinterpret_cast<Smem<BNT> *>(smem_raw);
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t4 = lane & 3;
    const int wm = warp & 1, wn = warp >> 1;

    while (true) {
        if (tid == 0) {
            long long tk = (long long)atomicAdd(L.task_counter, 1ull);
            if (ld_volatile(L.error) != kDevOk) tk = L.total_tasks;
            S.task = tk;
        }
        __syncthreads();
        const long long task = S.task;
        if (task >= L.total_tasks) break;
        int pi = 0;
        long long local = 0;
        if (L.interleave) {
            // seg_start[q - 1] (the first global index of the rounds with q
            // active problems) never increases with q; the segment holding
            // `task` is the smallest q with seg_start[q - 1] <= task.
            int lo = 1, hi = L.nprobs;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (L.seg_start[mid - 1] <= task) hi = mid; else lo = mid + 1;
            }
            const int q = lo;
            const long long o = task - L.seg_start[q - 1];
            local = L.seg_round[q - 1] + o / q;
            pi = L.order[(int)(o % q)];
        } else {
            while (pi + 1 < L.nprobs && L.probs[pi + 1].task_begin <= task) ++pi;
            local = task - L.probs[pi].task_begin;
        }
        const F64Problem &pr = L.probs[pi];
        setup_task(S, pr, *pr.g, local);
        __syncthreads();

        double acc[4][4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[i][j][v] = 0.0;

        const int K = S.K;
        const int nk = (K + BK - 1) / BK;
        unsigned row_ok = 0, col_ok = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            row_ok |= (unsigned)(sub_row<BNT>(wm, i) < S.rows) << i;
            col_ok |= (unsigned)(sub_col<BNT>(wn, i) < S.cols) << i;
        }
        double ra[1024 / BNT], rb[8];
        if (nk > 0) {
            load_slab(S, 0, ra, rb);
            store_slab(S, 0, ra, rb);
        }
        __syncthreads();
        for (int kt = 0; kt < nk; ++kt) {
            const bool more = kt + 1 < nk;
            if (more) load_slab(S, (kt + 1) * BK, ra, rb);
            mma_slab(S, kt & 1, acc, row_ok, col_ok);
            if (more) store_slab(S, (kt + 1) & 1, ra, rb);
            __syncthreads();
        }

        // Epilogue: coefficient-weighted stores into every destination tile.
        const int rows = S.rows, cols = S.cols;
        const long long ldc = S.ldc;
        for (int remaining = S.nD; remaining > 0; --remaining) {
            if (tid == 0) S.pick = pick_ready(S, L.error, L.timeout_ns);
            __syncthreads();
            const int d = S.pick;
            if (d < 0) break;
            const Dst dst = S.dst[d];
            const bool first = dst.pos == 0;
            const int cf = dst.coef;
            const double alpha = S.alpha, beta = S.beta;
            // Every read-modify-write term is one fma(w, v, o) with w = alpha * cf:
            // for w = +-1 it rounds exactly like o + v or o - v, so a single
            // FP64 operation per element replaces a per-mode choice (a mode
            // tested per element would let the compiler issue the add, the
            // subtract and the fma alike, on the FP64 pipe the leaf products
            // need).  The first contribution with beta = 0 stores w * v, a
            // sign flip (integer XOR) for w = +-1; it reads C only for
            // beta != 0 and scales it by beta.
            const double w = alpha * (double)cf;
            const bool unit = w == 1.0 || w == -1.0;
            const unsigned long long wsign = w < 0.0 ? 0x8000000000000000ull : 0ull;
            const bool load = !first || beta != 0.0;
            const bool scale_old = first && beta != 1.0;
            // mode: 0 store v with w's sign, 2 store w * v, 5 fma(w, v, o)
            const int mode = load ? 5 : (unit ? 0 : 2);
            // Column pairs (2 t4, 2 t4 + 1) are 16 bytes apart-aligned when the tile
            // start and ldc are even.  Read-modify-writes load a whole subtile row
            // (16 values) before the first store, so the loads overlap instead of
            // waiting for each other behind possibly aliasing stores.
            const bool pair_ok = ((((unsigned long long)dst.ptr) & 15ull) == 0) && ((ldc & 1) == 0);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                double o[4][2][2];
                if (load) {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const int row = sub_row<BNT>(wm, i) + g + 8 * h;
                            const int col = sub_col<BNT>(wn, j) + 2 * t4;
                            const double *p = dst.ptr + row * ldc + col;
                            o[j][h][0] = o[j][h][1] = 0.0;
                            if (row >= rows || col >= cols) continue;
                            if (pair_ok && col + 1 < cols) {
                                const double2 q = __ldcg(reinterpret_cast<const double2 *>(p));
                                o[j][h][0] = q.x;
                                o[j][h][1] = q.y;
                            } else {
                                o[j][h][0] = __ldcg(p);
                                if (col + 1 < cols) o[j][h][1] = __ldcg(p + 1);
                            }
                        }
                    if (scale_old) {
#pragma unroll
                        for (int j = 0; j < 4; ++j)
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                o[j][h][0] = beta * o[j][h][0];
                                o[j][h][1] = beta * o[j][h][1];
                            }
                    }
                }
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int row = sub_row<BNT>(wm, i) + g + 8 * h;
                        const int col = sub_col<BNT>(wn, j) + 2 * t4;
                        if (row >= rows || col >= cols) continue;
                        double *p = dst.ptr + row * ldc + col;
                        double out[2];
#pragma unroll
                        for (int c2 = 0; c2 < 2; ++c2) {
                            const double v = acc[i][j][2 * h + c2];
                            if (mode == 5)
                                out[c2] = fma(w, v, o[j][h][c2]);
                            else if (mode == 0)
                                out[c2] = __longlong_as_double(__double_as_longlong(v) ^ (long long)wsign);
                            else
                                out[c2] = w * v;
                        }
                        if (pair_ok && col + 1 < cols) {
                            *reinterpret_cast<double2 *>(p) = make_double2(out[0], out[1]);
                        } else {
                            p[0] = out[0];
                            if (col + 1 < cols) p[1] = out[1];
                        }
                    }
            }
            __syncthreads();
            if (tid == 0) {
                if (dst.chain != nullptr) {
                    __threadfence();
                    atomicAdd(dst.chain, 1u);
                }
                S.done[d] = 1;
            }
        }
        __syncthreads();
    }
}

}  // namespace

size_t f64_kernel_smem_bytes(int bn) { return bn == 64 ? sizeof(Smem<64>) : sizeof(Smem<128>); }

template <int MAXP, int BNT>
static cudaError_t launch_cfg(const F64Launch<MAXP> &L, int grid, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(fmm_f64_kernel<MAXP, BNT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sizeof(Smem<BNT>));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    fmm_f64_kernel<MAXP, BNT><<<grid, 2 * BNT, sizeof(Smem<BNT>), s>>>(L);
    return cudaGetLastError();
}

template <int BNT>
static int ctas_per_sm_cfg() {
    static int cached = -1;
    if (cached >= 0) return cached;
    if (cudaFuncSetAttribute(fmm_f64_kernel<1, BNT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(Smem<BNT>)) != cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fmm_f64_kernel<1, BNT>, 2 * BNT, sizeof(Smem<BNT>)) !=
        cudaSuccess)
        return 0;
    cached = nb;
    return nb;
}

int f64_kernel_ctas_per_sm(int bn) { return bn == 64 ? ctas_per_sm_cfg<64>() : ctas_per_sm_cfg<128>(); }

cudaError_t launch_f64_single(const F64Launch<1> &L, int grid, cudaStream_t s, int bn) {
    return bn == 64 ? launch_cfg<1, 64>(L, grid, s) : launch_cfg<1, 128>(L, grid, s);
}

cudaError_t launch_f64_batch(const F64Launch<kMaxBatchPerLaunch> &L, int grid, cudaStream_t s, int bn) {
    return bn == 64 ? launch_cfg<kMaxBatchPerLaunch, 64>(L, grid, s) : launch_cfg<kMaxBatchPerLaunch, 128>(L, grid, s);
}

}  // namespace fmm
