// Emulated-FP64 leaf products (Ozaki scheme) for the fast-matrix-multiplication
// library, sm_103a.
//
// The leaf products P_r = S_r T_r of a fully materialized plan (Section 2,
// equation `strassen`; S_r, T_r formed in FP64) are computed from low-
// precision slices on the tensor cores (Ozaki, Ogita, Oishi, Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59, 2012; the
// integer-slice form follows Ootomo, Ozaki, Yokota, IJHPCA 2024):
//
//  * every row i of S_r is scaled by a power of two 2^(E_i - 1) at least its
//    largest magnitude and rounded to a fixed-point integer Y with s*5 bits,
//    which is split exactly into s balanced base-32 digits d_1..d_s
//    (most significant first; d_1 in [-16, 16], the others in [-16, 15]) read
//    as bit fields of Y + 16 (32^s - 1) / 31; every column j of T_r likewise;
//    digits are stored as e4m3 bytes, which hold these integers exactly;
//  * for each diagonal g = t + u (2 <= g <= s + 1, the triangular truncation
//    of the slice expansion) the kernel accumulates
//    D_g = sum_{t+u=g} Shat_t That_u over the full K in FP32 on mma.sync
//    m16n8k32 e4m3 -- exact, since |D_g| <= s * K * 256 < 2^24 -- and folds
//    D_g into a per-element int64 fixed-point sum on the integer pipe;
//  * the epilogue converts the int64 sum to FP64 once, applies 2^(E_i + F_j
//    - 5(s+1) + L) and performs the FP64 post-additions C_l (+)= W[l][r] P_r in
//    ascending r, ordered by the same per-tile counters as the FP64 kernel.
// Slicing, folding and scaling use integer arithmetic; FP64 work is one
// conversion and one multiply per element of P_r plus the post-additions.
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include "fmm_device.cuh"
#include "fmm_internal.h"

namespace fmm {
namespace {

using dev::chain_wait;
using dev::ld_volatile;
using dev::neg;

constexpr int OB = kOzDigitBits;   // bits per digit
constexpr int BM = 128, BN = 128, BKB = 128;  // CTA tile and K slab (bytes = e4m3 elements)
constexpr int NT = 256;
constexpr int STAGES = 4;

struct Dst {
    double *ptr;
    unsigned *chain;
    int coef;
    int pos;
};

struct Smem {
    unsigned char a[STAGES][BM * BKB];
    unsigned char b[STAGES][BN * BKB];
    Dst dst[kMaxTerms];
    long long task;
    int nD;
    int ok;
};

__device__ __forceinline__ int biased_exponent(double x) {
    return (int)((unsigned long long)__double_as_longlong(x) >> 52) & 0x7FF;
}

// With bs = BS: round(x * 2^(bs - E)) as an integer with |result| < 2^(bs - 1), where every
// |x| of the row or column is below 2^(E - 1) (integer pipe only), halves
// rounded away from zero.  x = M 2^(ex - 1075) with the 53-bit significand M,
// so the value is M 2^sh with sh = ex - 1075 + bs - E; since ex <= E + 1021,
// sh <= bs - 54 = K.  With M pre-shifted by K (M 2^K < 2^59 for bs <= 60) one
// rounding right shift by d = K - sh >= 0 covers both signs of sh without a
// branch: for sh >= 0 the added half-unit lies below the shifted-out zeros.
template <int BS>
__device__ __forceinline__ long long to_fixed(double x, int E) {
    constexpr int K = BS > 54 ? BS - 54 : 0;
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int ex0 = (int)(b >> 52) & 0x7FF;
    const int ex = ex0 > 0 ? ex0 : 1;
    const long long M = (long long)(b & 0xFFFFFFFFFFFFFULL) | (ex0 > 0 ? 1LL << 52 : 0LL);
    int d = K - (ex - 1075 + BS - E);
    d = d < 63 ? d : 63;
    // unsigned: the half-unit 2^(d - 1) reaches 2^62 (d = 63 for elements 57 binades or more below the
    // line's largest), and the sum stays below 2^63
    const unsigned long long half = (1ULL << d) >> 1;
    const long long Y = (long long)((((unsigned long long)M << K) + half) >> d);
    return (b >> 63) ? -Y : Y;
}

// Digits by bit fields: with O = 16 (32^s - 1) / 31, Z = Y + O has plain
// base-32 digits z_t in [0, 31] (the top one in [0, 32]) and Y's balanced
// digits are z_t - 16, so each digit is a shift and a mask.
__device__ __forceinline__ long long digit_offset(int s) { return ((1LL << (OB * s)) - 1) / 31 * 16; }

// Field t of Z (most significant first) is (Z >> 5 (S - 1 - t)) & 31, a
// value in [0, 32] (the top field may be 32).
// The binary16 pair (0x6400 | f0, 0x6400 | f1) of field t of z0 and z1 as
// one 32-bit word, built in place: z0's field shifted down to bit 0, z1's to
// bit 16, both masked and the constant halves set with bitwise operations
// only (no per-field assembly of the pair).  The top field (t = 0) takes six
// bits: its value is at most 32.
template <int S, int T>
__device__ __forceinline__ unsigned half2_fields(long long z0, long long z1) {
    constexpr int sh = OB * (S - 1 - T);
    constexpr unsigned mask = T == 0 ? 0x3Fu : 0x1Fu;
    const unsigned a = (unsigned)(z0 >> sh);
    const unsigned b = sh >= 16 ? (unsigned)(z1 >> (sh >= 16 ? sh - 16 : 0))
                                : (unsigned)((unsigned long long)z1 << (sh >= 16 ? 0 : 16 - sh));
    return (a & mask) | (b & (mask << 16)) | 0x64006400u;
}

// The e4m3 bytes of two balanced digits f0 - 16, f1 - 16 (f in [0, 32]), f0's
// in the low byte, from their binary16 pair w = (0x6400 | f0, 0x6400 | f1):
// the pattern 0x6400 | f is 1024 + f, subtracting 1040 leaves f - 16 exactly,
// and the hardware conversion of a binary16 pair to an e4m3 pair is exact for
// these integers.  Two digits per conversion and no table lookup.
__device__ __forceinline__ unsigned e4m3x2_of_half2(unsigned w) {
    __half2_raw h;
    h.x = (unsigned short)(w & 0xFFFFu);
    h.y = (unsigned short)(w >> 16);
    const __half2 d = __hsub2(__half2(h), __float2half2_rn(1040.0f));
    return (unsigned)__nv_cvt_halfraw2_to_fp8x2(__half2_raw(d), __NV_SATFINITE, __NV_E4M3);
}

template <int S, int T>
__device__ __forceinline__ void pack_digit4(const long long (&Z)[4], unsigned (&packed)[kOzMaxSlices]) {
    if constexpr (T < S) {
        packed[T] = e4m3x2_of_half2(half2_fields<S, T>(Z[0], Z[1])) |
                    (e4m3x2_of_half2(half2_fields<S, T>(Z[2], Z[3])) << 16);
        pack_digit4<S, T + 1>(Z, packed);
    }
}

// Digit t of four elements (Z[q] = the element's fixed-point value plus the
// digit offset; an element outside the matrix has Z = offset, all digits 0)
// as byte q of packed[t].  S is a compile-time constant, so every field is a
// constant shift.
template <int S>
__device__ __forceinline__ void pack_digits4(const long long (&Z)[4], unsigned (&packed)[kOzMaxSlices]) {
    pack_digit4<S, 0>(Z, packed);
}

// ---------------------------------------------------------------------------
// Exponents and slices, fused.  For every row (left operand) or column (right
// operand) the kernels first take the largest biased exponent (mx, 0 for an
// all-zero line; E = max(mx, 1) - 1021 bounds the line by 2^(E - 1)), then
// split each element into s digits.  Output layout [mat][t][Mp][Kp] bytes
// (K contiguous); padding rows/columns stay zero from the plan's first clear.
// All per-slice arrays are indexed with compile-time indices (registers).
// ---------------------------------------------------------------------------

// Left operand: one warp per row r of X (rows x cols, ld); lane j handles
// elements 4(j + 32 i) .. +3, so each slice row is written with coalesced
// 4-byte stores.
template <int S>
__global__ void slice_rows_kernel(const double *__restrict__ X, long long ld, long long mat_stride, int rows,
                                  int cols, int *__restrict__ mx, int pitch, int Mp, int Kp,
                                  unsigned char *__restrict__ out) {
    constexpr int s = S;
    const int mat = blockIdx.y;
    const double *Xm = X + (long long)mat * mat_stride;
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const long long O = digit_offset(s);
    for (int r = warp; r < rows; r += nwarps) {
        const double *row = Xm + (long long)r * ld;
        int m = 0;
        for (int c = lane; c < cols; c += 32) m = max(m, biased_exponent(__ldg(row + c)));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) mx[(long long)mat * pitch + r] = m;
        const int E = max(m, 1) - 1021;
        unsigned char *orow = out + ((long long)mat * s * Mp + r) * Kp;
        const long long slice_stride = (long long)Mp * Kp;
        for (int c4 = lane; c4 * 4 < cols; c4 += 32) {
            unsigned packed[kOzMaxSlices];
            long long Z[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int c = c4 * 4 + q;
                Z[q] = (c < cols ? to_fixed<OB * S>(__ldg(row + c), E) : 0) + O;
            }
            pack_digits4<S>(Z, packed);
#pragma unroll
            for (int t = 0; t < kOzMaxSlices; ++t)
                if (t < s) *reinterpret_cast<unsigned *>(orow + t * slice_stride + c4 * 4) = packed[t];
        }
    }
}

// Right operand: one CTA (32 x 8 threads) per strip of 32 columns of X
// (rows = K): the column maxima first, then 32 x 32 tiles.  Thread (tx, ty)
// splits the four consecutive K rows 4 ty .. 4 ty + 3 of column tx, so each
// of its digit planes is one 32-bit word; the words are transposed through
// shared memory so that slice row c (K contiguous) is written with coalesced
// stores.
template <int S>
__global__ void slice_cols_kernel(const double *__restrict__ X, long long ld, long long mat_stride, int rows,
                                  int cols, int *__restrict__ mx, int pitch, int Mp, int Kp,
                                  unsigned char *__restrict__ out) {
    constexpr int s = S;
    __shared__ unsigned tile[S][32][9];  // [slice][column][K word], padded: conflict-free both ways
    __shared__ int colmax[8][32];
    const long long O = digit_offset(s);
    const int mat = blockIdx.y;
    const double *Xm = X + (long long)mat * mat_stride;
    const int c0 = blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int c = c0 + tx;
    int m = 0;
    if (c < cols)
        for (int k = ty; k < rows; k += 8) m = max(m, biased_exponent(__ldg(Xm + (long long)k * ld + c)));
    colmax[ty][tx] = m;
    __syncthreads();
    if (ty == 0) {
#pragma unroll
        for (int j = 1; j < 8; ++j) m = max(m, colmax[j][tx]);
        colmax[0][tx] = m;
        if (c < cols) mx[(long long)mat * pitch + c] = m;
    }
    __syncthreads();
    const int E = max(colmax[0][tx], 1) - 1021;
    const int cc = threadIdx.x >> 3, ch = threadIdx.x & 7;
    const long long slice_stride = (long long)Mp * Kp;
    unsigned char *obase = out + ((long long)mat * s * Mp + c0 + cc) * Kp;
    for (int k0 = 0; k0 < rows; k0 += 32) {
        unsigned packed[kOzMaxSlices];
        long long Z[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = k0 + 4 * ty + q;
            Z[q] = (c < cols && k < rows ? to_fixed<OB * S>(__ldg(Xm + (long long)k * ld + c), E) : 0) + O;
        }
        pack_digits4<S>(Z, packed);
#pragma unroll
        for (int t = 0; t < S; ++t) tile[t][tx][ty] = packed[t];
        __syncthreads();
        if (c0 + cc < Mp && k0 + ch * 4 < Kp) {
#pragma unroll
            for (int t = 0; t < S; ++t)
                *reinterpret_cast<unsigned *>(obase + t * slice_stride + k0 + ch * 4) = tile[t][cc][ch];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Slice GEMM with fused recombination and post-additions.
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void cp_async16(unsigned dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void ldsm_x4(unsigned addr, unsigned &r0, unsigned &r1, unsigned &r2, unsigned &r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void mma_e4m3(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k32.row.col.f32.e4m3.e4m3.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Iterates the (group g, slice pair (t, g - t), K slab) sequence of one tile.
struct StepIter {
    int g, t, kb;
};
__device__ __forceinline__ void step_first(StepIter &it, int s) {
    it.g = 2;
    it.t = 1;
    it.kb = 0;
    (void)s;
}
// Returns true when the step just left closed its group g.
__device__ __forceinline__ bool step_next(StepIter &it, int s, int nkb) {
    if (++it.kb < nkb) return false;
    it.kb = 0;
    if (++it.t <= min(s, it.g - 1)) return false;
    ++it.g;
    it.t = max(1, it.g - s);
    return true;
}

__device__ __forceinline__ void load_step(Smem &S, int stage, const OzParams &P, int r, int ti, int tj,
                                          const StepIter &it) {
    const int tid = threadIdx.x;
    const int u = it.g - it.t;  // slice of the right operand (1-based)
    const unsigned char *ga =
        P.sa + (((long long)r * P.s + (it.t - 1)) * P.Mp + (long long)ti * BM) * P.Kp + (long long)it.kb * BKB;
    const unsigned char *gb =
        P.sb + (((long long)r * P.s + (u - 1)) * P.Mp + (long long)tj * BN) * P.Kp + (long long)it.kb * BKB;
    const unsigned sa = smem_u32(S.a[stage]), sb = smem_u32(S.b[stage]);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int id = tid + NT * q;  // 0..1023
        const int row = id >> 3, ch = id & 7;
        const unsigned off = (unsigned)(row * BKB + ((ch ^ (row & 7)) << 4));
        cp_async16(sa + off, ga + (long long)row * P.Kp + ch * 16);
        cp_async16(sb + off, gb + (long long)row * P.Kp + ch * 16);
    }
}

__device__ __forceinline__ void mma_step(const Smem &S, int stage, float (&D)[4][4][4]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wm = warp & 1, wn = warp >> 1;  // 2 x 4 warps, warp tile 64 x 32
    const int q = lane >> 3, rr = lane & 7;
    const unsigned sa = smem_u32(S.a[stage]), sb = smem_u32(S.b[stage]);
#pragma unroll
    for (int kq = 0; kq < BKB / 32; ++kq) {
        unsigned b[4][2];
#pragma unroll
        for (int jp = 0; jp < 2; ++jp) {
            const int n = wn * 32 + (2 * jp + (q >> 1)) * 8 + rr;
            const int ch = kq * 2 + (q & 1);
            ldsm_x4(sb + n * BKB + ((ch ^ (n & 7)) << 4), b[2 * jp][0], b[2 * jp][1], b[2 * jp + 1][0],
                    b[2 * jp + 1][1]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            unsigned a[4];
            const int row = wm * 64 + i * 16 + (q & 1) * 8 + rr;
            const int ch = kq * 2 + (q >> 1);
            ldsm_x4(sa + row * BKB + ((ch ^ (row & 7)) << 4), a[0], a[1], a[2], a[3]);
#pragma unroll
            for (int j = 0; j < 4; ++j) mma_e4m3(D[i][j], a, b[j][0], b[j][1]);
        }
    }
}

__device__ __forceinline__ double pow2(int e) {
    return __longlong_as_double((long long)(e + 1023) << 52);
}

// v * 2^sc for any integer sc (exact unless the result leaves the double range).
__device__ __forceinline__ double scale2(double v, int sc) {
    while (sc > 1023) {
        v *= pow2(1023);
        sc -= 1023;
    }
    while (sc < -1022) {
        v *= pow2(-1022);
        sc += 1022;
    }
    return v * pow2(sc);
}

__global__ void __launch_bounds__(NT, 1) ozaki_gemm_kernel(const __grid_constant__ OzParams P) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem &S = *reinterpret_cast<Smem *>(smem_raw);
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int g8 = lane >> 2, t4 = lane & 3;
    const int wm = warp & 1, wn = warp >> 1;
    const int tiles = P.tiles_m * P.tiles_n;
    const int nkb = P.Kp / BKB;
    const int npairs = P.s * (P.s + 1) / 2;
    const int nsteps = npairs * nkb;

    while (true) {
        if (tid == 0) {
            long long tk = (long long)atomicAdd(P.task_counter, 1ull);
            if (ld_volatile(P.error) != kDevOk) tk = P.tasks;
            S.task = tk;
        }
        __syncthreads();
        const long long task = S.task;
        if (task >= P.tasks) break;
        const int r = (int)(task / tiles);
        const int t = (int)(task - (long long)r * tiles);
        const int ti = t / P.tiles_n, tj = t - ti * P.tiles_n;
        {  // destinations of product r
            const int wc = P.w_ptr[r], nD = P.w_ptr[r + 1] - wc;
            for (int e = tid; e < nD; e += NT) {
                const int4 en = P.w_ent[wc + e];
                const long long br = en.x / P.P, bc = en.x % P.P;
                S.dst[e].ptr = P.C + (br * P.m + (long long)ti * BM) * P.ldc + bc * P.m + (long long)tj * BN;
                S.dst[e].chain = P.chain + (long long)en.x * tiles + t;
                S.dst[e].coef = en.y;
                S.dst[e].pos = en.z;
            }
            if (tid == 0) S.nD = nD;
        }

        float D[4][4][4];
        long long acc[4][4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    D[i][j][v] = 0.f;
                    acc[i][j][v] = 0;
                }

        StepIter ld_it, mm_it;
        step_first(ld_it, P.s);
        step_first(mm_it, P.s);
        int issued = 0;
#pragma unroll 1
        for (int p = 0; p < STAGES - 1; ++p) {
            if (issued < nsteps) {
                load_step(S, issued % STAGES, P, r, ti, tj, ld_it);
                step_next(ld_it, P.s, nkb);
                ++issued;
            }
            cp_async_commit();
        }
#pragma unroll 1
        for (int step = 0; step < nsteps; ++step) {
            cp_async_wait<STAGES - 2>();
            __syncthreads();
            if (issued < nsteps) {
                load_step(S, issued % STAGES, P, r, ti, tj, ld_it);
                step_next(ld_it, P.s, nkb);
                ++issued;
            }
            cp_async_commit();
            mma_step(S, step % STAGES, D);
            const int g = mm_it.g;
            if (step_next(mm_it, P.s, nkb)) {
                // group g complete: fold D_g into the fixed-point sums
                const int sh = OB * (P.s + 1 - g) - P.L;
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j)
#pragma unroll
                        for (int v = 0; v < 4; ++v) {
                            const long long vi = (long long)__float2int_rn(D[i][j][v]);
                            acc[i][j][v] += sh >= 0 ? vi * (1LL << sh) : ((vi + (1LL << (-sh - 1))) >> (-sh));
                            D[i][j][v] = 0.f;
                        }
            }
        }
        cp_async_wait<0>();

        // P_r tile in FP64 (reusing the accumulator registers).
        const int rows = (int)min((long long)BM, P.m - (long long)ti * BM);
        const int cols = (int)min((long long)BN, P.m - (long long)tj * BN);
        double pv[4][4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int row = wm * 64 + i * 16 + g8 + 8 * h;
                const int ea = row < rows ? max(P.mxa[(long long)r * P.Mp + (long long)ti * BM + row], 1) - 1021 : 0;
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int c2 = 0; c2 < 2; ++c2) {
                        const int col = wn * 32 + j * 8 + 2 * t4 + c2;
                        const int eb =
                            col < cols ? max(P.mxb[(long long)r * P.Mp + (long long)tj * BN + col], 1) - 1021 : 0;
                        const long long a64 = acc[i][j][2 * h + c2];
                        pv[i][j][2 * h + c2] =
                            a64 == 0 ? 0.0 : scale2(__ll2double_rn(a64), ea + eb - OB * (P.s + 1) + P.L);
                    }
            }

        for (int d = 0; d < S.nD; ++d) {
            const Dst dst = S.dst[d];
            if (tid == 0) {
                bool ok = true;
                if (dst.pos > 0) ok = chain_wait(dst.chain, (unsigned)dst.pos, P.error, P.timeout_ns);
                S.ok = ok ? 1 : 0;
            }
            __syncthreads();
            if (!S.ok) break;
            const int cf = dst.coef;
            // C = alpha A B + beta C: alpha scales every coefficient; the first
            // contribution reads C only for beta != 0 and scales it by beta.
            const int unit = P.alpha == 1.0 ? cf : 0;
            const double cfd = P.alpha * (double)cf;
            const bool load = dst.pos != 0 || P.beta != 0.0;
            const double oscale = dst.pos == 0 ? P.beta : 1.0;
            const int mode = load ? (unit == 1 ? 3 : (unit == -1 ? 4 : 5)) : (unit == 1 ? 0 : (unit == -1 ? 1 : 2));
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int row = wm * 64 + i * 16 + g8 + 8 * h;
                        if (row >= rows) continue;
#pragma unroll
                        for (int c2 = 0; c2 < 2; ++c2) {
                            const int col = wn * 32 + j * 8 + 2 * t4 + c2;
                            if (col >= cols) continue;
                            double *p = dst.ptr + (long long)row * P.ldc + col;
                            const double v = pv[i][j][2 * h + c2];
                            double o = 0.0;
                            if (load) {
                                o = __ldcg(p);
                                if (oscale != 1.0) o = oscale * o;
                            }
                            double out;
                            switch (mode) {
                                case 0: out = v; break;
                                case 1: out = neg(v); break;
                                case 2: out = cfd * v; break;
                                case 3: out = o + v; break;
                                case 4: out = o - v; break;
                                default: out = fma(cfd, v, o); break;
                            }
                            *p = out;
                        }
                    }
            __syncthreads();
            if (tid == 0) {
                __threadfence();
                atomicAdd(dst.chain, 1u);
            }
        }
        __syncthreads();
    }
}

// Instantiates the slicing kernels for the slice count s (1 .. kOzMaxSlices).
template <bool ROWS, int S>
void launch_slices_one(dim3 grid, cudaStream_t st, const double *X, long long ld, long long mat_stride, int rows,
                       int cols, int *mx, int pitch, int Mp, int Kp, unsigned char *out) {
    if (ROWS)
        slice_rows_kernel<S><<<grid, 256, 0, st>>>(X, ld, mat_stride, rows, cols, mx, pitch, Mp, Kp, out);
    else
        slice_cols_kernel<S><<<grid, 256, 0, st>>>(X, ld, mat_stride, rows, cols, mx, pitch, Mp, Kp, out);
}
template <bool ROWS>
void launch_slices_s(int s, dim3 grid, cudaStream_t st, const double *X, long long ld, long long mat_stride, int rows,
                     int cols, int *mx, int pitch, int Mp, int Kp, unsigned char *out) {
    switch (s) {
#define FMM_SLICE_CASE(S_)                                                                              \
    case S_: launch_slices_one<ROWS, S_>(grid, st, X, ld, mat_stride, rows, cols, mx, pitch, Mp, Kp, out); break;
        FMM_SLICE_CASE(1) FMM_SLICE_CASE(2) FMM_SLICE_CASE(3) FMM_SLICE_CASE(4) FMM_SLICE_CASE(5) FMM_SLICE_CASE(6)
        FMM_SLICE_CASE(7) FMM_SLICE_CASE(8) FMM_SLICE_CASE(9) FMM_SLICE_CASE(10) FMM_SLICE_CASE(11)
        FMM_SLICE_CASE(12)
#undef FMM_SLICE_CASE
        default: break;
    }
}

}  // namespace

size_t ozaki_smem_bytes() { return sizeof(Smem); }

cudaError_t launch_ozaki_slices(const double *X, long long ld, long long mat_stride, int nmat, int rows, int cols,
                                bool by_rows, int *mx, int pitch, int s, int Mp, int Kp, unsigned char *out,
                                cudaStream_t st) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    for (int m0 = 0; m0 < nmat; m0 += 65535) {
        const int cnt = nmat - m0 < 65535 ? nmat - m0 : 65535;
        const double *Xm = X + (long long)m0 * mat_stride;
        unsigned char *om = out + (long long)m0 * s * Mp * Kp;
        int *mxm = mx + (long long)m0 * pitch;
        if (by_rows) {
            int bx = (rows * 32 + 255) / 256;  // one warp per row
            const int cap = (sms * 16 + cnt - 1) / cnt;
            if (bx > cap) bx = cap;
            if (bx < 1) bx = 1;
            launch_slices_s<true>(s, dim3(bx, cnt), st, Xm, ld, mat_stride, rows, cols, mxm, pitch, Mp, Kp, om);
        } else {
            launch_slices_s<false>(s, dim3((cols + 31) / 32, cnt), st, Xm, ld, mat_stride, rows, cols, mxm, pitch, Mp,
                                   Kp, om);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int ozaki_ctas_per_sm() {
    static int cached = -1;
    if (cached >= 0) return cached;
    if (cudaFuncSetAttribute(ozaki_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem)) !=
        cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, ozaki_gemm_kernel, NT, sizeof(Smem)) != cudaSuccess)
        return 0;
    cached = nb;
    return nb;
}

cudaError_t launch_ozaki_gemm(const OzParams &P, int grid, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e =
            cudaFuncSetAttribute(ozaki_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    ozaki_gemm_kernel<<<grid, NT, sizeof(Smem), s>>>(P);
    return cudaGetLastError();
}

}  // namespace fmm
