// Post-additions from stored leaf products (Section 2, equation `strassen`):
// C_l = alpha sum_r W[l][r] P_r + beta C_l for every C block l.  Two forms:
//   * the flattened sums of the emulated leaf (depth 1, or on request): the
//     terms of a block are taken in ascending r with the operation sequence of
//     ordered read-modify-writes (first term w P, or beta C and then every
//     term; then o + P, o - P or fma(w, P, o)), so the result is the one a
//     fused epilogue gives.  blockIdx.y is the block, CTAs stride over its
//     rows, threads over column pairs.  Bound by the FP64 adds (nnz(W) - P^2
//     per element of a block) and the P_r reads;
//   * the level-by-level passes further down, which sum W's Kronecker factors
//     from the leaf upwards (FP64 plans that store their products, and the
//     emulated leaf from depth 2).
#include <cuda_runtime.h>

#include "fmm_device.cuh"
#include "fmm_internal.h"

namespace fmm {
namespace {

constexpr int NB = 8;                  // terms whose loads are in flight together
constexpr int kMaxScaledTerms = 1024;  // coefficients of a block kept in shared memory

// Every term is one fma(w, P, c) with w = alpha * W[l][r] from a per-block
// table: no branch on the coefficient, one FP64 operation per element and
// term.  fma(+-1, v, c) equals c +- v exactly, so with alpha = 1 the result is
// bit for bit that of adds and subtracts; the first term (beta = 0) is w * v.
__global__ void __launch_bounds__(256) ozaki_postadd_kernel(const double *__restrict__ pout, long long m, int Pb,
                                                            const int *__restrict__ wl_ptr,
                                                            const int2 *__restrict__ wl_ent, double *__restrict__ C,
                                                            long long ldc, int l0, double alpha, double beta) {
    __shared__ double sw[kMaxScaledTerms];
    __shared__ long long soff[kMaxScaledTerms];
    const int l = l0 + (int)blockIdx.y;
    const long long br = l / Pb, bc = l % Pb;
    const int e0 = wl_ptr[l], e1 = wl_ptr[l + 1];
    const long long mm = m * m;
    for (int t = threadIdx.x; t < e1 - e0 && t < kMaxScaledTerms; t += blockDim.x) {
        const int2 en = wl_ent[e0 + t];  // {product r, coefficient}
        sw[t] = alpha * (double)en.y;
        soff[t] = (long long)en.x * mm;
    }
    __syncthreads();
    // coefficient and P_r offset of term e (from the table, or formed in place past its end)
    auto term = [&](int e, double &w, long long &off) {
        if (e - e0 < kMaxScaledTerms) {
            w = sw[e - e0];
            off = soff[e - e0];
        } else {
            const int2 en = wl_ent[e];
            w = alpha * (double)en.y;
            off = (long long)en.x * mm;
        }
    };
    const bool pairs = (m & 1) == 0 && (ldc & 1) == 0;  // 16-byte aligned column pairs
    const bool from_c = beta != 0.0;                    // the sum starts at beta C instead of the first term
    const int first = from_c ? e0 : e0 + 1;             // first term taken by the fma loop
    for (long long i = blockIdx.x; i < m; i += gridDim.x) {
        double *crow = C + (br * m + i) * ldc + bc * m;
        const double *prow = pout + i * m;
        if (pairs) {
            for (long long j = 2 * (long long)threadIdx.x; j < m; j += 2 * blockDim.x) {
                double2 c;
                if (from_c) {
                    c = __ldcg(reinterpret_cast<const double2 *>(crow + j));
                    if (beta != 1.0) { c.x = beta * c.x; c.y = beta * c.y; }
                } else {
                    double w;
                    long long off;
                    term(e0, w, off);
                    const double2 v = __ldg(reinterpret_cast<const double2 *>(prow + off + j));
                    c = make_double2(w * v.x, w * v.y);
                }
                for (int eb = first; eb < e1; eb += NB) {
                    double2 v[NB];
                    double w[NB];
#pragma unroll
                    for (int k = 0; k < NB; ++k)
                        if (eb + k < e1) {
                            long long off;
                            term(eb + k, w[k], off);
                            v[k] = __ldg(reinterpret_cast<const double2 *>(prow + off + j));
                        }
#pragma unroll
                    for (int k = 0; k < NB; ++k) {
                        if (eb + k >= e1) break;
                        c.x = fma(w[k], v[k].x, c.x);
                        c.y = fma(w[k], v[k].y, c.y);
                    }
                }
                *reinterpret_cast<double2 *>(crow + j) = c;
            }
        } else {
            for (long long j = threadIdx.x; j < m; j += blockDim.x) {
                double c;
                if (from_c) {
                    c = __ldcg(crow + j);
                    if (beta != 1.0) c = beta * c;
                } else {
                    double w;
                    long long off;
                    term(e0, w, off);
                    c = w * __ldg(prow + off + j);
                }
                for (int eb = first; eb < e1; eb += NB) {
                    double v[NB];
                    double w[NB];
#pragma unroll
                    for (int k = 0; k < NB; ++k)
                        if (eb + k < e1) {
                            long long off;
                            term(eb + k, w[k], off);
                            v[k] = __ldg(prow + off + j);
                        }
#pragma unroll
                    for (int k = 0; k < NB; ++k) {
                        if (eb + k >= e1) break;
                        c = fma(w[k], v[k], c);
                    }
                }
                crow[j] = c;
            }
        }
    }
}

// Sign of a coefficient applied to v on the integer pipe (hi_word: the high
// word of the coefficient as a double; used where the coefficient is +-1).
__device__ __forceinline__ double times_unit(double v, int hi_word) {
    const unsigned long long sign = (unsigned long long)((unsigned)hi_word & 0x80000000u) << 32;
    return __longlong_as_double((long long)((unsigned long long)__double_as_longlong(v) ^ sign));
}

// ---------------------------------------------------------------------------
// Level-by-level post-additions of a plan with stored leaf products (FP64
// leaf or emulated leaf; Section 2, equation `eq:recursion` read from the leaf upwards: the blocks of
// every product of one level are sums of the products of the level below).
// One pass sums one Kronecker factor of W (or two 2 x 2 factors) for every
// (prefix, suffix) group: each thread takes one position of the m x m blocks
// and keeps its running sums in its own column of shared memory.  Work units
// of a.chunk positions of one group are spread over a persistent grid.
// Every term of a sum is one fma(c, v, s) with the integer coefficient c;
// the first term of each sum is c v (a sign flip for c = +-1), so a pass
// costs nnz(W_f) - (blocks) fma per group and position.  Bound by those FP64
// operations (about 0.5 T/s) or by the block reads and writes.
constexpr int kLevelThreads = 128;
constexpr int kLevelMaxChunk = 8 * kLevelThreads;
constexpr int kLevelMaxR = 8;  // products of each factor of a pair pass
constexpr int kLevelLoads = 8;  // products whose loads are in flight together (single-factor pass)

__device__ __forceinline__ double coef_of(int lo, int hi) { return __hiloint2double(hi, lo); }

// Walks the positions [p0, p1) of a unit, kLevelThreads apart, keeping the
// (row, column) of the position inside its m x m block for the stores into C.
struct LevelPos {
    long long pos, y, x;
    __device__ LevelPos(long long p, long long m) : pos(p), y(p / m), x(p - (p / m) * m) {}
    __device__ void next(long long m) {
        pos += kLevelThreads;
        x += kLevelThreads;
        while (x >= m) {
            x -= m;
            ++y;
        }
    }
};

// The result of output o (ordinal among the pass's outputs) at this position:
// stored as is in an intermediate block, or as alpha v + beta C into C.
__device__ __forceinline__ void level_store(const LevelPass &a, long long o, const LevelPos &w, double v) {
    if (!a.last) {
        a.out[o * a.mm + w.pos] = v;
        return;
    }
    const int2 blk = a.c_blk[o];
    double *c = a.out + ((long long)blk.x * a.m + w.y) * a.ldc + (long long)blk.y * a.m + w.x;
    switch (a.store) {  // uniform, decided on the host (no FP64 compare per element)
        case 1: *c = v; break;
        case 2: *c = a.alpha * v; break;
        case 3: *c = fma(a.alpha, v, __ldcg(c)); break;
        default: *c = fma(a.alpha, v, a.beta * __ldcg(c)); break;
    }
}

__global__ void __launch_bounds__(kLevelThreads) level_single_kernel(const __grid_constant__ LevelPass a) {
    extern __shared__ double cs[];  // [qb][kLevelThreads]
    const int tid = threadIdx.x;
    const long long chunks = (a.mm + a.chunk - 1) / a.chunk;
    const long long units = (long long)a.np * a.ns * chunks;
    const long long istride = (long long)a.ns * a.mm;  // between consecutive products of a group
    for (long long u = blockIdx.x; u < units; u += gridDim.x) {
        const long long grp = u / chunks, p0 = (u - grp * chunks) * a.chunk;
        const long long p1 = p0 + a.chunk < a.mm ? p0 + a.chunk : a.mm;
        const long long x = grp / a.ns, sfx = grp - x * a.ns;
        const double *in = a.in + (x * a.rb * a.ns + sfx) * a.mm;
        const long long obase = x * a.qb * a.ns + sfx;
        for (LevelPos w(p0 + tid, a.m); w.pos < p1; w.next(a.m)) {
            for (int r0 = 0; r0 < a.rb; r0 += kLevelLoads) {
                double v[kLevelLoads];
#pragma unroll
                for (int k = 0; k < kLevelLoads; ++k)
                    if (r0 + k < a.rb) v[k] = __ldcs(in + (long long)(r0 + k) * istride + w.pos);
#pragma unroll
                for (int k = 0; k < kLevelLoads; ++k) {
                    if (r0 + k >= a.rb) break;
                    for (int e = a.b_ptr[r0 + k]; e < a.b_ptr[r0 + k + 1]; ++e) {
                        const int4 en = a.b_ent[e];  // uniform across the CTA
                        double *acc = &cs[en.x * kLevelThreads + tid];
                        if (en.w & 1)
                            *acc = (en.w & 2) ? times_unit(v[k], en.z) : coef_of(en.y, en.z) * v[k];
                        else
                            *acc = fma(coef_of(en.y, en.z), v[k], *acc);
                    }
                }
            }
            for (int q = 0; q < a.qb; ++q) level_store(a, obase + (long long)q * a.ns, w, cs[q * kLevelThreads + tid]);
        }
    }
}

template <bool UNIT>
__global__ void __launch_bounds__(kLevelThreads) level_pair_kernel(const __grid_constant__ LevelPass a) {
    __shared__ double ps[kLevelMaxR][kLevelThreads];
    __shared__ double cs[16][kLevelThreads];
    const int tid = threadIdx.x;
    const long long chunks = (a.mm + a.chunk - 1) / a.chunk;
    const long long units = (long long)a.np * a.ns * chunks;
    const long long istride = (long long)a.ns * a.mm;
    for (long long u = blockIdx.x; u < units; u += gridDim.x) {
        const long long grp = u / chunks, p0 = (u - grp * chunks) * a.chunk;
        const long long p1 = p0 + a.chunk < a.mm ? p0 + a.chunk : a.mm;
        const long long x = grp / a.ns, sfx = grp - x * a.ns;
        const double *in = a.in + (x * a.ra * a.rb * a.ns + sfx) * a.mm;
        const long long obase = x * 16 * a.ns + sfx;
        for (LevelPos w(p0 + tid, a.m); w.pos < p1; w.next(a.m)) {
            for (int ra = 0; ra < a.ra; ++ra) {
                const double *pr = in + (long long)ra * a.rb * istride + w.pos;
#pragma unroll
                for (int rb = 0; rb < kLevelMaxR; ++rb)
                    if (rb < a.rb) ps[rb][tid] = __ldcs(pr + (long long)rb * istride);
                double ub[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int e0 = a.b_ptr[q], e1 = a.b_ptr[q + 1];
                    const int4 f = a.b_ent[e0];  // every row of W_b has a term (checked on the host)
                    ub[q] = UNIT ? times_unit(ps[f.x][tid], f.z) : coef_of(f.y, f.z) * ps[f.x][tid];
                    for (int k = e0 + 1; k < e1; ++k) {
                        const int4 en = a.b_ent[k];
                        ub[q] = fma(coef_of(en.y, en.z), ps[en.x][tid], ub[q]);
                    }
                }
                for (int k = a.a_ptr[ra]; k < a.a_ptr[ra + 1]; ++k) {
                    const int4 en = a.a_ent[k];
                    const int qa = en.x;
                    if (en.w & 1) {  // the first term of row qa (uniform: the table decides)
                        if (en.w & 2) {
#pragma unroll
                            for (int q = 0; q < 4; ++q) cs[4 * qa + q][tid] = times_unit(ub[q], en.z);
                        } else {
                            const double c = coef_of(en.y, en.z);
#pragma unroll
                            for (int q = 0; q < 4; ++q) cs[4 * qa + q][tid] = c * ub[q];
                        }
                    } else {
                        const double c = coef_of(en.y, en.z);
#pragma unroll
                        for (int q = 0; q < 4; ++q) cs[4 * qa + q][tid] = fma(c, ub[q], cs[4 * qa + q][tid]);
                    }
                }
            }
#pragma unroll 4
            for (int l = 0; l < 16; ++l) level_store(a, obase + (long long)l * a.ns, w, cs[l][tid]);
        }
    }
}

}  // namespace

cudaError_t launch_ozaki_postadd(const double *pout, long long m, int P, const int *wl_ptr, const int2 *wl_ent,
                                 double *C, long long ldc, double alpha, double beta, cudaStream_t s) {
    if (m <= 0 || P <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long bx = ((long long)sms * 16 + P * P - 1) / ((long long)P * P);
    if (bx > m) bx = m;
    if (bx < 1) bx = 1;
    for (int l0 = 0; l0 < P * P; l0 += 65535) {
        const int cnt = P * P - l0 < 65535 ? P * P - l0 : 65535;
        dim3 grid((unsigned)bx, (unsigned)cnt);
        ozaki_postadd_kernel<<<grid, 256, 0, s>>>(pout, m, P, wl_ptr, wl_ent, C, ldc, l0, alpha, beta);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_level_pass(const LevelPass &a0, cudaStream_t s) {
    if (a0.mm <= 0 || a0.np <= 0 || a0.ns <= 0) return cudaSuccess;
    LevelPass a = a0;
    a.store = a.beta != 0.0 ? (a.beta == 1.0 ? 3 : 4) : (a.alpha == 1.0 ? 1 : 2);
    const bool pair = a.ra > 1;
    if (pair ? (a.qa != 4 || a.qb != 4 || a.ra > kLevelMaxR || a.rb > kLevelMaxR || a.rb < 1)
             : (a.qb < 1 || a.qb > kLevelMaxQ || a.rb < 1))
        return cudaErrorInvalidValue;
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = pair ? 0 : (size_t)a.qb * kLevelThreads * sizeof(double);
    cudaError_t e = pair ? (a.unit_b ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, level_pair_kernel<true>,
                                                                                    kLevelThreads, 0)
                                     : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, level_pair_kernel<false>,
                                                                                    kLevelThreads, 0))
                         : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, level_single_kernel, kLevelThreads,
                                                                         smem);
    if (e != cudaSuccess || occ < 1) {
        cudaGetLastError();
        occ = 1;
    }
    const long long slots = (long long)(sms > 0 ? sms : 1) * occ;
    // units of up to 1024 positions, smaller while there would be fewer than 8 per resident CTA (the
    // last wave of a pass with few groups left most of the GPU idle)
    a.chunk = kLevelMaxChunk;
    while (a.chunk > kLevelThreads && (long long)a.np * a.ns * ((a.mm + a.chunk - 1) / a.chunk) < 8 * slots)
        a.chunk /= 2;
    const long long units = (long long)a.np * a.ns * ((a.mm + a.chunk - 1) / a.chunk);
    const unsigned grid = (unsigned)(units < slots ? units : slots);
    if (pair) {
        if (a.unit_b)
            level_pair_kernel<true><<<grid, kLevelThreads, 0, s>>>(a);
        else
            level_pair_kernel<false><<<grid, kLevelThreads, 0, s>>>(a);
    } else {
        if (smem > 48 * 1024) {
            e = cudaFuncSetAttribute(level_single_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        level_single_kernel<<<grid, kLevelThreads, smem, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace fmm
