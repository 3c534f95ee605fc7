// Post-additions of the emulated leaf (Section 2, equation `strassen`):
// C_l = alpha sum_r W[l][r] P_r + beta C_l for every C block l, from the leaf
// products P_r that the tcgen05 slice GEMM stores in full.  Two forms: the
// flattened sums below, and the level-by-level sums further down for two
// levels of a 2 x 2 algorithm.  In the flattened form the terms of a
// block are taken in ascending r with the operation sequence of ordered
// read-modify-writes (first term w P, or beta C and then every term; then
// o + P, o - P or fma(w, P, o)), so the result is the one a fused epilogue
// gives.  blockIdx.y is the block, CTAs stride over its rows, threads over
// column pairs.  Bound by the FP64 adds (nnz(W) - P^2 per element of a block)
// and the P_r reads.
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
                                                            long long ldc, unsigned *chain,
                                                            const int *__restrict__ w_row_nnz, int tiles, int l0,
                                                            double alpha, double beta) {
    __shared__ double sw[kMaxScaledTerms];
    __shared__ long long soff[kMaxScaledTerms];
    const int l = l0 + (int)blockIdx.y;
    const long long br = l / Pb, bc = l % Pb;
    const int e0 = wl_ptr[l], e1 = wl_ptr[l + 1];
    const long long mm = m * m;
    if (chain != nullptr && blockIdx.x == 0)
        for (int t = threadIdx.x; t < tiles; t += blockDim.x) chain[(long long)l * tiles + t] = (unsigned)w_row_nnz[l];
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

// Post-additions of a two-level plan of a 2 x 2 algorithm, taken level by
// level as the recursion defines them (Section 2, equation `eq:recursion`):
// for each outer product r1 its inner products P_{r1 R2 + r2} form the four
// blocks of that product, U_q = sum_{r2} Wi[q][r2] P_{r1 R2 + r2} (ascending
// r2), which are then added into the C blocks, C_(l1, q) = alpha sum_{r1}
// Wo[l1][r1] U_q + beta C (ascending r1).  Each P_r entry is read once (the
// flattened form reads it once per C block that uses it) and the sums take
// (nnz(Wi) - 4) R1 + 4 (nnz(Wo) - 4) fma per position instead of
// 16 (nnz(Wi) nnz(Wo) / 16 - 1).  C block (l1, q) is block row 2 i1 + i2,
// column 2 j1 + j2 of the 4 x 4 grid (l1 = 2 i1 + j1, q = 2 i2 + j2).
// Each thread keeps its products and its 16 running sums in its own column of
// shared memory, indexed by the tables.  Tables: rows q of Wi as {r2, low
// word, high word of the coefficient as a double, 0}; columns r1 of Wo as
// {l1, coefficient, 1 if this is the first term of row l1, 0}.
// UNIT: every coefficient of Wi is +-1, so the first term of an inner sum is
// a sign flip (integer pipe) instead of a multiply.
constexpr int kTwoStepThreads = 128;
constexpr int kTwoStepMaxR = 8;
__device__ __forceinline__ double times_unit(double v, int hi_word) {
    const unsigned long long sign = (unsigned long long)((unsigned)hi_word & 0x80000000u) << 32;
    return __longlong_as_double((long long)((unsigned long long)__double_as_longlong(v) ^ sign));
}
template <bool UNIT>
__global__ void __launch_bounds__(kTwoStepThreads)
    ozaki_postadd_two_steps_kernel(const double *__restrict__ pout, long long m, int R1, int R2,
                                   const int *__restrict__ wi_ptr, const int4 *__restrict__ wi_ent,
                                   const int *__restrict__ wo_ptr, const int4 *__restrict__ wo_ent,
                                   double *__restrict__ C, long long ldc, unsigned *chain,
                                   const int *__restrict__ w_row_nnz, int tiles, double alpha, double beta) {
    __shared__ double ps[kTwoStepMaxR][kTwoStepThreads];
    __shared__ double cs[16][kTwoStepThreads];
    __shared__ double sw[4 * kTwoStepMaxR];  // alpha * Wo coefficients, in wo_ent order
    const int tid = threadIdx.x;
    if (chain != nullptr && blockIdx.x == 0)
        for (int t = tid; t < 16 * tiles; t += blockDim.x) chain[t] = (unsigned)w_row_nnz[t / tiles];
    for (int k = tid; k < wo_ptr[R1]; k += blockDim.x) sw[k] = alpha * (double)wo_ent[k].y;
    __syncthreads();
    const long long mm = m * m;
    const bool from_c = beta != 0.0;
    for (dev::PosWalk w(m, mm); w.c < 1; w.next()) {
        const long long y = w.y, x = w.x, pos = y * m + x;
        auto cptr = [&](int l1, int q) {
            return C + ((long long)(2 * (l1 >> 1) + (q >> 1)) * m + y) * ldc +
                   (long long)(2 * (l1 & 1) + (q & 1)) * m + x;
        };
        if (from_c) {
#pragma unroll
            for (int l = 0; l < 16; ++l) {
                const double c = __ldcg(cptr(l >> 2, l & 3));
                cs[l][tid] = beta == 1.0 ? c : beta * c;
            }
        }
        for (int r1 = 0; r1 < R1; ++r1) {
            const double *pr = pout + (long long)r1 * R2 * mm + pos;
#pragma unroll
            for (int r2 = 0; r2 < kTwoStepMaxR; ++r2)
                if (r2 < R2) ps[r2][tid] = __ldg(pr + (long long)r2 * mm);
            double u[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int e0 = wi_ptr[q], e1 = wi_ptr[q + 1];
                const int4 f = wi_ent[e0];  // every row of Wi has a term (checked on the host)
                u[q] = UNIT ? times_unit(ps[f.x][tid], f.z) : __hiloint2double(f.z, f.y) * ps[f.x][tid];
                for (int k = e0 + 1; k < e1; ++k) {
                    const int4 en = wi_ent[k];
                    u[q] = fma(__hiloint2double(en.z, en.y), ps[en.x][tid], u[q]);
                }
            }
            for (int k = wo_ptr[r1]; k < wo_ptr[r1 + 1]; ++k) {
                const int4 en = wo_ent[k];
                const double wk = sw[k];
                const int l1 = en.x;
                if (en.z && !from_c) {  // the first term of row l1 (a uniform branch: the table decides)
                    if (wk == 1.0 || wk == -1.0) {
                        const int hi = __double2hiint(wk);
#pragma unroll
                        for (int q = 0; q < 4; ++q) cs[4 * l1 + q][tid] = times_unit(u[q], hi);
                    } else {
#pragma unroll
                        for (int q = 0; q < 4; ++q) cs[4 * l1 + q][tid] = wk * u[q];
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q) cs[4 * l1 + q][tid] = fma(wk, u[q], cs[4 * l1 + q][tid]);
                }
            }
        }
#pragma unroll
        for (int l = 0; l < 16; ++l) *cptr(l >> 2, l & 3) = cs[l][tid];
    }
}

}  // namespace

cudaError_t launch_ozaki_postadd(const double *pout, long long m, int P, const int *wl_ptr, const int2 *wl_ent,
                                 double *C, long long ldc, unsigned *chain, const int *w_row_nnz, int tiles,
                                 double alpha, double beta, cudaStream_t s) {
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
        ozaki_postadd_kernel<<<grid, 256, 0, s>>>(pout, m, P, wl_ptr, wl_ent, C, ldc, chain, w_row_nnz, tiles, l0,
                                                   alpha, beta);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_ozaki_postadd_two_steps(const double *pout, long long m, int R1, int R2, const int *wi_ptr,
                                           const int4 *wi_ent, const int *wo_ptr, const int4 *wo_ent, double *C,
                                           long long ldc, unsigned *chain, const int *w_row_nnz, int tiles,
                                           double alpha, double beta, bool unit_inner, cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    if (R1 < 1 || R1 > kTwoStepMaxR || R2 < 1 || R2 > kTwoStepMaxR) return cudaErrorInvalidValue;
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ozaki_postadd_two_steps_kernel<true>, kTwoStepThreads,
                                                      0) != cudaSuccess ||
        occ < 1) {
        cudaGetLastError();
        occ = 1;
    }
    const long long need = (m * m + kTwoStepThreads - 1) / kTwoStepThreads;
    const long long slots = (long long)(sms > 0 ? sms : 1) * occ;
    const unsigned grid = (unsigned)(need < slots ? need : slots);
    if (unit_inner)
        ozaki_postadd_two_steps_kernel<true><<<grid, kTwoStepThreads, 0, s>>>(
            pout, m, R1, R2, wi_ptr, wi_ent, wo_ptr, wo_ent, C, ldc, chain, w_row_nnz, tiles, alpha, beta);
    else
        ozaki_postadd_two_steps_kernel<false><<<grid, kTwoStepThreads, 0, s>>>(
            pout, m, R1, R2, wi_ptr, wi_ent, wo_ptr, wo_ent, C, ldc, chain, w_row_nnz, tiles, alpha, beta);
    return cudaGetLastError();
}

}  // namespace fmm
