// Post-additions of the emulated leaf (Section 2, equation `strassen`):
// C_l = alpha sum_r W[l][r] P_r + beta C_l for every C block l, from the leaf
// products P_r that the tcgen05 slice GEMM stores in full.  The terms of a
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

constexpr int NB = 8;              // terms whose loads are in flight together
constexpr int kMaxScaledTerms = 1024;  // alpha * W coefficients kept in shared memory per block

// One term.  UNIT (alpha = 1): the integer coefficient picks an add, a
// subtract or an fma, as a uniform branch, so each element pays one FP64
// operation per term.  Otherwise w is the precomputed alpha * W[l][r].
template <bool UNIT>
__device__ __forceinline__ double apply_term(double c, double v, int cf, double w, bool init) {
    if (UNIT) {
        if (init) {
            if (cf == 1) return v;
            if (cf == -1) return dev::neg(v);
            return (double)cf * v;
        }
        if (cf == 1) return c + v;
        if (cf == -1) return c - v;
        return fma((double)cf, v, c);
    }
    return init ? w * v : fma(w, v, c);
}

template <bool UNIT>
__global__ void __launch_bounds__(256) ozaki_postadd_kernel(const double *__restrict__ pout, long long m, int Pb,
                                                            const int *__restrict__ wl_ptr,
                                                            const int2 *__restrict__ wl_ent, double *__restrict__ C,
                                                            long long ldc, unsigned *chain,
                                                            const int *__restrict__ w_row_nnz, int tiles, int l0,
                                                            double alpha, double beta) {
    __shared__ double sw[UNIT ? 1 : kMaxScaledTerms];
    const int l = l0 + (int)blockIdx.y;
    const long long br = l / Pb, bc = l % Pb;
    const int e0 = wl_ptr[l], e1 = wl_ptr[l + 1];
    const long long mm = m * m;
    if (chain != nullptr && blockIdx.x == 0)
        for (int t = threadIdx.x; t < tiles; t += blockDim.x) chain[(long long)l * tiles + t] = (unsigned)w_row_nnz[l];
    if (!UNIT) {
        for (int t = threadIdx.x; t < e1 - e0 && t < kMaxScaledTerms; t += blockDim.x)
            sw[t] = alpha * (double)wl_ent[e0 + t].y;
        __syncthreads();
    }
    // the scaled coefficient of term e (shared table, or formed in place past its end)
    auto scaled = [&](int e, int cf) {
        if (UNIT) return 0.0;
        return e - e0 < kMaxScaledTerms ? sw[e - e0] : alpha * (double)cf;
    };
    const bool pairs = (m & 1) == 0 && (ldc & 1) == 0;  // 16-byte aligned column pairs
    const bool from_c = beta != 0.0;                    // the sum starts at beta C instead of the first term
    for (long long i = blockIdx.x; i < m; i += gridDim.x) {
        double *crow = C + (br * m + i) * ldc + bc * m;
        const double *prow = pout + i * m;
        if (pairs) {
            for (long long j = 2 * (long long)threadIdx.x; j < m; j += 2 * blockDim.x) {
                double2 c = make_double2(0.0, 0.0);
                if (from_c) {
                    c = __ldcg(reinterpret_cast<const double2 *>(crow + j));
                    if (beta != 1.0) { c.x = beta * c.x; c.y = beta * c.y; }
                }
                for (int eb = e0; eb < e1; eb += NB) {
                    double2 v[NB];
                    int cf[NB];
#pragma unroll
                    for (int k = 0; k < NB; ++k)
                        if (eb + k < e1) {
                            const int2 en = wl_ent[eb + k];  // {product r, coefficient}
                            cf[k] = en.y;
                            v[k] = __ldg(reinterpret_cast<const double2 *>(prow + (long long)en.x * mm + j));
                        }
#pragma unroll
                    for (int k = 0; k < NB; ++k) {
                        if (eb + k >= e1) break;
                        const bool init = eb + k == e0 && !from_c;
                        const double w = scaled(eb + k, cf[k]);
                        c.x = apply_term<UNIT>(c.x, v[k].x, cf[k], w, init);
                        c.y = apply_term<UNIT>(c.y, v[k].y, cf[k], w, init);
                    }
                }
                *reinterpret_cast<double2 *>(crow + j) = c;
            }
        } else {
            for (long long j = threadIdx.x; j < m; j += blockDim.x) {
                double c = 0.0;
                if (from_c) {
                    c = __ldcg(crow + j);
                    if (beta != 1.0) c = beta * c;
                }
                for (int eb = e0; eb < e1; eb += NB) {
                    double v[NB];
                    int cf[NB];
#pragma unroll
                    for (int k = 0; k < NB; ++k)
                        if (eb + k < e1) {
                            const int2 en = wl_ent[eb + k];
                            cf[k] = en.y;
                            v[k] = __ldg(prow + (long long)en.x * mm + j);
                        }
#pragma unroll
                    for (int k = 0; k < NB; ++k) {
                        if (eb + k >= e1) break;
                        c = apply_term<UNIT>(c, v[k], cf[k], scaled(eb + k, cf[k]), eb + k == e0 && !from_c);
                    }
                }
                crow[j] = c;
            }
        }
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
        if (alpha == 1.0)
            ozaki_postadd_kernel<true><<<grid, 256, 0, s>>>(pout, m, P, wl_ptr, wl_ent, C, ldc, chain, w_row_nnz,
                                                            tiles, l0, alpha, beta);
        else
            ozaki_postadd_kernel<false><<<grid, 256, 0, s>>>(pout, m, P, wl_ptr, wl_ent, C, ldc, chain, w_row_nnz,
                                                             tiles, l0, alpha, beta);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace fmm
