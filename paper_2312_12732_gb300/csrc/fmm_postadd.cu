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

}  // namespace fmm
