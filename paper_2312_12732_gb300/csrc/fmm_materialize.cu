// Materialized pre-additions of the fast-matrix-multiplication library
// (sm_103a): S_r = sum_i U[i][r] A_i and T_r = sum_j V[j][r] B_j (Section 2,
// equation `strassen`), formed level by level, or Kronecker factor by factor,
// for every product of the flattened recursion.  The kernels read their
// inputs once per output position and are bound by the FP64 pipe and by HBM.
//
// Every term costs one FP64 operation and no branch: table entries carry the
// coefficient as the bits of a double, a sum starts with its first term
// (a sign flip on the integer pipe when every coefficient of the step is +-1,
// else one multiply) and adds each further term with fma(c, v, s).  For
// c = +-1 that fma is the rounded s + v or s - v, so the sums are those of
// plain adds and subtracts.  A form that chose add, subtract or multiply per
// term from an integer coefficient made the compiler evaluate several of them
// (and convert the integer) for every term.
#include <cuda_runtime.h>

#include "fmm_device.cuh"
#include "fmm_internal.h"

namespace fmm {
namespace {

// entry {block row, block col, low word, high word of the coefficient as a double}
__device__ __forceinline__ double coef_of(const int4 &en) { return __hiloint2double(en.w, en.z); }

template <bool UNIT>
__device__ __forceinline__ double first_term(double v, const int4 &en) {
    if (UNIT) {
        const unsigned long long sign = (unsigned long long)((unsigned)en.w & 0x80000000u) << 32;
        return __longlong_as_double((long long)((unsigned long long)__double_as_longlong(v) ^ sign));
    }
    return coef_of(en) * v;
}

// One materialized recursion level.  blockIdx.y selects the input matrix;
// CTAs stride over rows y of the b x b output blocks and threads over
// columns x, so every load and store is coalesced and no index needs a
// division.  All R outputs of a position are formed from the p^2 inputs.
template <bool UNIT>
__global__ void materialize_level_kernel(const double *__restrict__ in, long long ld_in, long long in_stride,
                                         long long b, int p, int R, const int *__restrict__ ptr,
                                         const int4 *__restrict__ ent, double *__restrict__ out) {
    const long long total = b * b;
    const int c = blockIdx.y;
    const double *src = in + (long long)c * in_stride;
    double *dst = out + (long long)c * R * total;
    for (long long y = blockIdx.x; y < b; y += gridDim.x) {
        for (long long x = threadIdx.x; x < b; x += blockDim.x) {
            const double *pos = src + y * ld_in + x;
            for (int s = 0; s < R; ++s) {
                const int e0 = ptr[s], e1 = ptr[s + 1];
                double acc = 0.0;  // an all-zero column (a product that uses no block) stays zero
                if (e0 < e1) {
                    const int4 f = ent[e0];
                    acc = first_term<UNIT>(__ldg(pos + (long long)f.x * b * ld_in + (long long)f.y * b), f);
                    for (int k = e0 + 1; k < e1; ++k) {
                        const int4 en = ent[k];
                        acc = fma(coef_of(en), __ldg(pos + (long long)en.x * b * ld_in + (long long)en.y * b), acc);
                    }
                }
                dst[(long long)s * total + y * b + x] = acc;
            }
        }
    }
}


// Two consecutive materialization steps with 2 x 2 block grids (Strassen-like
// factors, at most 8 products each) in one pass: a thread reads the 16 inputs
// of one output position, forms the first step's R1 x 4 sums in registers and
// writes the R1 * R2 outputs.  The operations and their order are those of the
// two separate steps, so the results are identical; the first step's output
// never reaches HBM.
constexpr int kPairStepMaxR = 8;
template <bool UNIT>
__global__ void materialize_two_steps_kernel(const double *__restrict__ in, long long ld_in, long long in_stride,
                                             long long b2, int R1, const int *__restrict__ ptr1,
                                             const int4 *__restrict__ ent1, int R2, const int *__restrict__ ptr2,
                                             const int4 *__restrict__ ent2, double *__restrict__ out) {
    const long long total = b2 * b2;
    const long long b1 = 2 * b2;
    const int c = blockIdx.y;
    const double *src = in + (long long)c * in_stride;
    double *dst = out + (long long)c * R1 * R2 * total;
    for (long long y = blockIdx.x; y < b2; y += gridDim.x) {
        for (long long x = threadIdx.x; x < b2; x += blockDim.x) {
            // v[i1][j1][q]: input at outer block (i1, j1), inner block q = 2 i2 + j2
            double v[2][2][4];
#pragma unroll
            for (int i1 = 0; i1 < 2; ++i1)
#pragma unroll
                for (int j1 = 0; j1 < 2; ++j1)
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        v[i1][j1][q] = __ldg(src + (i1 * b1 + (q >> 1) * b2 + y) * ld_in + j1 * b1 + (q & 1) * b2 + x);
            for (int r1 = 0; r1 < R1; ++r1) {
                double t[4] = {0.0, 0.0, 0.0, 0.0};
                const int e0 = ptr1[r1], e1 = ptr1[r1 + 1];
                if (e0 < e1) {
                    const int4 f = ent1[e0];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        // selects, not a pointer, keep v in registers
                        const double w = f.x == 0 ? (f.y == 0 ? v[0][0][q] : v[0][1][q])
                                                  : (f.y == 0 ? v[1][0][q] : v[1][1][q]);
                        t[q] = first_term<UNIT>(w, f);
                    }
                }
                for (int k = e0 + 1; k < e1; ++k) {
                    const int4 en = ent1[k];
                    const double cf = coef_of(en);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const double w = en.x == 0 ? (en.y == 0 ? v[0][0][q] : v[0][1][q])
                                                   : (en.y == 0 ? v[1][0][q] : v[1][1][q]);
                        t[q] = fma(cf, w, t[q]);
                    }
                }
                double *o = dst + (long long)r1 * R2 * total + y * b2 + x;
                for (int r2 = 0; r2 < R2; ++r2) {
                    const int f0 = ptr2[r2], f1 = ptr2[r2 + 1];
                    double acc = 0.0;
                    if (f0 < f1) {
                        const int4 f = ent2[f0];
                        const int qf = 2 * f.x + f.y;
                        acc = first_term<UNIT>(qf == 0 ? t[0] : (qf == 1 ? t[1] : (qf == 2 ? t[2] : t[3])), f);
                    }
                    for (int k = f0 + 1; k < f1; ++k) {
                        const int4 en = ent2[k];
                        const int q = 2 * en.x + en.y;
                        acc = fma(coef_of(en), q == 0 ? t[0] : (q == 1 ? t[1] : (q == 2 ? t[2] : t[3])), acc);
                    }
                    o[(long long)r2 * total] = acc;
                }
            }
        }
    }
}

}  // namespace

cudaError_t launch_materialize_level(const double *in, long long ld_in, long long in_stride, int n_in,
                                     long long b_out, int p, int R, const int *ptr, const int4 *ent, bool unit,
                                     double *out, cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long bx = (long long)sms * 8 / (n_in > 0 ? n_in : 1);
    if (bx > b_out) bx = b_out;
    if (bx < 1) bx = 1;
    const int threads = b_out >= 256 ? 256 : (int)((b_out + 31) / 32 * 32);
    for (int c0 = 0; c0 < n_in; c0 += 65535) {
        const int cnt = n_in - c0 < 65535 ? n_in - c0 : 65535;
        dim3 grid((unsigned)bx, (unsigned)cnt);
        double *o = out + (long long)c0 * R * b_out * b_out;
        if (unit)
            materialize_level_kernel<true><<<grid, threads, 0, s>>>(in + (long long)c0 * in_stride, ld_in, in_stride,
                                                                    b_out, p, R, ptr, ent, o);
        else
            materialize_level_kernel<false><<<grid, threads, 0, s>>>(in + (long long)c0 * in_stride, ld_in, in_stride,
                                                                     b_out, p, R, ptr, ent, o);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_materialize_two_steps(const double *in, long long ld_in, long long in_stride, int n_in,
                                         long long b2, int R1, const int *ptr1, const int4 *ent1, int R2,
                                         const int *ptr2, const int4 *ent2, bool unit, double *out,
                                         cudaStream_t s) {
    if (R1 > kPairStepMaxR || R2 > kPairStepMaxR) return cudaErrorInvalidValue;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long bx = (long long)sms * 8 / (n_in > 0 ? n_in : 1);
    if (bx > b2) bx = b2;
    if (bx < 1) bx = 1;
    const int threads = b2 >= 256 ? 256 : (int)((b2 + 31) / 32 * 32);
    for (int c0 = 0; c0 < n_in; c0 += 65535) {
        const int cnt = n_in - c0 < 65535 ? n_in - c0 : 65535;
        dim3 grid((unsigned)bx, (unsigned)cnt);
        double *o = out + (long long)c0 * R1 * R2 * b2 * b2;
        if (unit)
            materialize_two_steps_kernel<true><<<grid, threads, 0, s>>>(in + (long long)c0 * in_stride, ld_in,
                                                                        in_stride, b2, R1, ptr1, ent1, R2, ptr2,
                                                                        ent2, o);
        else
            materialize_two_steps_kernel<false><<<grid, threads, 0, s>>>(in + (long long)c0 * in_stride, ld_in,
                                                                         in_stride, b2, R1, ptr1, ent1, R2, ptr2,
                                                                         ent2, o);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// C = beta C (the whole update when alpha = 0: A and B are not read).  With
// beta = 0 the kernel stores zeros without reading C, so NaN there is dropped.
__global__ void __launch_bounds__(256) scale_c_kernel(double *C, long long count, double beta) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += stride)
        C[t] = beta == 0.0 ? 0.0 : beta * C[t];
}

cudaError_t launch_scale_c(double *C, long long count, double beta, cudaStream_t s) {
    if (count <= 0 || beta == 1.0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long grid = (count + 255) / 256;
    if (grid > (long long)sms * 8) grid = (long long)sms * 8;
    scale_c_kernel<<<(unsigned)grid, 256, 0, s>>>(C, count, beta);
    return cudaGetLastError();
}

}  // namespace fmm
