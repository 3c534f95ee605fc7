// Element-wise kernels of the double-complex and single-precision products
// (Section 1 lists single precision and double complex among the types the
// algorithms deploy to).  A complex n x n matrix
// is interleaved (re, im) binary64; a complex plan splits its operands into
// real planes, runs real fast products on them and joins the result:
//   4M:  Re C = Re A Re B - Im A Im B,  Im C = Re A Im B + Im A Re B;
//   3M:  T1 = Re A Re B, T2 = Im A Im B, T3 = (Re A + Im A)(Re B + Im B),
//        Re C = T1 - T2, Im C = (T3 - T1) - T2.
// All are HBM-bound streams (16 B in, 16-24 B out per element, or the
// reverse), grid-stride over the n^2 elements with coalesced accesses.
#include <cuda_runtime.h>

#include "fmm_internal.h"

namespace fmm {
namespace {

__global__ void __launch_bounds__(256) split_complex_kernel(const double2 *__restrict__ X, long long count,
                                                            double *__restrict__ re, double *__restrict__ im,
                                                            double *__restrict__ sum) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += stride) {
        const double2 x = __ldg(X + t);
        re[t] = x.x;
        im[t] = x.y;
        if (sum != nullptr) sum[t] = x.x + x.y;
    }
}

__global__ void __launch_bounds__(256) join_complex_kernel(const double *__restrict__ re,
                                                           const double *__restrict__ im, double2 *__restrict__ C,
                                                           long long count) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += stride)
        C[t] = make_double2(re[t], im[t]);
}

// C = alpha (T1 - T2, (T3 - T1) - T2) + beta C; beta = 0 does not read C.
__global__ void __launch_bounds__(256) gauss_join_kernel(const double *__restrict__ T1, const double *__restrict__ T2,
                                                         const double *__restrict__ T3, double2 *__restrict__ C,
                                                         long long count, double alpha, double beta) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += stride) {
        const double t1 = T1[t], t2 = T2[t];
        double r = t1 - t2, i = (T3[t] - t1) - t2;
        if (alpha != 1.0) {
            r = alpha * r;
            i = alpha * i;
        }
        if (beta != 0.0) {
            const double2 c = C[t];
            r = fma(beta, c.x, r);
            i = fma(beta, c.y, i);
        }
        C[t] = make_double2(r, i);
    }
}

// Single precision operands (FMM_F32): exact widening to binary64, rounding
// back to nearest binary32, and C = beta C on binary32 (beta = 0: zeros, C not
// read).  HBM-bound streams like the complex planes.
__global__ void __launch_bounds__(256) f32_to_f64_kernel(const float *__restrict__ X, long long count,
                                                         double *__restrict__ out) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += stride)
        out[t] = (double)__ldg(X + t);
}

__global__ void __launch_bounds__(256) f64_to_f32_kernel(const double *__restrict__ X, long long count,
                                                         float *__restrict__ out) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += stride)
        out[t] = __double2float_rn(X[t]);
}

__global__ void __launch_bounds__(256) scale_f32_kernel(float *C, long long count, float beta) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += stride)
        C[t] = beta == 0.0f ? 0.0f : beta * C[t];
}

int stream_grid(long long count) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long g = (count + 255) / 256;
    if (g > (long long)sms * 8) g = (long long)sms * 8;
    return g < 1 ? 1 : (int)g;
}

}  // namespace

cudaError_t launch_split_complex(const double *X, long long count, double *re, double *im, double *sum,
                                 cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    split_complex_kernel<<<stream_grid(count), 256, 0, s>>>(reinterpret_cast<const double2 *>(X), count, re, im, sum);
    return cudaGetLastError();
}

cudaError_t launch_join_complex(const double *re, const double *im, double *C, long long count, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    join_complex_kernel<<<stream_grid(count), 256, 0, s>>>(re, im, reinterpret_cast<double2 *>(C), count);
    return cudaGetLastError();
}

cudaError_t launch_gauss_join(const double *T1, const double *T2, const double *T3, double *C, long long count,
                              double alpha, double beta, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    gauss_join_kernel<<<stream_grid(count), 256, 0, s>>>(T1, T2, T3, reinterpret_cast<double2 *>(C), count, alpha,
                                                         beta);
    return cudaGetLastError();
}

cudaError_t launch_f32_to_f64(const float *X, long long count, double *out, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    f32_to_f64_kernel<<<stream_grid(count), 256, 0, s>>>(X, count, out);
    return cudaGetLastError();
}

cudaError_t launch_f64_to_f32(const double *X, long long count, float *out, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    f64_to_f32_kernel<<<stream_grid(count), 256, 0, s>>>(X, count, out);
    return cudaGetLastError();
}

cudaError_t launch_scale_f32(float *C, long long count, float beta, cudaStream_t s) {
    if (count <= 0 || beta == 1.0f) return cudaSuccess;
    scale_f32_kernel<<<stream_grid(count), 256, 0, s>>>(C, count, beta);
    return cudaGetLastError();
}

}  // namespace fmm
