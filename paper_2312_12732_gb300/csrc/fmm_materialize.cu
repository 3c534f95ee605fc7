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

using dev::PosWalk;

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

// One materialized recursion level: all R outputs of a position are formed
// from the p^2 inputs.
template <bool UNIT>
__global__ void __launch_bounds__(256) materialize_level_kernel(const double *__restrict__ in, long long ld_in, long long in_stride,
                                         int n_in, long long b, int p, int R, const int *__restrict__ ptr,
                                         const int4 *__restrict__ ent, double *__restrict__ out) {
    const long long total = b * b;
    for (PosWalk w(b, total); w.c < n_in; w.next()) {
        {
            const long long c = w.c, y = w.y, x = w.x;
            const double *pos = in + c * in_stride + y * ld_in + x;
            double *dst = out + c * R * total;
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
constexpr int kWalkThreads = 256;
template <bool UNIT>
__global__ void __launch_bounds__(kWalkThreads) materialize_two_steps_kernel(const double *__restrict__ in, long long ld_in, long long in_stride,
                                             int n_in, long long b2, int R1, const int *__restrict__ ptr1,
                                             const int4 *__restrict__ ent1, int R2, const int *__restrict__ ptr2,
                                             const int4 *__restrict__ ent2, double *__restrict__ out) {
    const long long total = b2 * b2;
    const long long b1 = 2 * b2;
    for (PosWalk wk(b2, total); wk.c < n_in; wk.next()) {
        const long long y = wk.y, x = wk.x;
        const double *src = in + wk.c * in_stride;
        double *dst = out + wk.c * R1 * R2 * total;
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
                    // selects, not a pointer, keep v in registers (a per-thread column of shared memory
                    // addressed by the table measured no faster)
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

}  // namespace

namespace {

// One CTA of 256 threads per resident slot (the kernel's occupancy times the
// SM count), or fewer for small inputs: the linear walk then gives every
// thread the same share of positions and the grid runs as one wave.
template <class Kernel>
unsigned walk_grid(Kernel kernel, long long positions) {
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kWalkThreads, 0) != cudaSuccess || occ < 1) {
        cudaGetLastError();
        occ = 1;
    }
    const long long slots = (long long)(sms > 0 ? sms : 1) * occ;
    const long long need = (positions + kWalkThreads - 1) / kWalkThreads;
    return (unsigned)(need < slots ? need : slots);
}

}  // namespace

cudaError_t launch_materialize_level(const double *in, long long ld_in, long long in_stride, int n_in,
                                     long long b_out, int p, int R, const int *ptr, const int4 *ent, bool unit,
                                     double *out, cudaStream_t s) {
    const long long positions = (long long)n_in * b_out * b_out;
    if (positions <= 0) return cudaSuccess;
    if (unit)
        materialize_level_kernel<true><<<walk_grid(materialize_level_kernel<true>, positions), kWalkThreads, 0, s>>>(
            in, ld_in, in_stride, n_in, b_out, p, R, ptr, ent, out);
    else
        materialize_level_kernel<false><<<walk_grid(materialize_level_kernel<false>, positions), kWalkThreads, 0, s>>>(
            in, ld_in, in_stride, n_in, b_out, p, R, ptr, ent, out);
    return cudaGetLastError();
}

cudaError_t launch_materialize_two_steps(const double *in, long long ld_in, long long in_stride, int n_in,
                                         long long b2, int R1, const int *ptr1, const int4 *ent1, int R2,
                                         const int *ptr2, const int4 *ent2, bool unit, double *out,
                                         cudaStream_t s) {
    if (R1 > kPairStepMaxR || R2 > kPairStepMaxR) return cudaErrorInvalidValue;
    const long long positions = (long long)n_in * b2 * b2;
    if (positions <= 0) return cudaSuccess;
    if (unit)
        materialize_two_steps_kernel<true>
            <<<walk_grid(materialize_two_steps_kernel<true>, positions), kWalkThreads, 0, s>>>(
                in, ld_in, in_stride, n_in, b2, R1, ptr1, ent1, R2, ptr2, ent2, out);
    else
        materialize_two_steps_kernel<false>
            <<<walk_grid(materialize_two_steps_kernel<false>, positions), kWalkThreads, 0, s>>>(
                in, ld_in, in_stride, n_in, b2, R1, ptr1, ent1, R2, ptr2, ent2, out);
    return cudaGetLastError();
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
