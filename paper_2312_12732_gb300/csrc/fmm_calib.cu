// Calibration kernels: sustained FP64 throughput of this GPU on the DMMA path
// (mma.sync m16n8k4 f64, the instruction the leaf kernel issues) and on plain
// DFMA, so that leaf-kernel rates can be read against what the FP64 pipe
// actually delivers.  Register-only loops of fixed length; each thread writes
// one value so that the work is not optimised away.
#include <cuda_runtime.h>

#include "fmm_internal.h"

namespace fmm {
namespace {

__global__ void __launch_bounds__(256) dmma_loop(double *out, int iters) {
    double a[2] = {1e-3 * threadIdx.x, 1e-3 * (threadIdx.x + 1)};
    double b = 1e-3 * (threadIdx.x + 2);
    double c[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int v = 0; v < 4; ++v) c[j][v] = 0.0;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < 8; ++j)
            asm volatile(
                "mma.sync.aligned.m16n8k4.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};"
                : "+d"(c[j][0]), "+d"(c[j][1]), "+d"(c[j][2]), "+d"(c[j][3])
                : "d"(a[0]), "d"(a[1]), "d"(b));
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int v = 0; v < 4; ++v) s += c[j][v];
    out[(long long)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) dfma_loop(double *out, int iters) {
    double x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = 1e-3 * (threadIdx.x + j);
    const double y = 0.999999, z = 1e-7;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = fma(x[j], y, z);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += x[j];
    out[(long long)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) e4m3_loop(float *out, int iters) {
    unsigned a[4], b0 = 0x38383838u, b1 = 0x38383838u;
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = 0x38383838u ^ ((threadIdx.x * 2654435761u) & 0x01010101u);
    float c[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int v = 0; v < 4; ++v) c[j][v] = 0.f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < 8; ++j)
            asm volatile(
                "mma.sync.aligned.m16n8k32.row.col.f32.e4m3.e4m3.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                "{%0,%1,%2,%3};"
                : "+f"(c[j][0]), "+f"(c[j][1]), "+f"(c[j][2]), "+f"(c[j][3])
                : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int v = 0; v < 4; ++v) s += c[j][v];
    out[(long long)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

cudaError_t measure_e4m3_peak(cudaStream_t s, double *tflops) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int blocks = sms * 2, threads = 256, iters = 8192;
    float *out = nullptr;
    e = cudaMalloc(&out, sizeof(float) * blocks * threads);
    if (e != cudaSuccess) return e;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    e4m3_loop<<<blocks, threads, 0, s>>>(out, 16);
    cudaEventRecord(e0, s);
    e4m3_loop<<<blocks, threads, 0, s>>>(out, iters);
    cudaEventRecord(e1, s);
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double fl = 2.0 * 16 * 8 * 32 * 8.0 * iters * blocks * (threads / 32);
        if (tflops) *tflops = fl / (ms * 1e-3) / 1e12;
        e = cudaGetLastError();
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    return e;
}

cudaError_t measure_fp64_peaks(cudaStream_t s, double *dmma_tflops, double *dfma_tflops) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int blocks = sms * 2, threads = 256;
    double *out = nullptr;
    e = cudaMalloc(&out, sizeof(double) * blocks * threads);
    if (e != cudaSuccess) return e;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float ms = 0.f;
    const int it_mma = 2048, it_fma = 16384;
    dmma_loop<<<blocks, threads, 0, s>>>(out, 8);  // warm-up
    cudaEventRecord(e0, s);
    dmma_loop<<<blocks, threads, 0, s>>>(out, it_mma);
    cudaEventRecord(e1, s);
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) {
        cudaEventElapsedTime(&ms, e0, e1);
        const double fl = 2.0 * 16 * 8 * 4 * 8.0 * it_mma * blocks * (threads / 32);
        if (dmma_tflops) *dmma_tflops = fl / (ms * 1e-3) / 1e12;
        dfma_loop<<<blocks, threads, 0, s>>>(out, 8);
        cudaEventRecord(e0, s);
        dfma_loop<<<blocks, threads, 0, s>>>(out, it_fma);
        cudaEventRecord(e1, s);
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) {
            cudaEventElapsedTime(&ms, e0, e1);
            const double fl2 = 2.0 * 8 * (double)it_fma * blocks * threads;
            if (dfma_tflops) *dfma_tflops = fl2 / (ms * 1e-3) / 1e12;
        }
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    return e;
}

}  // namespace fmm
