// Device helpers shared by the library's kernels (bounded waits on the
// post-addition ordering counters, integer-pipe sign flips, the balanced walk
// over matrix positions).
#pragma once

#include <cuda_runtime.h>

#include "fmm_internal.h"

namespace fmm {
namespace dev {

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_volatile(const int *p) { return *reinterpret_cast<const volatile int *>(p); }

// Waits until *ctr == target.  Bounded: gives up after timeout_ns or as soon
// as another CTA has flagged an error.  Returns true on success.
__device__ __forceinline__ bool chain_wait(const unsigned *ctr, unsigned target, int *error, long long timeout_ns) {
    const unsigned long long t0 = global_ns();
    unsigned sleep = 32;
    while (true) {
        const unsigned v = ld_acquire(ctr);
        if (v == target) return true;
        if (ld_volatile(error) != kDevOk) return false;
        if ((long long)(global_ns() - t0) > timeout_ns) {
            atomicCAS(error, kDevOk, kDevTimeout);
            return false;
        }
        __nanosleep(sleep);
        if (sleep < 256) sleep <<= 1;
    }
}

// Sign flip on the integer pipe (FP64 units are the scarce resource).
__device__ __forceinline__ double neg(double v) {
    return __longlong_as_double(__double_as_longlong(v) ^ (long long)0x8000000000000000ULL);
}

// The positions (c, y, x) of matrices of side b, walked in the linear order
// c b^2 + y b + x: each thread starts at its global index and advances by the
// grid's thread count, whose split into
// (dc, dy, dx) is taken once, so the loop needs no division.  Every thread
// gets the same number of positions (to within one), and a warp's positions
// are consecutive in x, so loads and stores stay coalesced.
struct PosWalk {
    long long c, y, x, dc, dy, dx, b;
    __device__ PosWalk(long long b_, long long bb) : b(b_) {
        const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
        const long long G = (long long)gridDim.x * blockDim.x;
        c = i / bb;
        y = (i - c * bb) / b;
        x = i - c * bb - y * b;
        dc = G / bb;
        dy = (G - dc * bb) / b;
        dx = G - dc * bb - dy * b;
    }
    __device__ __forceinline__ void next() {
        x += dx;
        if (x >= b) { x -= b; ++y; }
        y += dy;
        if (y >= b) { y -= b; ++c; }
        c += dc;
    }
};

}  // namespace dev
}  // namespace fmm
