// Device helpers shared by the library's kernels (bounded waits on the
// post-addition ordering counters, integer-pipe sign flips).
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

}  // namespace dev
}  // namespace fmm
