// Emulated-FP64 slice GEMM on the 5th-generation tensor cores (tcgen05),
// sm_103a.  Same arithmetic as the mma.sync kernel in fmm_ozaki.cu (Ozaki
// scheme: diagonal groups D_g = sum_{t+u=g} Shat_t That_u of e4m3 slices,
// exact in FP32, folded into int64, one correctly rounded conversion to FP64
// per element), organised the Blackwell way, in two forms:
//
//   ozaki_tc_kernel (one CTA per tile)
//     warp 0     TMA producer: fetches tile tasks in increasing order, streams
//                128 x 256-byte slabs of both slice operands (two 128B-swizzled
//                boxes each) into a 3-stage shared-memory ring with
//                cp.async.bulk.tensor;
//     warp 1     MMA issuer: one thread issues tcgen05.mma kind::f8f6f4
//                (M = 128, N = 128, K = 32) into one of four TMEM
//                accumulators and releases ring slots / hands finished groups
//                over with tcgen05.commit;
//     warps 2-9  epilogue: each thread owns one tile row and 64 columns, reads
//                D_g with tcgen05.ld, folds it into 64 int64 registers while
//                later groups accumulate, converts to FP64 and stores the tile
//                of P_r.
//   ozaki_tc_pair_kernel (CTA pairs, tcgen05 cta_group::2, one pair per
//     cluster; every CTA fetches its own tiles; the default) described above
//     the kernel.
//
// ozaki_postadd_kernel (fmm_postadd.cu) then forms C_l = sum_r W[l][r] P_r in ascending r.
// Every mbarrier wait is bounded by %globaltimer; on expiry the CTA records a
// timeout, stops issuing, waits (bounded) for its own copies and MMAs in
// flight, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_runtime.h>

#include "fmm_device.cuh"
#include "fmm_internal.h"

namespace fmm {
namespace {

using dev::global_ns;
using dev::ld_volatile;

constexpr int OB = kOzDigitBits;
constexpr int TM = 128, TN = 128, BOX = 128;  // tile rows, tile cols, K bytes per TMA box
// Two 128-byte K boxes per operand and stage: the MMA thread waits once per
// eight MMAs.  An mbarrier wait costs the issuing thread about as long as two
// MMAs of this shape take on the tensor pipe, so one wait per four MMAs left
// the pipe idle a third of the time.
constexpr int KBOX = 2, SLAB = BOX * KBOX;     // K bytes per stage
constexpr int STAGES = 3;
constexpr int NTHREADS = 320;                  // 10 warps
constexpr int EPI_WARP0 = 2, NEPI = 8;
// Four 128-column FP32 accumulators (all of TMEM): the MMA threads can run
// three diagonal groups ahead of the epilogue, which covers the conversion and
// store of one task while the next task's first groups accumulate.
constexpr int NBUF = 4;
constexpr int TMEM_COLS = NBUF * 128;
constexpr int TASK_RING = 2;
constexpr uint32_t STAGE_BYTES = 2u * TM * SLAB;

struct __align__(8) Bars {
    unsigned long long full[STAGES], empty[STAGES];
    unsigned long long accfull[NBUF], accempty[NBUF];
    unsigned long long tfull[TASK_RING], tempty[TASK_RING];
    unsigned long long drain;
    long long task[TASK_RING];
    unsigned tmem_base;
    int abort;
};

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long *b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase with the given parity; false on timeout or abort.
__device__ __forceinline__ bool mbar_wait(unsigned long long *b, uint32_t parity, volatile int *abort,
                                          int *gerror, long long timeout_ns) {
    if (mbar_test(b, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (true) {
        if (mbar_test(b, parity)) return true;
        if (*abort) return false;
        if ((long long)(global_ns() - t0) > timeout_ns) {
            *abort = 1;
            atomicCAS(gerror, kDevOk, kDevTimeout);
            return false;
        }
    }
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            su32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(su32(bar))
        : "memory");
}

// Shared-memory matrix descriptor: K-major, 128B swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor: kind::f8f6f4, A = B = e4m3, D = f32, both K-major.
constexpr uint32_t kIdesc = (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(TN >> 3) << 17) |
                            ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ void mma_e4m3(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(kIdesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(unsigned long long *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
}


// v * 2^e rounded to nearest even, built with integer operations only (the
// FP64 pipe is the GPU's scarcest unit).  Normal results: normalise |v| so its
// leading bit is bit 63, keep 53 bits, round on the guard bit with the sticky
// bits and the last kept bit, and add the rounded significand (whose leading
// bit is worth one exponent step) onto the exponent field, so that a carry out
// of the significand bumps the exponent by itself (up to infinity).
// Subnormal results: the significand is |v| scaled to units of 2^-1074 and
// rounded once, the same way.
__device__ __forceinline__ double ldexp_i64_rn(long long v, int e) {
    const unsigned long long sign = (unsigned long long)v & (1ull << 63);
    const unsigned long long a = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
    const int lz = __clzll((long long)a);
    const int E = 63 - lz + e;  // exponent of the leading bit
    unsigned long long bits;
    if (E >= -1022) {
        const unsigned long long m = a << (lz & 63);  // leading bit at 63
        const unsigned long long keep = m >> 11;      // 53 bits
        const unsigned long long up = (m >> 10) & ((m & 0x3FFull) != 0 ? 1ull : (keep & 1ull));
        bits = E > 1023 ? 0x7FF0000000000000ull : ((unsigned long long)(E + 1022) << 52) + keep + up;
    } else {
        const int t = e + 1074;  // |v| * 2^t is the significand in units of 2^-1074
        if (t >= 0) {
            bits = a << t;
        } else if (t <= -64) {
            bits = 0;  // below half of the smallest subnormal (|v| < 2^63)
        } else {
            const int sh = -t;
            const unsigned long long q = a >> sh, rem = a & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
            bits = q + ((rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull);
        }
    }
    return a == 0 ? 0.0 : __longlong_as_double((long long)(sign | bits));
}

// Epilogue of one tile task (product r, tile ti, tj), run by the NEPI epilogue
// warps: folds the diagonal groups g = 2 .. s+1 from TMEM into int64 (each
// thread owns one tile row and 64 columns) while later groups accumulate in
// the other TMEM buffers, converts and scales once to FP64 and stores the
// tile of P_r.  The post-additions C_l = sum_r W[l][r] P_r run afterwards in
// ozaki_postadd_kernel: fused here they made the epilogue's per-task burst
// longer than the MMA threads' lookahead.  Groups are numbered globally per CTA (G0 = first group of this
// task); group G lives in accumulator G mod NBUF.  release(buf) hands an
// accumulator back to the MMA thread.  `emit` is false for the padding tile of a CTA pair (no rows of C):
// its groups are still drained.  Returns false when the CTA must stop.
template <int EW0, class Release>
__device__ __forceinline__ bool epilogue_tile(const OzParams &P, unsigned long long *accfull, volatile int *abort,
                                              uint32_t tmem, int r, int ti, int tj, bool emit, int G0, int H,
                                              Release release) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int e = warp - EW0;            // 0..7
    const int quad = warp & 3;           // TMEM lane quadrant of this warp
    const int row = quad * 32 + lane;    // tile row owned by this thread
    const int half = e >> 2;             // column half
    const int col0 = half * 64;
    const int s = P.s;
    long long acc[64];
#pragma unroll
    for (int j = 0; j < 64; ++j) acc[j] = 0;
    for (int V = 0; V < H * s; ++V) {
        // group V of the task is diagonal g over K piece V / s; the global group index G0 + V selects
        // the accumulator and its use parity
        const int g = 2 + V % s;
        const int G = G0 + V;
        const uint32_t buf = (uint32_t)(G % NBUF), bphase = (uint32_t)((G / NBUF) & 1);
        if (!mbar_wait(&accfull[buf], bphase, abort, P.error, P.timeout_ns)) return false;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int sh = OB * (s + 1 - g) - P.L;
        const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + buf * TN + col0;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            uint32_t v[16];
            tmem_ld16(taddr + c * 16, v);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const long long vi = (long long)__float2int_rn(__uint_as_float(v[j]));
                acc[c * 16 + j] += sh >= 0 ? vi * (1LL << sh) : ((vi + (1LL << (-sh - 1))) >> (-sh));
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) release(buf);
    }
    if (!emit) return true;

    // FP64 values of this thread's 64 elements of P_r, converted in place
    // (the bits replace the int64 sums, so both never occupy registers at once)
    const int rows = (int)min((long long)TM, P.m - (long long)ti * TM);
    const int cols = (int)min((long long)TN, P.m - (long long)tj * TN);
    const int ea = row < rows ? max(P.mxa[(long long)r * P.Mp + (long long)ti * TM + row], 1) - 1021 : 0;
    // column exponents: 64 consecutive ints, 16-byte aligned (Mp, TN and col0 are multiples of 64);
    // padding columns hold zeros, which only ever scale zero sums
    const int4 *mxb4 = reinterpret_cast<const int4 *>(P.mxb + (long long)r * P.Mp + (long long)tj * TN + col0);
    const int base_sc = ea - 1021 - OB * (s + 1) + P.L;
#pragma unroll
    for (int j4 = 0; j4 < 16; ++j4) {
        const int4 e4 = __ldg(mxb4 + j4);
        const int ebs[4] = {e4.x, e4.y, e4.z, e4.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int j = 4 * j4 + u;
            acc[j] = __double_as_longlong(ldexp_i64_rn(acc[j], base_sc + max(ebs[u], 1)));
        }
    }

    // store this thread's 64 elements of the P_r tile (row-major, leading
    // dimension m): whole 32-byte sectors when the row is aligned
    if (row < rows) {
        double *prow = P.pout + (long long)r * P.m * P.m + ((long long)ti * TM + row) * P.m + (long long)tj * TN + col0;
        const bool vec = (((unsigned long long)prow) & 31ull) == 0;
        const int nv = vec ? max(0, min(64, cols - col0)) / 4 : 0;
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            if (u >= nv) break;
            asm volatile("st.global.v4.f64 [%0], {%1,%2,%3,%4};" ::"l"(prow + 4 * u),
                         "d"(__longlong_as_double(acc[4 * u])), "d"(__longlong_as_double(acc[4 * u + 1])),
                         "d"(__longlong_as_double(acc[4 * u + 2])), "d"(__longlong_as_double(acc[4 * u + 3]))
                         : "memory");
        }
#pragma unroll
        for (int j = 0; j < 64; ++j) {
            if (j < 4 * nv) continue;
            if (col0 + j >= cols) break;
            prow[j] = __longlong_as_double(acc[j]);
        }
    }
    return true;
}

// Ten warps put three warps on some of the SM's four register-file partitions
// (16K registers each), which caps the kernel at 168 registers per thread.
__global__ void __launch_bounds__(NTHREADS, 1)
    ozaki_tc_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
                    const __grid_constant__ OzParams P) {
    extern __shared__ unsigned char smem_raw[];
    // 1024-byte alignment for the 128B-swizzled stages
    unsigned char *base =
        (unsigned char *)(((unsigned long long)smem_raw + 1023ull) & ~1023ull);
    unsigned char *stage_mem = base;  // STAGES x (A slab 16 KB, B slab 16 KB)
    Bars &B = *reinterpret_cast<Bars *>(base + STAGES * STAGE_BYTES);
    volatile int *abort = &B.abort;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tiles = P.tiles_m * P.tiles_n;
    const int nbox = P.Kp / BOX;                 // 128-byte K boxes per slice row
    const int nkb = (nbox + KBOX - 1) / KBOX;    // stages per slice pair (the last may hold one box)
    const int s = P.s;

    if (tid == 0) {
        for (int i = 0; i < STAGES; ++i) {
            mbar_init(&B.full[i], 1);
            mbar_init(&B.empty[i], 1);
        }
        for (int i = 0; i < NBUF; ++i) {
            mbar_init(&B.accfull[i], 1);
            mbar_init(&B.accempty[i], NEPI);
        }
        for (int i = 0; i < TASK_RING; ++i) {
            mbar_init(&B.tfull[i], 1);
            mbar_init(&B.tempty[i], 1 + NEPI);
        }
        mbar_init(&B.drain, 1);
        B.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&B.tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = B.tmem_base;

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"(&map_a) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(&map_b) : "memory");
            uint32_t stage = 0, sphase = 0;  // ring position and its wrap parity
            long long issued_tx = 0;          // stages issued (for draining)
            int tslot = 0;
            uint32_t tphase = 0;
            while (!*abort) {
                long long task = (long long)atomicAdd(P.task_counter, 1ull);
                if (ld_volatile(P.error) != kDevOk) task = P.tasks;
                if (!mbar_wait(&B.tempty[tslot], tphase ^ 1u, abort, P.error, P.timeout_ns)) break;
                B.task[tslot] = task;
                mbar_arrive(&B.tfull[tslot]);
                if (++tslot == TASK_RING) {
                    tslot = 0;
                    tphase ^= 1u;
                }
                if (task >= P.tasks) break;
                const int r = (int)(task / tiles);
                const int t = (int)(task - (long long)r * tiles);
                const int ti = t / P.tiles_n, tj = t - ti * P.tiles_n;
                bool ok = true;
                for (int g = 2; g <= s + 1 && ok; ++g)
                    for (int ta = max(1, g - s); ta <= min(s, g - 1) && ok; ++ta)
                        for (int kb = 0; kb < nkb; ++kb) {
                            if (!mbar_wait(&B.empty[stage], sphase ^ 1u, abort, P.error, P.timeout_ns)) {
                                ok = false;
                                break;
                            }
                            unsigned char *sa = stage_mem + stage * STAGE_BYTES;
                            unsigned char *sb = sa + TM * SLAB;
                            const int boxes = min(KBOX, nbox - kb * KBOX);
                            mbar_expect_tx(&B.full[stage], (uint32_t)boxes * (TM + TN) * BOX);
                            const int ya = (r * s + (ta - 1)) * P.Mp + ti * TM;
                            const int yb = (r * s + (g - ta - 1)) * P.Mp + tj * TN;
                            for (int bx = 0; bx < boxes; ++bx) {
                                const int x = (kb * KBOX + bx) * BOX;
                                tma_load_2d(sa + bx * TM * BOX, &map_a, x, ya, &B.full[stage]);
                                tma_load_2d(sb + bx * TN * BOX, &map_b, x, yb, &B.full[stage]);
                            }
                            ++issued_tx;
                            if (++stage == STAGES) {
                                stage = 0;
                                sphase ^= 1u;
                            }
                        }
                if (!ok) break;
            }
            if (*abort) {
                // wait (bounded) for the copies this thread issued into the ring
                uint32_t st2 = stage, ph2 = sphase;
                for (int k = 0; k < STAGES && issued_tx > 0; ++k, --issued_tx) {
                    if (st2 == 0) {
                        st2 = STAGES - 1;
                        ph2 ^= 1u;
                    } else {
                        --st2;
                    }
                    const unsigned long long t0 = global_ns();
                    while (!mbar_test(&B.full[st2], ph2) && (long long)(global_ns() - t0) < P.timeout_ns) {
                    }
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            uint32_t stage = 0, sphase = 0;
            uint32_t buf = 0, bphase = 0;  // accumulator buffer and its wrap parity
            int tslot = 0;
            uint32_t tphase = 0;
            const uint32_t sbase = su32(stage_mem);
            bool any = false;
            while (!*abort) {
                if (!mbar_wait(&B.tfull[tslot], tphase, abort, P.error, P.timeout_ns)) break;
                const long long task = B.task[tslot];
                mbar_arrive(&B.tempty[tslot]);
                if (++tslot == TASK_RING) {
                    tslot = 0;
                    tphase ^= 1u;
                }
                if (task >= P.tasks) break;
                bool ok = true;
                for (int g = 2; g <= s + 1 && ok; ++g) {
                    if (!mbar_wait(&B.accempty[buf], bphase ^ 1u, abort, P.error, P.timeout_ns)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t dtm = tmem + buf * TN;
                    bool first = true;
                    for (int ta = max(1, g - s); ta <= min(s, g - 1) && ok; ++ta)
                        for (int kb = 0; kb < nkb; ++kb) {
                            if (!mbar_wait(&B.full[stage], sphase, abort, P.error, P.timeout_ns)) {
                                ok = false;
                                break;
                            }
                            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                            const uint32_t sa = sbase + stage * STAGE_BYTES;
                            const uint64_t da = desc_sw128(sa), db = desc_sw128(sa + TM * SLAB);
                            const int kmma = min(KBOX, nbox - kb * KBOX) * (BOX / 32);
#pragma unroll
                            for (int k = 0; k < SLAB / 32; ++k) {
                                if (k >= kmma) break;
                                // 32-byte K step inside a box, 16 KB box stride (descriptor units of 16 B)
                                const uint64_t adv = (uint64_t)(((k % (BOX / 32)) * 32) >> 4);
                                const uint64_t boxa = (uint64_t)(((k / (BOX / 32)) * TM * BOX) >> 4);
                                const uint64_t boxb = (uint64_t)(((k / (BOX / 32)) * TN * BOX) >> 4);
                                mma_e4m3(dtm, da + boxa + adv, db + boxb + adv, first ? 0u : 1u);
                                first = false;
                            }
                            mma_commit(&B.empty[stage]);
                            any = true;
                            if (++stage == STAGES) {
                                stage = 0;
                                sphase ^= 1u;
                            }
                        }
                    if (!ok) break;
                    mma_commit(&B.accfull[buf]);
                    if (++buf == NBUF) {
                        buf = 0;
                        bphase ^= 1u;
                    }
                }
                if (!ok) break;
            }
            if (any) {
                // all MMAs issued by this thread complete before TMEM is released
                mma_commit(&B.drain);
                const unsigned long long t0 = global_ns();
                while (!mbar_test(&B.drain, 0) && (long long)(global_ns() - t0) < P.timeout_ns) {
                }
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue
        int tslot = 0, tseq = 0;
        uint32_t tphase = 0;
        while (!*abort) {
            if (!mbar_wait(&B.tfull[tslot], tphase, abort, P.error, P.timeout_ns)) break;
            const long long task = B.task[tslot];
            __syncwarp();
            if (lane == 0) mbar_arrive(&B.tempty[tslot]);
            if (++tslot == TASK_RING) {
                tslot = 0;
                tphase ^= 1u;
            }
            if (task >= P.tasks) break;
            const int r = (int)(task / tiles);
            const int t = (int)(task - (long long)r * tiles);
            const int ti = t / P.tiles_n, tj = t - ti * P.tiles_n;
            if (!epilogue_tile<EPI_WARP0>(P, B.accfull, abort, tmem, r, ti, tj, true, tseq * s, 1,
                                          [&](uint32_t b) { mbar_arrive(&B.accempty[b]); }))
                break;
            ++tseq;
        }
    }

    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

// ---------------------------------------------------------------- CTA pairs
// Cluster helpers for the pair kernel (shared::cluster addressing).
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t mapa(uint32_t saddr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Arrive on an mbarrier of the peer CTA.  The release form orders this
// thread's earlier memory accesses (a slot read, a remote store) before the
// arrival; the relaxed form is used after tcgen05.wait::ld, where the TMEM
// reads it must follow have already completed.
__device__ __forceinline__ void arrive_remote_release(uint32_t caddr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(caddr) : "memory");
}
__device__ __forceinline__ void arrive_remote_relaxed(uint32_t caddr) {
    asm volatile("mbarrier.arrive.relaxed.cluster.shared::cluster.b64 _, [%0];" ::"r"(caddr) : "memory");
}
__device__ __forceinline__ void st_cluster_s64(uint32_t caddr, long long v) {
    asm volatile("st.shared::cluster.s64 [%0], %1;" ::"r"(caddr), "l"(v) : "memory");
}
// Bounded wait with cluster-scope acquire, for phases completed by the peer's release arrivals.
__device__ __forceinline__ bool mbar_test_cl(unsigned long long *b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_cl(unsigned long long *b, uint32_t parity, volatile int *abort,
                                             int *gerror, long long timeout_ns) {
    if (mbar_test_cl(b, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (true) {
        if (mbar_test_cl(b, parity)) return true;
        if (*abort) return false;
        if ((long long)(global_ns() - t0) > timeout_ns) {
            *abort = 1;
            atomicCAS(gerror, kDevOk, kDevTimeout);
            return false;
        }
    }
}
// TMA load into this CTA's shared memory whose completion is signalled on the
// leader CTA's mbarrier (caddr: shared::cluster address).
__device__ __forceinline__ void tma_load_2d_pair(void *dst, const CUtensorMap *map, int x, int y, uint32_t caddr) {
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
        "%3}], [%4];" ::"r"(su32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(caddr)
        : "memory");
}
// 2-SM MMA: M = 256 (128 rows in each CTA's TMEM), N = 128 (64 rows of B in each CTA's shared memory).
constexpr uint32_t kIdescPair = (1u << 4) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)((2 * TM) >> 4) << 24);
__device__ __forceinline__ void mma_e4m3_pair(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(kIdescPair), "r"(accumulate)
        : "memory");
}
// Arrives on the mbarrier at this offset in both CTAs of the pair (`mask` = 3) once the MMAs issued
// so far complete.
__device__ __forceinline__ void mma_commit_pair(unsigned long long *bar, unsigned short mask) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            su32(bar)),
        "h"(mask)
        : "memory");
}
__device__ __forceinline__ void mma_commit_pair_local(unsigned long long *bar) {
    asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                 : "memory");
}

constexpr int TNH = TN / 2;                                    // rows of B held by each CTA of a pair
// Two rings of four one-box stages (24 KB each per CTA): with two MMA threads
// the per-stage waits hide behind the other thread's MMAs, and small stages
// keep more of the ring's bytes in flight while one stage is being read.
constexpr int NRING = 2, RSTAGES = 4, P_KBOX = 1, P_SLAB = BOX * P_KBOX;
constexpr uint32_t P_STAGE_A = (uint32_t)P_KBOX * TM * BOX;    // 16 KB
constexpr uint32_t P_STAGE_BYTES = P_STAGE_A + (uint32_t)P_KBOX * TNH * BOX;  // + 8 KB
constexpr int P_EPI_WARP0 = 4;
constexpr int P_NTHREADS = (P_EPI_WARP0 + NEPI) * 32;          // 12 warps

// Ring (and MMA thread) of global diagonal group G: the pattern 0, 1, 1, 0
// repeating.  Group g of a task holds g - 1 slice pairs for g <= s + 1, so
// with s = 12 each thread gets 39 of the 78 pairs (alternating 0, 1 gave 36
// and 42, and the in-order epilogue made the lighter thread wait for the
// other); thread 0 uses accumulators 0 and 3, thread 1 uses 1 and 2.
__device__ __forceinline__ int ring_of_group(int G) { return ((G + 1) >> 1) & 1; }

struct __align__(8) PairBars {
    unsigned long long full[NRING][RSTAGES], empty[NRING][RSTAGES];
    unsigned long long accfull[NBUF], accempty[NBUF];
    unsigned long long tfull[TASK_RING], tempty[TASK_RING];
    unsigned long long drain[NRING];
    long long task[TASK_RING];
    unsigned tmem_base;
    int abort;
};

// Slice GEMM on CTA pairs, one pair per cluster of two CTAs.  A task is
// product r, the tile-row pair tp and two adjacent tile columns 2 tj2,
// 2 tj2 + 1; CTA rp of the pair owns tile row ti = 2 tp + rp, and the pair
// takes the two columns one after the other (the task is published as two
// items).  Every CTA fetches its own tiles from global memory: no copy lands
// in another CTA's shared memory except through the pair's own 2-SM copies.
// Each CTA streams its 128 rows of the left slices and its 64-row half of the
// right slices; the leader's MMA threads issue 256 x 128 x 32 MMAs (tcgen05
// cta_group::2) that read both CTAs' shared memory and accumulate into both
// CTAs' TMEM.  Per SM this stages 3/4 of the operand bytes of the one-CTA
// kernel per MMA flop.
// The tensor pipe queues only about one MMA ahead of its issuing thread, so
// every barrier wait of a lone issuer idles the pipe.  Two issuers therefore
// share the work: diagonal groups are numbered globally (G), group G runs on
// ring ring_of_group(G) (its own producer, its own stages, its own MMA
// thread) and accumulates in TMEM buffer G mod 4; while one MMA thread waits,
// the other issues.
// Warps: 0, 1 producers of rings 0, 1 (both CTAs); 2, 3 MMA threads of rings
// 0, 1 (leader; warp 2 also allocates TMEM in both CTAs); 4-11 epilogue.
// Barriers (same offsets in both CTAs):
//   full[q][k]   leader only: its producer's expect_tx plus both CTAs' bytes
//   empty[q][k]  both: MMA thread q's commit (to both CTAs) once stage k is read
//   accfull[b]   both: the commit (to both CTAs) closing the group in buffer b
//   accempty[b]  leader only: 2 x NEPI epilogue warps (NEPI of them remote)
//   tfull/tempty task ring: ring 0's producer in the leader fetches tasks and
//                publishes them to both CTAs; every other role of both CTAs
//                releases the slot on the leader's tempty.
__global__ void __launch_bounds__(P_NTHREADS, 1)
    ozaki_tc_pair_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_bh,
                         const __grid_constant__ OzParams P) {
    constexpr int CL = 2;  // the pair is the cluster
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = (unsigned char *)(((unsigned long long)smem_raw + 1023ull) & ~1023ull);
    unsigned char *stage_mem = base;  // NRING x RSTAGES x (A 32 KB, B half 16 KB)
    PairBars &B = *reinterpret_cast<PairBars *>(base + NRING * RSTAGES * P_STAGE_BYTES);
    volatile int *abort = &B.abort;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t rank = cluster_rank();
    const int rp = (int)rank & 1;
    const bool lead = rp == 0;        // pair leader: MMA threads, full / accempty barriers
    const bool fetcher = rank == 0;   // fetches tasks and publishes them to the peer
    constexpr uint32_t pair_lead = 0;
    constexpr unsigned short pair_mask = 3;
    const int pairs_m = (P.tiles_m + 1) / 2;
    const int tn2 = (P.tiles_n + 1) / 2;
    const int ptiles = pairs_m * tn2;
    const int nbox = P.Kp / BOX;
    const int nkb = (nbox + P_KBOX - 1) / P_KBOX;
    const int s = P.s;
    // K pieces per slice pair: each piece of each diagonal is a group of its own, so a task streams
    // 1/H of its slice panels at a time (a smaller working set in L2); the host keeps H <= nkb
    const int H = P.kparts < 1 ? 1 : (P.kparts > nkb ? nkb : P.kparts);

    if (tid == 0) {
        for (int q = 0; q < NRING; ++q)
            for (int i = 0; i < RSTAGES; ++i) {
                mbar_init(&B.full[q][i], 1);
                mbar_init(&B.empty[q][i], 1);  // the pair's MMA thread q releases the stage
            }
        for (int i = 0; i < NBUF; ++i) {
            mbar_init(&B.accfull[i], 1);
            mbar_init(&B.accempty[i], 2 * NEPI);
        }
        // consumers of a task slot (counted on the fetcher): the fetcher's producer 1,
        // two MMA threads and NEPI epilogue warps; the peer's two producers and NEPI
        // epilogue warps
        for (int i = 0; i < TASK_RING; ++i) {
            mbar_init(&B.tfull[i], 1);
            mbar_init(&B.tempty[i], (3 + NEPI) + (CL - 1) * (2 + NEPI));
        }
        for (int q = 0; q < NRING; ++q) mbar_init(&B.drain[q], 1);
        B.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&B.tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    cluster_sync();  // the peer's barriers and TMEM exist before any remote use
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = B.tmem_base;

    // Register split: the launch gives every thread 168 registers (384 x 168 =
    // 64512).  The producer / MMA warpgroup (warps 0-3) hands back 112 each
    // and the two epilogue warpgroups take them: 128 x 56 + 256 x 224 = 64512,
    // so the increase can always be granted.  Every warp executes its step
    // unconditionally here.
    if (warp < P_EPI_WARP0) asm volatile("setmaxnreg.dec.sync.aligned.u32 56;" ::: "memory");
    else asm volatile("setmaxnreg.inc.sync.aligned.u32 224;" ::: "memory");

    if (warp < NRING) {
        // ------------------------------------------------------------ producer of ring q (both CTAs)
        const int q = warp;
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"(&map_a) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(&map_bh) : "memory");
            uint32_t stage = 0, sphase = 0;
            int tslot = 0, tseq = 0;
            uint32_t tphase = 0;
            bool issued = false;
            long long pending = -1;  // a lone pair's second item of the current task
            while (!*abort) {
                long long item;  // 2 task + column offset (a lone pair's second column)
                if (fetcher && q == 0) {
                    if (pending >= 0) {
                        item = pending;
                        pending = -1;
                    } else {
                        long long task = (long long)atomicAdd(P.task_counter, 1ull);
                        if (ld_volatile(P.error) != kDevOk || task > P.tasks) task = P.tasks;
                        item = 2 * task;
                        if (task < P.tasks && 2 * ((task % ptiles) % tn2) + 1 < P.tiles_n) pending = item + 1;
                    }
                    if (!mbar_wait_cl(&B.tempty[tslot], tphase ^ 1u, abort, P.error, P.timeout_ns)) break;
                    B.task[tslot] = item;
                    for (int c = 1; c < CL; ++c) st_cluster_s64(mapa(su32(&B.task[tslot]), c), item);
                    mbar_arrive(&B.tfull[tslot]);
                    for (int c = 1; c < CL; ++c) arrive_remote_release(mapa(su32(&B.tfull[tslot]), c));
                } else {
                    if (!mbar_wait_cl(&B.tfull[tslot], tphase, abort, P.error, P.timeout_ns)) break;
                    item = B.task[tslot];
                    if (fetcher) mbar_arrive(&B.tempty[tslot]);
                    else arrive_remote_release(mapa(su32(&B.tempty[tslot]), 0));
                }
                if (++tslot == TASK_RING) {
                    tslot = 0;
                    tphase ^= 1u;
                }
                const long long task = item >> 1;
                if (task >= P.tasks) break;
                const int r = (int)(task / ptiles);
                const int t2 = (int)(task - (long long)r * ptiles);
                const int tp = t2 / tn2;
                const int tj = 2 * (t2 - tp * tn2) + (int)(item & 1);
                const int ti = 2 * tp + rp;
                bool ok = true;
                for (int V = 0; V < H * s && ok; ++V) {
                    if (ring_of_group(tseq * H * s + V) != q) continue;
                    const int g = 2 + V % s, kh = V / s;
                    const int kb0 = kh * nkb / H, kb1 = (kh + 1) * nkb / H;
                    for (int ta = max(1, g - s); ta <= min(s, g - 1) && ok; ++ta)
                        for (int kb = kb0; kb < kb1; ++kb) {
                            if (!mbar_wait(&B.empty[q][stage], sphase ^ 1u, abort, P.error, P.timeout_ns)) {
                                ok = false;
                                break;
                            }
                            unsigned char *sa = stage_mem + (q * RSTAGES + stage) * P_STAGE_BYTES;
                            unsigned char *sb = sa + P_STAGE_A;
                            const int boxes = min(P_KBOX, nbox - kb * P_KBOX);
                            const uint32_t full_lead = mapa(su32(&B.full[q][stage]), pair_lead);
                            if (lead) mbar_expect_tx(&B.full[q][stage], (uint32_t)(2 * boxes * (TM + TNH) * BOX));
                            const int ya = (r * s + (ta - 1)) * P.Mp + ti * TM;
                            const int yb = (r * s + (g - ta - 1)) * P.Mp + tj * TN + rp * TNH;
                            for (int bx = 0; bx < boxes; ++bx) {
                                const int x = (kb * P_KBOX + bx) * BOX;
                                tma_load_2d_pair(sa + bx * TM * BOX, &map_a, x, ya, full_lead);
                                tma_load_2d_pair(sb + bx * TNH * BOX, &map_bh, x, yb, full_lead);
                            }
                            issued = true;
                            if (++stage == RSTAGES) {
                                stage = 0;
                                sphase ^= 1u;
                            }
                        }
                }
                if (!ok) break;
                ++tseq;
            }
            if (*abort && issued) {
                // copies signal the leader's barriers, which this thread cannot
                // wait on: give any copy still in flight time to land
                const unsigned long long t0 = global_ns();
                while ((long long)(global_ns() - t0) < 100000) {
                }
            }
        }
    } else if (warp < 2 * NRING) {
        // ------------------------------------------------------------ MMA thread of ring q (leader CTA)
        const int q = warp - NRING;
        if (lead && lane == 0) {
            uint32_t stage = 0, sphase = 0;
            int tslot = 0, tseq = 0;
            uint32_t tphase = 0;
            const uint32_t sbase = su32(stage_mem) + (uint32_t)(q * RSTAGES) * P_STAGE_BYTES;
            bool any = false;
            while (!*abort) {
                if (!mbar_wait_cl(&B.tfull[tslot], tphase, abort, P.error, P.timeout_ns)) break;
                const long long task = B.task[tslot] >> 1;
                if (fetcher) mbar_arrive(&B.tempty[tslot]);
                else arrive_remote_release(mapa(su32(&B.tempty[tslot]), 0));
                if (++tslot == TASK_RING) {
                    tslot = 0;
                    tphase ^= 1u;
                }
                if (task >= P.tasks) break;
                bool ok = true;
                for (int V = 0; V < H * s && ok; ++V) {
                    const int G = tseq * H * s + V;
                    if (ring_of_group(G) != q) continue;
                    const int g = 2 + V % s, kh = V / s;
                    const int kb0 = kh * nkb / H, kb1 = (kh + 1) * nkb / H;
                    const uint32_t buf = (uint32_t)(G % NBUF), bphase = (uint32_t)((G / NBUF) & 1);
                    if (!mbar_wait(&B.accempty[buf], bphase ^ 1u, abort, P.error, P.timeout_ns)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t dtm = tmem + buf * TN;
                    bool first = true;
                    for (int ta = max(1, g - s); ta <= min(s, g - 1) && ok; ++ta)
                        for (int kb = kb0; kb < kb1; ++kb) {
                            if (!mbar_wait(&B.full[q][stage], sphase, abort, P.error, P.timeout_ns)) {
                                ok = false;
                                break;
                            }
                            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                            const uint32_t sa = sbase + stage * P_STAGE_BYTES;
                            const uint64_t da = desc_sw128(sa), db = desc_sw128(sa + P_STAGE_A);
                            const int kmma = min(P_KBOX, nbox - kb * P_KBOX) * (BOX / 32);
#pragma unroll
                            for (int k = 0; k < P_SLAB / 32; ++k) {
                                if (k >= kmma) break;
                                // 32-byte K step inside a box; boxes 16 KB (A) and 8 KB (B half) apart
                                const uint64_t adv = (uint64_t)(((k % (BOX / 32)) * 32) >> 4);
                                const uint64_t boxa = (uint64_t)(((k / (BOX / 32)) * TM * BOX) >> 4);
                                const uint64_t boxb = (uint64_t)(((k / (BOX / 32)) * TNH * BOX) >> 4);
                                mma_e4m3_pair(dtm, da + boxa + adv, db + boxb + adv, first ? 0u : 1u);
                                first = false;
                            }
                            mma_commit_pair(&B.empty[q][stage], pair_mask);
                            any = true;
                            if (++stage == RSTAGES) {
                                stage = 0;
                                sphase ^= 1u;
                            }
                        }
                    if (!ok) break;
                    mma_commit_pair(&B.accfull[buf], pair_mask);
                }
                if (!ok) break;
                ++tseq;
            }
            if (any) {
                // all MMAs complete before either CTA releases TMEM or shared memory
                mma_commit_pair_local(&B.drain[q]);
                const unsigned long long t0 = global_ns();
                while (!mbar_test(&B.drain[q], 0) && (long long)(global_ns() - t0) < P.timeout_ns) {
                }
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue (both CTAs)
        int tslot = 0, tseq = 0;
        uint32_t tphase = 0;
        while (!*abort) {
            if (!mbar_wait_cl(&B.tfull[tslot], tphase, abort, P.error, P.timeout_ns)) break;
            const long long item = B.task[tslot];
            const long long task = item >> 1;
            __syncwarp();
            if (lane == 0) {
                if (fetcher) mbar_arrive(&B.tempty[tslot]);
                else arrive_remote_release(mapa(su32(&B.tempty[tslot]), 0));
            }
            if (++tslot == TASK_RING) {
                tslot = 0;
                tphase ^= 1u;
            }
            if (task >= P.tasks) break;
            const int r = (int)(task / ptiles);
            const int t2 = (int)(task - (long long)r * ptiles);
            const int tp = t2 / tn2;
            const int tj = 2 * (t2 - tp * tn2) + (int)(item & 1);
            const int ti = 2 * tp + rp;
            if (!epilogue_tile<P_EPI_WARP0>(P, B.accfull, abort, tmem, r, ti, tj, ti < P.tiles_m && tj < P.tiles_n,
                                            tseq * H * s, H, [&](uint32_t b) {
                                                if (lead) mbar_arrive(&B.accempty[b]);
                                                else arrive_remote_relaxed(mapa(su32(&B.accempty[b]), pair_lead));
                                            }))
                break;
            ++tseq;
        }
    }

    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    cluster_sync();  // neither CTA leaves while the pair's MMAs or copies may touch it
    if (warp == 2)
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

constexpr size_t kSmemBytes = 1024 + STAGES * STAGE_BYTES + sizeof(Bars);
constexpr size_t kPairSmemBytes = 1024 + NRING * RSTAGES * P_STAGE_BYTES + sizeof(PairBars);

}  // namespace

cudaError_t launch_ozaki_tc(const CUtensorMap &map_a, const CUtensorMap &map_b, const OzParams &P, int grid,
                            cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e =
            cudaFuncSetAttribute(ozaki_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    ozaki_tc_kernel<<<grid, NTHREADS, kSmemBytes, s>>>(map_a, map_b, P);
    return cudaGetLastError();
}

namespace {
bool pair_attr() {
    static int state = 0;  // 0 unset, 1 ok, -1 failed
    if (state == 0)
        state = cudaFuncSetAttribute(ozaki_tc_pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kPairSmemBytes) == cudaSuccess ? 1 : -1;
    if (state < 0) cudaGetLastError();
    return state > 0;
}

// clusters of two CTAs (one pair each)
cudaLaunchConfig_t pair_config(cudaLaunchAttribute *at, int ctas, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3((unsigned)ctas);
    cfg.blockDim = dim3(P_NTHREADS);
    cfg.dynamicSmemBytes = kPairSmemBytes;
    cfg.stream = s;
    cfg.attrs = at;
    return cfg;
}
}  // namespace

cudaError_t launch_ozaki_tc_pair(const CUtensorMap &map_a, const CUtensorMap &map_bh, const OzParams &P, int ctas,
                                 cudaStream_t s) {
    if (!pair_attr()) return cudaErrorInvalidValue;
    cudaLaunchAttribute at[1];
    cudaLaunchConfig_t cfg = pair_config(at, ctas, s);
    return cudaLaunchKernelEx(&cfg, ozaki_tc_pair_kernel, map_a, map_bh, P);
}

int ozaki_tc_max_pairs() {
    static int cached = -1;
    if (cached >= 0) return cached;
    if (!pair_attr()) return 0;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaLaunchAttribute at[1];
    cudaLaunchConfig_t cfg = pair_config(at, sms / 2 * 2, nullptr);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, ozaki_tc_pair_kernel, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cached = n;
    return n;
}

}  // namespace fmm
