// fmm_gemm_noalloc: C = A * B without allocating any memory.
//
// Some callers cannot allocate device memory at all: code running inside a
// custom allocator or memory-pool callback, processes whose device memory is
// fully reserved up front by a framework, and hard real-time paths where a
// cudaMalloc (which may synchronize the device) is not allowed.  For them this
// entry point runs the fused schedule of the FP64 leaf kernel with every piece
// of scratch state -- the per-call ordering counters, the task counter, the
// error word and the flattened coefficient tables -- in one file-scope
// __device__ array of fixed size, and plans on the host with fixed-size static
// buffers as well (no heap, no cudaMalloc/cudaFree, no allocating library
// call).  The array exists on every GPU that loads the library and stays
// allocated until the process exits.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "fmm.h"
#include "fmm_internal.h"

namespace {

constexpr size_t kScratchBytes = (size_t)FMM_NOALLOC_SCRATCH_BYTES;

// The scratch array.  In host code its name is only a host-side stand-in, so
// the device address is fetched with cudaGetSymbolAddress (once per device).
static __device__ __align__(256) unsigned char g_fmm_noalloc_scratch[kScratchBytes];

// Host image of the scratch layout (tables and geometry), rebuilt per call
// under g_mutex and copied to the device with one cudaMemcpyAsync.
static unsigned char g_host_image[kScratchBytes];
static std::mutex g_mutex;

constexpr int kMaxDevices = 64;
static void *g_dev_ptr[kMaxDevices];
static bool g_dev_ready[kMaxDevices];

// Testing hooks for the next calls (fmm_noalloc_set_debug): the bound on
// every device-side wait, and whether one ordering counter is poisoned.
static double g_wait_timeout_s = 5.0;
static int g_poison_chain = 0;

constexpr int kMaxP = 4;                     // split factor
constexpr int kMaxDepth = 4;                 // recursion levels
constexpr long long kMaxBlocks = 1LL << 16;  // (p^depth)^2 C blocks

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

long long ipow(long long b, int e) {
    long long r = 1;
    while (e-- > 0) r *= b;
    return r;
}

// Coefficient bounds that keep the checks and the flattened tables exact:
// p^2 R below 2^28 (int indices), R max|U| max|V| max|W| below 2^62 (every
// partial Brent sum fits int64), and max|X|^depth below 2^31 for each table
// (flattened coefficients are products of `depth` entries and stay int32).
bool coefficients_in_range(const fmm_algo_t *a, int depth) {
    const long long cnt = (long long)a->p * a->p * a->R;
    if (cnt >= (1LL << 28)) return false;
    double mx[3] = {0, 0, 0};
    const int32_t *X[3] = {a->U, a->V, a->W};
    for (int t = 0; t < 3; ++t)
        for (long long x = 0; x < cnt; ++x) {
            const double v = X[t][x] < 0 ? -(double)X[t][x] : (double)X[t][x];
            if (v > mx[t]) mx[t] = v;
        }
    if ((double)a->R * mx[0] * mx[1] * mx[2] >= 4611686018427387904.0) return false;  // 2^62
    for (int t = 0; t < 3; ++t) {
        double pw = 1.0;
        for (int l = 0; l < depth; ++l) pw *= mx[t];
        if (pw >= 2147483648.0) return false;  // 2^31
    }
    return true;
}

// Exact Brent check without heap storage: every one of the p^6 equations.
bool brent_ok(const fmm_algo_t *a) {
    const int p = a->p, R = a->R;
    for (int i = 0; i < p; ++i)
        for (int j = 0; j < p; ++j)
            for (int j2 = 0; j2 < p; ++j2)
                for (int k = 0; k < p; ++k)
                    for (int i2 = 0; i2 < p; ++i2)
                        for (int k2 = 0; k2 < p; ++k2) {
                            long long s = 0;
                            for (int r = 0; r < R; ++r)
                                s += (long long)a->U[(i * p + j) * R + r] * a->V[(j2 * p + k) * R + r] *
                                     a->W[(i2 * p + k2) * R + r];
                            if (s != ((j == j2 && i == i2 && k == k2) ? 1 : 0)) return false;
                        }
    return true;
}

// Writes the flattened column r of X (depth levels, first level outermost)
// into out[] as {block, coefficient}, sorted by block like the planner of
// fmm_plan_create, and returns its length, or -1 if it exceeds cap.
int flatten_column(const int32_t *X, int p, int R, int depth, long long r, int2 *out, int cap) {
    int digit[kMaxDepth];
    long long rr = r;
    for (int l = depth - 1; l >= 0; --l) {
        digit[l] = (int)(rr % R);
        rr /= R;
    }
    int nzx[kMaxDepth][kMaxP * kMaxP], nzc[kMaxDepth][kMaxP * kMaxP], cnt[kMaxDepth];
    for (int l = 0; l < depth; ++l) {
        cnt[l] = 0;
        for (int x = 0; x < p * p; ++x) {
            const int32_t v = X[x * R + digit[l]];
            if (v) {
                nzx[l][cnt[l]] = x;
                nzc[l][cnt[l]] = v;
                ++cnt[l];
            }
        }
        if (cnt[l] == 0) return 0;
    }
    const int P = (int)ipow(p, depth);
    int idx[kMaxDepth] = {0};
    int n = 0;
    while (true) {
        int row = 0, col = 0, coef = 1;
        for (int l = 0; l < depth; ++l) {
            const int x = nzx[l][idx[l]];
            row = row * p + x / p;
            col = col * p + x % p;
            coef *= nzc[l][idx[l]];
        }
        if (n >= cap) return -1;
        out[n++] = make_int2(row * P + col, coef);
        int l = depth - 1;
        while (l >= 0 && ++idx[l] == cnt[l]) idx[l--] = 0;
        if (l < 0) break;
    }
    for (int a = 1; a < n; ++a) {  // insertion sort by block index
        const int2 e = out[a];
        int b = a - 1;
        while (b >= 0 && out[b].x > e.x) {
            out[b + 1] = out[b];
            --b;
        }
        out[b + 1] = e;
    }
    return n;
}

// Device address of the scratch array on the current device; the first call
// on a device looks it up (this set-up should happen before any capture).
cudaError_t scratch_ptr(void **ptr) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    if (!g_dev_ready[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_fmm_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_dev_ptr[dev] = p;
        g_dev_ready[dev] = true;
    }
    *ptr = g_dev_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" fmm_status_t fmm_gemm_noalloc(int64_t n, const fmm_algo_t *algo, int depth, const double *A,
                                         const double *B, double *C, void *stream) {
    if (!algo || !A || !B || !C || n < 1 || depth < 0 || algo->p < 2 || algo->R < 1 || !algo->U || !algo->V ||
        !algo->W)
        return FMM_ERR_INVALID;
    if (n > (1LL << 31) / 2) return FMM_ERR_UNSUPPORTED;
    const int p = algo->p, R0 = algo->R;
    if (p > kMaxP || depth > kMaxDepth) return FMM_ERR_SCRATCH_LIMIT;
    if (!coefficients_in_range(algo, depth)) return FMM_ERR_UNSUPPORTED;
    if (!brent_ok(algo)) return FMM_ERR_BRENT;
    const long long P = ipow(p, depth), Rt = ipow(R0, depth);
    if (P > n) return FMM_ERR_INVALID;
    if (P * P > kMaxBlocks || Rt > (1LL << 24)) return FMM_ERR_SCRATCH_LIMIT;

    const long long m = n / P, nc = P * m, q = n - nc;
    const int tiles_m = (int)((m + fmm::kBM - 1) / fmm::kBM), tiles_n = (int)((m + fmm::kBN - 1) / fmm::kBN);
    const long long tiles = (long long)tiles_m * tiles_n;

    std::lock_guard<std::mutex> lock(g_mutex);
    void *dev = nullptr;
    if (scratch_ptr(&dev) != cudaSuccess) return FMM_ERR_CUDA;

    // Layout: [error int][pad][task counter u64][chain counters] | geometry | tables.
    size_t off = align256(16 + (size_t)(P * P * tiles) * sizeof(unsigned));
    const size_t counters_bytes = off;
    if (counters_bytes > kScratchBytes) return FMM_ERR_SCRATCH_LIMIT;
    const size_t o_geom = off;
    off = align256(off + sizeof(fmm::F64Geom));
    const size_t o_uptr = off;
    off = align256(off + (size_t)(Rt + 1) * sizeof(int));
    const size_t o_vptr = off;
    off = align256(off + (size_t)(Rt + 1) * sizeof(int));
    const size_t o_wptr = off;
    off = align256(off + (size_t)(Rt + 1) * sizeof(int));
    const size_t o_wrow = off;
    off = align256(off + (size_t)(P * P) * sizeof(int));
    if (off > kScratchBytes) return FMM_ERR_SCRATCH_LIMIT;
    {  // whole layout, from the flattened nonzero counts nnz(X)^depth
        long long nz[3] = {0, 0, 0};
        for (long long x = 0; x < (long long)p * p * R0; ++x) {
            nz[0] += algo->U[x] != 0;
            nz[1] += algo->V[x] != 0;
            nz[2] += algo->W[x] != 0;
        }
        double need = (double)off;
        need += (double)ipow(nz[0], depth) * sizeof(int2) + 256.0;
        need += (double)ipow(nz[1], depth) * sizeof(int2) + 256.0;
        need += (double)ipow(nz[2], depth) * sizeof(int4);
        if (need > (double)kScratchBytes) return FMM_ERR_SCRATCH_LIMIT;
    }
    unsigned char *img = g_host_image;
    int *u_ptr = (int *)(img + o_uptr), *v_ptr = (int *)(img + o_vptr), *w_ptr = (int *)(img + o_wptr);
    int *w_row = (int *)(img + o_wrow);
    std::memset(w_row, 0, (size_t)(P * P) * sizeof(int));

    // Entry arrays follow; their sizes are only known while flattening, so
    // each is written into the space that remains and checked as it grows.
    const size_t o_uent = off;
    int2 col[fmm::kMaxTerms];
    size_t used = 0;
    const size_t room = kScratchBytes - off;
    u_ptr[0] = 0;
    for (long long r = 0; r < Rt; ++r) {
        const int k = flatten_column(algo->U, p, R0, depth, r, col, fmm::kMaxTerms);
        if (k < 0) return FMM_ERR_UNSUPPORTED;
        if (used + (size_t)k * sizeof(int2) > room) return FMM_ERR_SCRATCH_LIMIT;
        std::memcpy(img + o_uent + used, col, (size_t)k * sizeof(int2));
        used += (size_t)k * sizeof(int2);
        u_ptr[r + 1] = u_ptr[r] + k;
    }
    off = align256(o_uent + used);
    const size_t o_vent = off;
    used = 0;
    if (off > kScratchBytes) return FMM_ERR_SCRATCH_LIMIT;
    const size_t room_v = kScratchBytes - off;
    v_ptr[0] = 0;
    for (long long r = 0; r < Rt; ++r) {
        const int k = flatten_column(algo->V, p, R0, depth, r, col, fmm::kMaxTerms);
        if (k < 0) return FMM_ERR_UNSUPPORTED;
        if (used + (size_t)k * sizeof(int2) > room_v) return FMM_ERR_SCRATCH_LIMIT;
        std::memcpy(img + o_vent + used, col, (size_t)k * sizeof(int2));
        used += (size_t)k * sizeof(int2);
        v_ptr[r + 1] = v_ptr[r] + k;
    }
    off = align256(o_vent + used);
    const size_t o_went = off;
    used = 0;
    if (off > kScratchBytes) return FMM_ERR_SCRATCH_LIMIT;
    const size_t room_w = kScratchBytes - off;
    w_ptr[0] = 0;
    for (long long r = 0; r < Rt; ++r) {
        const int k = flatten_column(algo->W, p, R0, depth, r, col, fmm::kMaxTerms);
        if (k < 0) return FMM_ERR_UNSUPPORTED;
        if (used + (size_t)k * sizeof(int4) > room_w) return FMM_ERR_SCRATCH_LIMIT;
        int4 *dst = (int4 *)(img + o_went + used);
        for (int e = 0; e < k; ++e) dst[e] = make_int4(col[e].x, col[e].y, w_row[col[e].x]++, 0);
        used += (size_t)k * sizeof(int4);
        w_ptr[r + 1] = w_ptr[r] + k;
    }
    const size_t total = o_went + used;

    unsigned char *dbase = (unsigned char *)dev;
    fmm::F64Geom g{};
    g.n = n; g.m = m; g.n_core = nc;
    g.ld_src_a = n; g.ld_src_b = n;
    g.sub_stride_a = 0; g.sub_stride_b = 0;
    g.P = (int)P; g.P_src = (int)P; g.R_src = (int)Rt; g.nsub = 1;
    g.tiles_m = tiles_m; g.tiles_n = tiles_n;
    g.u_ptr = (const int *)(dbase + o_uptr);
    g.u_ent = (const int2 *)(dbase + o_uent);
    g.v_ptr = (const int *)(dbase + o_vptr);
    g.v_ent = (const int2 *)(dbase + o_vent);
    g.w_ptr = (const int *)(dbase + o_wptr);
    g.w_ent = (const int4 *)(dbase + o_went);
    g.w_row_nnz = (const int *)(dbase + o_wrow);
    g.tasks_core = tiles * Rt;
    if (q > 0) {
        g.rb_tm = (int)((nc + fmm::kBM - 1) / fmm::kBM);
        g.rb_tn = (int)((q + fmm::kBN - 1) / fmm::kBN);
        g.bb_tm = (int)((q + fmm::kBM - 1) / fmm::kBM);
        g.bb_tn = (int)((n + fmm::kBN - 1) / fmm::kBN);
        g.tasks_right = (long long)g.rb_tm * g.rb_tn;
        g.tasks_bottom = (long long)g.bb_tm * g.bb_tn;
        g.tasks_rankq = P * P * tiles;
    }
    std::memcpy(img + o_geom, &g, sizeof(g));

    cudaStream_t st = (cudaStream_t)stream;
    // The tables are copied from g_host_image, which the next call rewrites: a
    // copy recorded into a graph would read whatever the last call left there.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return FMM_ERR_CUDA;
    if (cap != cudaStreamCaptureStatusNone) return FMM_ERR_UNSUPPORTED;
    // Tables and geometry (the source is copied out before the call returns),
    // then the counters and the error word, which must start at zero on every call.
    if (cudaMemcpyAsync(dbase + o_geom, img + o_geom, total - o_geom, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return FMM_ERR_CUDA;
    if (cudaMemsetAsync(dbase, 0, counters_bytes, st) != cudaSuccess) return FMM_ERR_CUDA;
    if (g_poison_chain && cudaMemsetAsync(dbase + 16, 0xFF, sizeof(unsigned), st) != cudaSuccess)
        return FMM_ERR_CUDA;

    fmm::F64Launch<1> L{};
    L.nprobs = 1;
    L.total_tasks = g.tasks_core + g.tasks_right + g.tasks_bottom + g.tasks_rankq;
    L.task_counter = (unsigned long long *)(dbase + 8);
    L.error = (int *)dbase;
    L.timeout_ns = (long long)(g_wait_timeout_s * 1e9);
    fmm::F64Problem &pr = L.probs[0];
    pr.g = (const fmm::F64Geom *)(dbase + o_geom);
    pr.A = A; pr.B = B; pr.SA = A; pr.SB = B; pr.C = C;
    pr.chain = (unsigned *)(dbase + 16);
    pr.task_begin = 0;
    pr.alpha = 1.0;
    pr.alpha_peel = 1.0;
    pr.beta = 0.0;
    int sms = 0, devno = 0;
    cudaGetDevice(&devno);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, devno);
    const int per_sm = fmm::f64_kernel_ctas_per_sm();
    if (per_sm <= 0) return FMM_ERR_CUDA;
    long long grid = (long long)sms * per_sm;
    if (grid > L.total_tasks) grid = L.total_tasks;
    if (grid < 1) grid = 1;
    return fmm::launch_f64_single(L, (int)grid, st) == cudaSuccess ? FMM_OK : FMM_ERR_CUDA;
}

extern "C" fmm_status_t fmm_noalloc_sync_status(void *stream) {
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return FMM_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mutex);
    // offset 0 of the array on the current device holds the last call's error word
    int err = 0;
    if (cudaMemcpyFromSymbol(&err, g_fmm_noalloc_scratch, sizeof(int), 0, cudaMemcpyDeviceToHost) != cudaSuccess)
        return FMM_ERR_CUDA;
    if (err != fmm::kDevOk) {
        const int zero = 0;
        if (cudaMemcpyToSymbol(g_fmm_noalloc_scratch, &zero, sizeof(int), 0, cudaMemcpyHostToDevice) != cudaSuccess)
            return FMM_ERR_CUDA;
        return FMM_ERR_TIMEOUT;
    }
    return FMM_OK;
}

extern "C" fmm_status_t fmm_noalloc_set_debug(double wait_timeout_s, int poison_chain) {
    if (!(wait_timeout_s > 0.0) || wait_timeout_s > 3600.0) return FMM_ERR_INVALID;
    std::lock_guard<std::mutex> lock(g_mutex);
    g_wait_timeout_s = wait_timeout_s;
    g_poison_chain = poison_chain ? 1 : 0;
    return FMM_OK;
}
