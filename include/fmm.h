/*
 * fmm.h -- C ABI of a GB300 (sm_103a) library for recursive bilinear fast
 * matrix multiplication in FP64, after D'Alberto, "Strassen's Matrix
 * Multiplication Algorithm Is Still Faster" (arXiv 2312.12732).
 *
 * The operation is C = A * B for square n x n binary64 matrices (Section 2,
 * definition of the matrix product).  Section 3 states it as C = alpha A B;
 * fmm_gemm overwrites C with A B, and fmm_gemm_ex computes alpha A B + beta C.
 * Double-complex operands are supported through the FMM_C128 dtypes
 * (Section 1 lists double complex among the deployable types).  A bilinear
 * algorithm <p,p,p;R> is given by three integer p^2 x R matrices (U, V, W),
 * or by integer numerators over one denominator per matrix
 * (fmm_algo_rational_t; Section 2 allows non-integer coefficients): with the
 * operands split by the factor p into row-major blocks A_0 .. A_{p^2-1}
 * (Section 2, the single-index partition), product r is
 *     P_r = S_r * T_r,   S_r = sum_i U[i][r] A_i,   T_r = sum_j V[j][r] B_j,
 * and block l of C is C_l = sum_r W[l][r] P_r (Section 2, equation
 * `strassen`; the library names the left combination S and the right one T).
 * W indexes the blocks of C in row-major order.  `depth` levels of recursion
 * (Section 2, recursion with the same split factor) are flattened into the
 * Kronecker power of (U, V, W) with blocks re-indexed row-major over the
 * p^depth x p^depth grid (Section 2, the Kronecker-product composition).
 *
 * Conventions for every entry point:
 *   - matrices are row-major and contiguous (leading dimension n);
 *   - device pointers refer to memory of the current CUDA device; host
 *     pointers are ordinary (pageable or pinned) host memory;
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default);
 *   - calls that launch GPU work are asynchronous on `stream` unless stated;
 *   - the library never takes ownership of caller memory;
 *   - every function returns an fmm_status_t; on error no GPU work was
 *     enqueued unless the error is FMM_ERR_CUDA from a launch.
 *
 * Environment variables (none is needed; each is read when it applies):
 *   FMM_LOG          1: one line on stderr per plan created or rejected (size,
 *                    algorithm shape, depth, dtype, leaf size, product range,
 *                    materialized levels, tile, tasks, workspace, or the
 *                    reason of the rejection); 2: also one line per
 *                    multiplication enqueued.  Read at every call.
 *   FMM_TILE_N       64 or 128: the FP64 leaf tile width when a plan does not
 *                    set one (read at plan creation).
 *   FMM_OZAKI_ENGINE see FMM_F64_OZAKI (read at plan creation).
 *   FMM_OZAKI_POSTADD flat: an FMM_F64_OZAKI plan of depth 2 or more applies
 *                    its post-additions in the flattened form (every C block
 *                    summed over all leaf products in ascending order)
 *                    instead of level by level (read at plan creation).
 *   FMM_OZAKI_KPARTS k (1..8): the CTA-pair slice GEMM of FMM_F64_OZAKI plans
 *                    splits each slice pair's K range into k pieces, each
 *                    accumulated on its own (default K / 1024 pieces, at least
 *                    1 and at most 4; read at plan creation).
 *   FMM_F64_POSTADD  fused or levels: the post-additions of an FMM_F64 plan
 *                    whose options leave them to the planner (see
 *                    fmm_plan_options_t.post_additions; read at plan creation).
 *   FMM_FORCE_DEPTH  d: fmm_autotune times only depth-d candidates.
 */
#ifndef FMM_H_
#define FMM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FMM_OK = 0,
    FMM_ERR_INVALID = 1,     /* bad argument: NULL pointer, n < 1, p < 2, R < 1, leaf size < 1 */
    FMM_ERR_BRENT = 2,       /* (U, V, W) fails the Brent equations in exact integer arithmetic */
    FMM_ERR_UNSUPPORTED = 3, /* valid request the library does not implement (dtype, limits) */
    FMM_ERR_OOM = 4,         /* a device or host allocation failed */
    FMM_ERR_CUDA = 5,        /* a CUDA runtime call or kernel launch failed */
    FMM_ERR_TIMEOUT = 6,     /* a bounded device-side wait gave up (reported by fmm_sync_status) */
    FMM_ERR_NOT_FOUND = 7,   /* unknown built-in algorithm name */
    FMM_ERR_SCRATCH_LIMIT = 8 /* fmm_gemm_noalloc: request needs more than its static scratch */
} fmm_status_t;

typedef enum {
    FMM_F64 = 0,       /* binary64 operands, FP64 tensor-core (DMMA) leaf products */
    FMM_F64_OZAKI = 1, /* binary64 operands; S_r/T_r formed in FP64, leaf products emulated from
                          e4m3 slices (Ozaki scheme) on the tensor cores, post-additions in FP64.
                          Read at plan creation: FMM_OZAKI_ENGINE=tc1 or mma_sync selects the
                          one-CTA tcgen05 or the mma.sync slice GEMM instead of CTA pairs */
    /* Double complex (Section 1 lists double complex among the types the
     * algorithms deploy to): A, B, C are n x n row-major arrays of interleaved
     * (re, im) binary64 pairs, 16-byte aligned, so each pointer addresses 2 n^2
     * doubles.  The plan holds an FMM_F64 plan of the same algorithm and depth
     * and splits the operands into real planes. */
    FMM_C128 = 2,      /* four real fast products: Re C = Re A Re B - Im A Im B,
                          Im C = Re A Im B + Im A Re B (each part as accurate as a real product) */
    FMM_C128_3M = 3,   /* three real fast products (Gauss): T1 = Re A Re B, T2 = Im A Im B,
                          T3 = (Re A + Im A)(Re B + Im B); Re C = T1 - T2, Im C = (T3 - T1) - T2;
                          25% fewer products, error bounded normwise rather than per part */
    FMM_F32 = 4        /* binary32 operands (Section 1 lists single precision among the deployable
                          types), run through fmm_gemm_f32_ex only: A and B widen exactly to binary64,
                          the product runs as an FMM_F64_OZAKI plan with 6 slices by default (30 bits
                          for 24-bit significands; opts->ozaki_slices overrides), and C is rounded to
                          nearest binary32 once */
} fmm_dtype_t;

/* A bilinear algorithm <p,p,p;R>.  U, V, W are row-major p^2 x R int32
 * arrays (entry [i][r] at index i*R + r).  The library copies them. */
typedef struct {
    int p;
    int R;
    const int32_t *U;
    const int32_t *V;
    const int32_t *W;
} fmm_algo_t;

/* A bilinear algorithm <p,p,p;R> with rational coefficients (Section 2: the
 * coefficients of a, b, c need not be integers): entry [i][r] of U is
 * U[i*R + r] / den_u, likewise V over den_v and W over den_w.  Numerators are
 * row-major p^2 x R int32 arrays; each denominator is one positive int32
 * common to its matrix.  The library copies the numerators. */
typedef struct {
    int p;
    int R;
    const int32_t *U;
    const int32_t *V;
    const int32_t *W;
    int32_t den_u, den_v, den_w;
} fmm_algo_rational_t;

typedef struct fmm_plan fmm_plan_t;

/* How the pre-additions S_r / T_r of the recursion levels are formed.
 *   FMM_SCHED_AUTO   -- the planner chooses (the default);
 *   FMM_SCHED_FUSED  -- every level is combined on the fly while staging the
 *                       leaf operands (no S_r / T_r in device memory);
 *   FMM_SCHED_HYBRID -- the top `materialize_levels` levels are formed level
 *                       by level in plan workspace by an elementwise pass,
 *                       the remaining levels are fused into staging.
 * The post-additions C_l = sum_r W[l][r] P_r of an FMM_F64 plan are fused into
 * the leaf kernel's epilogue or run from stored leaf products
 * (fmm_plan_options_t.post_additions); the emulated leaf (FMM_F64_OZAKI,
 * FMM_F32) always stores its leaf products and sums them in separate kernels:
 * at depth 1 in ascending product order per C block, from depth 2 level by
 * level as the recursion forms the blocks (the passes of the stored FMM_F64
 * form; FMM_OZAKI_POSTADD=flat selects the flattened order instead). */
typedef enum { FMM_SCHED_AUTO = 0, FMM_SCHED_FUSED = 1, FMM_SCHED_HYBRID = 2 } fmm_schedule_t;

/* Optional knobs for fmm_plan_create_ex.  Zero-initialise, then set fields;
 * a zero field means "library default". */
typedef struct {
    fmm_schedule_t schedule;
    int materialize_levels;  /* FMM_SCHED_HYBRID: 0 .. depth */
    int ozaki_slices;        /* FMM_F64_OZAKI and FMM_F32: slices per operand, 2..12
                                (default 12 for FMM_F64_OZAKI: 60 bits, within 2x of the
                                FP64 path's error on uniform, normal and wide-exponent
                                inputs; default 6 for FMM_F32: 30 bits) */
    double wait_timeout_s;   /* bound on every device-side wait (default 5 s) */
    int debug_poison_chain;  /* testing only: 1 = after the per-call reset, set one
                                post-addition ordering counter to a value no task
                                writes, so that its waiters time out */
    int record_kernel_time;  /* 1 = record CUDA events around each call's work on
                                its stream (see fmm_plan_last_kernel_ms) */
    int tile_n;              /* FMM_F64 leaf tile width: 128 (one 8-warp CTA per SM)
                                or 64 (two 4-warp CTAs per SM); 0 = planner's choice */
    /* Product sharding (Section 2: the R^depth leaf products are independent,
     * each can be computed on its own).  shard_count > 1 makes an FMM_F64
     * plan compute only shard `shard_index` of its leaf products: the
     * R^materialized_levels sub-problems are split into shard_count
     * contiguous ranges of sizes differing by at most one
     * (fmm_shard_range), and the plan's C is the sum over its own products
     * of W[l][r] P_r, zero elsewhere; the shard whose range starts at product
     * 0 also runs the peel fix-ups of a non-divisible n.  The full product is
     * the elementwise sum of the shard_count partial C's (for example an
     * all-reduce across GPUs, one shard per GPU).  A sharded plan takes
     * beta = 0 only and cannot join a batched launch.  0 or 1 = the whole
     * product.  FMM_ERR_UNSUPPORTED for another dtype, or for more shards
     * than sub-problems (a fused schedule has one); FMM_ERR_INVALID for
     * shard_index outside [0, shard_count). */
    int shard_count;
    int shard_index;
    /* FMM_F64 post-additions (Section 2: C_l = sum_r W[l][r] P_r, or level by
     * level as the recursion forms the blocks):
     *   0 -- the planner's choice (FMM_F64_POSTADD=fused or levels overrides it):
     *        stored when the fused form's adds, (nnz(W flattened) - p^(2 depth)) m^2,
     *        reach 0.4 % of the leaf flops 2 R^depth m^3 and the buffers take at
     *        most a quarter of the free device memory, fused otherwise;
     *   1 -- fused into the leaf kernel's epilogue: each leaf tile is added into
     *        every C block of its W column, in ascending product order;
     *   2 -- stored: each leaf product P_r is written once to plan workspace
     *        (R^depth m^2 doubles, plus an intermediate buffer), then separate
     *        passes sum W's Kronecker factors level by level, innermost first
     *        (two 2 x 2 factors per pass where both have at most 8 products),
     *        the last pass writing C = alpha sum + beta C; a non-divisible n's
     *        rank-q fix-ups run after it.  Fewer FP64 operations than the fused
     *        sums (for Strassen at depth d, 12^d - 4^d adds per position of a
     *        leaf block become 8 (7^d - 4^d) / 3: 20480 and 5720 at depth 4),
     *        and no ordering waits.  FMM_ERR_UNSUPPORTED with
     *        shard_count > 1, debug_poison_chain, or a factor of W wider than
     *        8 x 8 blocks; ignored at depth 0 and for other dtypes (the
     *        emulated leaf always stores its products).
     * In a batched launch each plan keeps its form: stored plans write their
     * products in the grouped leaf launch, then run their passes, then their
     * rank-q fix-ups in one more grouped launch per tile width. */
    int post_additions;
} fmm_plan_options_t;

/* Read-only description of a plan (all sizes in elements). */
typedef struct {
    int64_t n;              /* problem size */
    int p, depth;           /* split factor, recursion depth */
    int64_t P;              /* blocks per side after flattening = p^depth */
    int64_t R_total;        /* leaf products = R^depth */
    int64_t m;              /* leaf block size = floor(n / P) */
    int64_t n_core;         /* P * m, the part that goes through the fast algorithm */
    int64_t tasks;          /* GPU tile tasks per multiplication */
    int materialized_levels;
    double flops_leaf;      /* 2 * R_total * m^3 */
    double flops_executed;  /* FP64 work: leaf (FMM_F64) + additions + peel fix-ups, as scheduled */
    size_t workspace_bytes;
    int ozaki_slices;       /* FMM_F64_OZAKI: slices per operand (0 otherwise) */
    double flops_lowp;      /* FMM_F64_OZAKI: e4m3 tensor-core flops of the slice products */
    int tile_n;             /* leaf tile width of the FP64 kernel (128 or 64) */
    int materialize_passes; /* kernel passes per operand that form the materialized S_r / T_r
                               (a level, a Kronecker factor of one, or two 2 x 2 factors fused) */
    double coef_scale;      /* (den_u den_v den_w)^-depth for a rational plan, 1 otherwise */
    int64_t product_begin;  /* leaf products [product_begin, product_end) of this plan's shard */
    int64_t product_end;    /* (0 and R_total for an unsharded plan) */
    int post_passes;        /* level-by-level post-addition passes of stored leaf products (FMM_F64
                               stored form, FMM_F64_OZAKI from depth 2); 0: fused or flattened */
} fmm_plan_info_t;

/* The contiguous range [*begin, *end) of `units` work units that shard
 * shard_index of shard_count takes: shard k starts at floor(k units /
 * shard_count), so range sizes differ by at most one and the ranges cover
 * [0, units) in order.  Host-only, no GPU work (the partition a sharded plan
 * uses, in units of sub-problems).  FMM_ERR_INVALID for units < 0,
 * shard_count < 1, shard_index outside [0, shard_count) or a NULL output. */
fmm_status_t fmm_shard_range(int64_t units, int shard_count, int shard_index, int64_t *begin, int64_t *end);

/* Status code to a static, NUL-terminated English string (never NULL). */
const char *fmm_status_string(fmm_status_t s);

/* Built-in algorithms by name (static storage, valid for the process):
 *   "classic2"      -- <2,2,2;8> classic block product (Section 3, the printed graph)
 *   "strassen"      -- the Strassen tables printed in Section 2, with the rows of
 *                      c^t placed by their printed labels C0, C2, C1, C3
 *   "strassen1969"  -- Strassen's original 18-addition form
 *   "winograd"      -- Strassen-Winograd, flat form of the 15-addition variant
 *   "laderman"      -- Laderman's <3,3,3;23> (1976)
 * Returns FMM_ERR_NOT_FOUND for any other name, FMM_ERR_INVALID for NULL. */
fmm_status_t fmm_algo_builtin(const char *name, fmm_algo_t *out);

/* Number of the p^6 Brent equations that (U, V, W) violates, computed exactly
 * in int64 (Section 2, equation `strassen` read entry-wise); 0 means the
 * algorithm multiplies exactly.  Host-only.  Returns -1 for invalid input. */
int64_t fmm_algo_brent_mismatches(const fmm_algo_t *algo);

/* Rectangular algorithms <m,k,n;R> (Section 2: a square problem of split
 * factor 6 or 12 can be solved through non-square basic products, 2x3x3 with
 * 3x2x3 and so on, composed by Kronecker products).  A is split into an m x k
 * grid of blocks, B into k x n, C into m x n, each indexed row-major; U is
 * (m k) x R, V is (k n) x R, W is (m n) x R, int32, entry [i][r] at i*R + r.
 * Plans multiply square operands: a rectangular algorithm reaches them as a
 * factor of a square composition (fmm_algo_rect_compose, then
 * fmm_algo_rect_as_square). */
typedef struct {
    int m, k, n;
    int R;
    const int32_t *U;
    const int32_t *V;
    const int32_t *W;
} fmm_algo_rect_t;

/* Failed Brent equations of a rectangular algorithm: the (m k n)^2 index
 * triples (i,j) of A, (j2,l) of B, (i2,l2) of C for which
 * sum_r U V W != delta(j,j2) delta(i,i2) delta(l,l2), summed exactly in int64
 * over the nonzeros of each product (exact for coefficients below 2^21 in
 * magnitude).  -1 for invalid input. */
int64_t fmm_algo_rect_brent_mismatches(const fmm_algo_rect_t *algo);

/* Built-in rectangular algorithms (tables owned by the library):
 * "strassen_2x2x3" is <2,2,3;11>, Strassen's seven products on the first two
 * block columns of B and C plus the four classic products A_i0 B_02,
 * A_i1 B_12 for the third.  FMM_ERR_NOT_FOUND for other names. */
fmm_status_t fmm_algo_rect_builtin(const char *name, fmm_algo_rect_t *out);

/* The classic <m,k,n; m k n> into caller arrays U[(m k) (m k n)],
 * V[(k n) (m k n)], W[(m n) (m k n)] (product (i,j,l) = A_ij B_jl into C_il).
 * FMM_ERR_UNSUPPORTED for m k n > 2^20. */
fmm_status_t fmm_algo_rect_classic(int m, int k, int n, int32_t *U, int32_t *V, int32_t *W, fmm_algo_rect_t *out);

/* Symmetries every algorithm has, into caller arrays of the input's sizes:
 * transpose gives <n,k,m> from (A B)^T = B^T A^T (tables V^T, U^T, W^T, with
 * ^T transposing the block grid); cyclic gives <k,n,m> from the rotation of
 * the trilinear form sum A_ab B_bd C_ad (tables V, W^T, U^T). */
fmm_status_t fmm_algo_rect_transpose(const fmm_algo_rect_t *in, int32_t *U, int32_t *V, int32_t *W,
                                     fmm_algo_rect_t *out);
fmm_status_t fmm_algo_rect_cyclic(const fmm_algo_rect_t *in, int32_t *U, int32_t *V, int32_t *W,
                                  fmm_algo_rect_t *out);

/* Kronecker composition <m1 m2, k1 k2, n1 n2; R1 R2> into caller arrays of
 * (m k) R, (k n) R and (m n) R entries; composed blocks are re-indexed
 * row-major (block (a1 r2 + a2, b1 c2 + b2) of each grid) and product
 * (r1, r2) is r1 R2 + r2, so the first factor is the outer recursion level
 * (Section 2: the order of the factors changes temporary space and error).
 * FMM_ERR_UNSUPPORTED if a table would reach 2^30 entries. */
fmm_status_t fmm_algo_rect_compose(const fmm_algo_rect_t *first, const fmm_algo_rect_t *second, int32_t *U,
                                   int32_t *V, int32_t *W, fmm_algo_rect_t *out);

/* A square view <p,p,p;R> (p = m = k = n) of a rectangular algorithm, sharing
 * its tables; FMM_ERR_UNSUPPORTED unless m = k = n. */
fmm_status_t fmm_algo_rect_as_square(const fmm_algo_rect_t *in, fmm_algo_t *out);

/* The Brent equations of a rational algorithm, multiplied through by
 * den_u den_v den_w: sum_r U V W = den_u den_v den_w delta delta delta over the
 * numerators, exact in int64.  Returns the number of violated equations, or -1
 * for invalid input (a NULL table, p < 2, R < 1, a denominator < 1, or
 * numerators so large that R max|U| max|V| max|W| or the denominators'
 * product reaches 2^62). */
int64_t fmm_algo_rational_brent_mismatches(const fmm_algo_rational_t *algo);

/* Relabel an algorithm given in the paper's printed format, where the rows of
 * c^t index the blocks of C transposed (Section 2: printed order C0, C2, C1,
 * C3 for p = 2), into this library's row-major W.  `ct` and `W_out` are
 * p^2 x R int32 row-major; W_out[(i*p + k)][r] = ct[(k*p + i)][r]. */
fmm_status_t fmm_algo_from_transposed_c(int p, int R, const int32_t *ct, int32_t *W_out);

/* Two-level composition (Section 2, Kronecker products of the factor
 * matrices): first factor outermost.  Nested block ((i1,j1),(i2,j2)) becomes
 * block (i1*p2 + i2)*(p1*p2) + (j1*p2 + j2); product (r1, r2) becomes
 * r1*R2 + r2.  The caller provides U_out/V_out/W_out with (p1 p2)^2 * R1 R2
 * int32 entries each; out->U/V/W are set to them. */
fmm_status_t fmm_algo_compose(const fmm_algo_t *first, const fmm_algo_t *second, int32_t *U_out,
                              int32_t *V_out, int32_t *W_out, fmm_algo_t *out);

/* Create a plan for C = A * B with n x n operands, `depth` levels of `algo`.
 * depth = 0 is the classic product.  Validates arguments (FMM_ERR_INVALID),
 * the Brent equations (FMM_ERR_BRENT), the dtype (FMM_ERR_UNSUPPORTED),
 * flattens the recursion, lays out the tile-task schedule, uploads the
 * coefficient tables and allocates the device workspace (FMM_ERR_OOM) on the
 * current device.  The plan owns that workspace.  Blocking (host + a
 * synchronous upload).  Not thread-safe with respect to the same plan. */
fmm_status_t fmm_plan_create(fmm_plan_t **out, int64_t n, const fmm_algo_t *algo, int depth,
                             fmm_dtype_t dtype);
fmm_status_t fmm_plan_create_ex(fmm_plan_t **out, int64_t n, const fmm_algo_t *algo, int depth,
                                fmm_dtype_t dtype, const fmm_plan_options_t *opts);

/* A plan for a rational algorithm (opts may be NULL).  Checks the rational
 * Brent equations (FMM_ERR_BRENT; FMM_ERR_INVALID for what
 * fmm_algo_rational_brent_mismatches rejects), then plans the integer
 * numerator tables as fmm_plan_create_ex does and applies the product of the
 * denominators, (den_u den_v den_w)^-depth, once per leaf product in the
 * post-additions (folded into alpha: w -> alpha * scale * w; with stored leaf
 * products, alpha * scale once per element of C in the last pass); the peel fix-ups
 * of non-divisible sizes are plain products and are not scaled.  With
 * power-of-two denominators the scale is exact, so integer-valued inputs still
 * give exact results while every intermediate stays below 2^53.  Every call
 * on the plan (fmm_gemm, fmm_gemm_ex, the batched calls) works as for an
 * integer plan; fmm_plan_info_t.coef_scale reports the scale. */
fmm_status_t fmm_plan_create_rational(fmm_plan_t **out, int64_t n, const fmm_algo_rational_t *algo, int depth,
                                      fmm_dtype_t dtype, const fmm_plan_options_t *opts);

/* C = A * B on `stream`.  A, B, C: device pointers to n x n row-major
 * binary64; C is overwritten; A and B are read only and must not overlap C.
 * Asynchronous.  Two calls on the same plan must not overlap in time (they
 * share the plan's workspace); issue them on one stream.  FMM_ERR_CUDA if a
 * launch fails.  Device-side wait timeouts surface at fmm_sync_status. */
fmm_status_t fmm_gemm(const fmm_plan_t *plan, const double *A, const double *B, double *C,
                      void *stream);

/* C = alpha * A * B + beta * C on `stream`: the scaled product as Section 3
 * states it (C = alpha A B), with the BLAS beta term.  Same operands, plan
 * rules and errors as fmm_gemm, which is alpha = 1, beta = 0.
 *   - beta = 0: C is written without being read (NaN or Inf in C is dropped).
 *   - alpha = 0: A and B are not read and no product runs; C = beta * C
 *     (zeros for beta = 0), one elementwise kernel.
 *   - otherwise every coefficient w of W is applied as alpha * w, and the first
 *     contribution to each element of C adds it to beta * C (C read once);
 *     the rest of the schedule, and its determinism, is that of fmm_gemm.
 * FMM_ERR_INVALID for a NULL pointer or a non-finite alpha or beta. */
fmm_status_t fmm_gemm_ex(const fmm_plan_t *plan, double alpha, const double *A, const double *B,
                         double beta, double *C, void *stream);

/* C = alpha * A * B + beta * C for an FMM_F32 plan: A, B, C are n x n
 * row-major binary32 device arrays, alpha and beta binary32 (the scalar rules
 * of fmm_gemm_ex: beta = 0 leaves C unread, alpha = 0 leaves A and B unread).
 * The plan's three binary64 planes hold the widened operands and the product
 * before its single rounding.  FMM_ERR_INVALID for another dtype; fmm_gemm
 * and fmm_gemm_ex return FMM_ERR_INVALID for an FMM_F32 plan. */
fmm_status_t fmm_gemm_f32_ex(const fmm_plan_t *plan, float alpha, const float *A, const float *B, float beta,
                             float *C, void *stream);

/* Same as fmm_gemm with HOST buffers: copies A and B to plan-owned device
 * buffers (allocated on first use, freed by fmm_plan_destroy), multiplies,
 * copies C back and synchronizes `stream` before returning.  Blocking.
 * For an FMM_F64 or FMM_F64_OZAKI plan, B is copied on a plan-owned stream
 * (created on first use) while A's copy and A's pre-addition passes run on
 * `stream`; B's passes wait for its copy.  With page-locked sources the two
 * overlap; a pageable source's copy returns only once it is done.  For an
 * FMM_C128 plan the buffers hold interleaved complex pairs and for an
 * FMM_F32 plan binary32 values (pass their addresses cast to these types);
 * both copy A, then B, on `stream`.  On GB300 (Grace host) buffers from
 * fmm_host_alloc copy at about 210 GB/s host to device and 193 GB/s back;
 * other page-locked and pageable buffers reach 180-210 GB/s on a fresh host
 * but can fall far below that later (see fmm_host_alloc).  FMM_ERR_OOM if
 * the device buffers cannot be allocated, FMM_ERR_CUDA if a copy or launch
 * fails. */
fmm_status_t fmm_gemm_host(fmm_plan_t *plan, const double *A_host, const double *B_host,
                           double *C_host, void *stream);

/* Page-locked host memory for the buffers of fmm_gemm_host (usable for any
 * copy to or from the GPU).  No counterpart in the paper, whose timings
 * exclude host transfers.  On Linux with transparent huge pages, a request of
 * at least one huge page (hpage_pmd_size: 2 MiB with 4 KiB base pages,
 * 512 MiB with 64 KiB pages) is mapped at a huge-page boundary, rounded up to
 * whole huge pages, advised to use them and registered with the CUDA driver
 * (portable to every context); smaller requests, and systems where that
 * fails, get cudaHostAlloc memory.  Why: on GB300 (Grace host, 64 KiB base
 * pages), once other processes had used and freed much memory, host-to-device
 * copies from cudaHostAlloc buffers fell to 12-16 GB/s while huge-page buffers
 * kept 210 GB/s (193 GB/s back).  On success *out holds the address (aligned
 * to at least the base page); the caller owns it until fmm_host_free.
 * FMM_ERR_INVALID for out == NULL, FMM_ERR_OOM if no page-locked memory could
 * be had (also without a CUDA driver). */
fmm_status_t fmm_host_alloc(void **out, size_t bytes);

/* Releases memory from fmm_host_alloc; NULL is a no-op.  FMM_ERR_INVALID for
 * an address that fmm_host_alloc did not return or that was freed already. */
fmm_status_t fmm_host_free(void *p);

/* The transparent huge-page size fmm_host_alloc uses, in bytes (0 if the
 * system has none). */
int64_t fmm_host_huge_page_bytes(void);

/* Batched: count independent products C[i] = A[i] * B[i], each with its own
 * plan (sizes and algorithms may differ), as one persistent grouped launch
 * over the union of their tile tasks (one per leaf tile width present).
 * Plans with stored leaf products (fmm_plan_options_t.post_additions) then
 * run their post-addition passes and one more grouped launch of their rank-q
 * fix-ups.  plans/A/B/C are HOST arrays of
 * `count` entries; A[i], B[i], C[i] are device pointers.  All plans must be
 * FMM_F64 and not in use by another call at the same time.  Asynchronous. */
fmm_status_t fmm_gemm_batched(fmm_plan_t *const *plans, const double *const *A,
                              const double *const *B, double *const *C, int count, void *stream);

/* Batched C[i] = alpha[i] * A[i] * B[i] + beta[i] * C[i] with the rules of
 * fmm_gemm_ex per product.  alpha and beta are HOST arrays of `count` values,
 * or NULL for all ones (alpha) / all zeros (beta).  Products with alpha[i] = 0
 * run as a scaling of C[i] before the grouped launch and are left out of it. */
fmm_status_t fmm_gemm_batched_ex(fmm_plan_t *const *plans, const double *alpha, const double *const *A,
                                 const double *const *B, const double *beta, double *const *C, int count,
                                 void *stream);

/* A batched multiplication captured once into a CUDA graph (the counter
 * resets, materialization passes, grouped leaf launches and post-addition
 * passes of fmm_gemm_batched), replayed with fmm_batch_graph_launch.  The plans and the
 * A/B/C pointers are baked into the graph: they must stay valid and unchanged
 * until fmm_batch_graph_destroy.  Creation captures on a private stream and
 * does not run the work. */
typedef struct fmm_batch_graph fmm_batch_graph_t;
fmm_status_t fmm_batch_graph_create(fmm_batch_graph_t **out, fmm_plan_t *const *plans, const double *const *A,
                                    const double *const *B, double *const *C, int count);
/* Enqueue one replay of the captured batch on `stream` (asynchronous). */
fmm_status_t fmm_batch_graph_launch(const fmm_batch_graph_t *g, void *stream);
/* Free the graph (NULL-safe).  No replay may be pending. */
void fmm_batch_graph_destroy(fmm_batch_graph_t *g);

/* Autotuner, with no counterpart in the paper beyond its observation that the
 * best algorithm depends on the problem size and that each call has a fixed
 * overhead (Section 3): times one FMM_F64 multiplication of size n on scratch
 * operands for every candidate configuration and returns the fastest.  The
 * candidates are
 *   - depth 0 (the classic product, algos[0]'s split factor is irrelevant);
 *   - every algorithm (index into `algos`) at every depth 1..max_depth whose
 *     leaf n / p^depth is at least min_leaf;
 *   - for each of those, both leaf tile widths (tile_n 64 and 128) and, at
 *     depth 1 when the planner would materialize it, both the default
 *     (materialized) and the fused schedule.
 * With FMM_FORCE_DEPTH=d set, only the depth-d candidates are timed
 * (depth0_ms is then 1e30 unless d = 0); FMM_ERR_INVALID if none qualifies.
 * Each candidate runs once untimed, then up to `reps` timed runs (CUDA events
 * on `stream`; reps < 1 means 5); its time is the median.  A candidate whose
 * first timed run is more than 1.5 times the best median so far stops there.
 * Blocking; allocates and frees 3 n^2 doubles and the candidate plans on the
 * current device. */
typedef struct {
    int algo_index;          /* index into the candidate list */
    int depth;
    double ms;               /* median time of the best candidate */
    int tile_n;              /* its leaf tile width (64 or 128) */
    fmm_schedule_t schedule; /* its schedule (FMM_SCHED_AUTO or FMM_SCHED_FUSED) */
    double depth0_ms;        /* median time of the best depth-0 candidate */
    int candidates;          /* configurations timed */
} fmm_tune_result_t;
fmm_status_t fmm_autotune(int64_t n, const fmm_algo_t *const *algos, int nalgos, int max_depth, int64_t min_leaf,
                          int reps, void *stream, fmm_tune_result_t *best);

/* Synchronize `stream`, then read and clear the plan's device error flag:
 * FMM_OK, FMM_ERR_TIMEOUT (a bounded wait expired; C is unspecified) or
 * FMM_ERR_CUDA. */
fmm_status_t fmm_sync_status(const fmm_plan_t *plan, void *stream);

/* Timing of the most recent fmm_gemm on a plan created with
 * record_kernel_time = 1: `leaf_ms` is the leaf-product kernel alone,
 * `total_ms` the whole call (counter reset, materialization, leaf kernel),
 * both measured with CUDA events on the call's stream.  For a complex plan
 * (FMM_C128, FMM_C128_3M) both are the whole call: split, real products and
 * join.  Waits for the call's end event.  FMM_ERR_INVALID if timing was not
 * enabled or no call was made. */
fmm_status_t fmm_plan_last_kernel_ms(const fmm_plan_t *plan, float *leaf_ms, float *total_ms);

/* Phase times of the most recent fmm_gemm on a plan created with
 * record_kernel_time = 1, in milliseconds, measured with CUDA events on the
 * call's stream: phases[0] counter reset and materialized pre-additions,
 * phases[1] exponents and slicing (FMM_F64_OZAKI; 0 otherwise), phases[2]
 * the leaf-product kernel, phases[3] the peel tasks run after an emulated
 * leaf (0 otherwise), phases[4] the post-additions C_l = sum_r W[l][r] P_r
 * that the emulated leaf runs as a separate kernel (0 otherwise).  Fills
 * min(count, 5) entries; waits for the call.  FMM_ERR_INVALID for a complex
 * plan (its real plan records the phases of each real product separately). */
fmm_status_t fmm_plan_last_phase_ms(const fmm_plan_t *plan, float *phases, int count);

/* Calibration, with no counterpart in the paper: measures the FP64
 * throughput the current device delivers on the leaf kernel's instruction
 * (mma.sync m16n8k4 f64, "DMMA") and on scalar DFMA, in TFLOP/s, with CUDA
 * events on `stream` (about 0.1 s of GPU time; allocates and frees a small
 * scratch buffer).  Blocking.  Either output pointer may be NULL. */
fmm_status_t fmm_measure_fp64_peak(void *stream, double *dmma_tflops, double *dfma_tflops);

/* Calibration, with no counterpart in the paper: throughput of the emulated
 * leaf's instruction (mma.sync m16n8k32 e4m3 with FP32 accumulation) on the
 * current device, in TFLOP/s, timed like fmm_measure_fp64_peak.  Blocking. */
fmm_status_t fmm_measure_e4m3_peak(void *stream, double *tflops);

/* Size of the static device scratch array used by fmm_gemm_noalloc. */
#define FMM_NOALLOC_SCRATCH_BYTES (4u << 20)

/* C = A * B without allocating any memory; there is no counterpart in the
 * paper.  For callers that cannot allocate device memory at all -- code
 * running inside an allocator or memory-pool callback, frameworks that
 * reserve all device memory up front, real-time paths where cudaMalloc and
 * its implicit synchronization are not allowed.
 *
 * Runs the fused schedule (every recursion level combined while staging the
 * leaf operands) of `depth` levels of `algo` on n x n row-major binary64
 * device matrices A, B, C (C overwritten, A and B not overlapping C), on
 * `stream`.  All scratch state (ordering counters, task counter, error word,
 * flattened coefficient tables) lives in one file-scope __device__ array of
 * FMM_NOALLOC_SCRATCH_BYTES (4 MiB) that every GPU loading the library holds
 * until the process exits; host-side planning uses fixed static buffers.  The
 * call makes no cudaMalloc, cudaFree or other allocating call.
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * Each call copies its tables into the array and clears the counters and the
 * error word on `stream` before launching; the copy comes from one host
 * buffer that the next call rewrites, so a call made while `stream` is being
 * captured into a CUDA graph returns FMM_ERR_UNSUPPORTED and enqueues
 * nothing.  Every call shares the one array, which keeps the last call's
 * contents: calls that overlap on the GPU (for example on different streams)
 * race and give wrong results.  Host calls are serialized by a mutex.  A
 * device-side wait that times out ends the kernel with C unspecified; read it
 * with fmm_noalloc_sync_status before the next call.
 *
 * Errors: FMM_ERR_INVALID (NULL pointer, n < 1, p < 2, R < 1, depth < 0,
 * leaf size < 1), FMM_ERR_BRENT, FMM_ERR_SCRATCH_LIMIT (p > 4, depth > 4, or
 * tables plus counters larger than FMM_NOALLOC_SCRATCH_BYTES),
 * FMM_ERR_UNSUPPORTED (a flattened column with more than 256 terms, n > 2^30,
 * p^2 R >= 2^28, R max|U| max|V| max|W| >= 2^62, max|X|^depth >= 2^31 for a
 * table X, or `stream` capturing), FMM_ERR_CUDA. */
fmm_status_t fmm_gemm_noalloc(int64_t n, const fmm_algo_t *algo, int depth, const double *A, const double *B,
                              double *C, void *stream);

/* Device status of the most recent fmm_gemm_noalloc call on the current
 * device, without allocating (no counterpart in the paper): synchronizes
 * `stream` (the stream of that call), reads the error word kept at the start
 * of the static scratch array and clears it.  FMM_OK, FMM_ERR_TIMEOUT (a
 * bounded device-side wait expired; that call's C is unspecified) or
 * FMM_ERR_CUDA.  Only the latest call's status is kept: each call clears it. */
fmm_status_t fmm_noalloc_sync_status(void *stream);

/* Testing only (no counterpart in the paper): the bound on every device-side
 * wait of later fmm_gemm_noalloc calls (default 5 s), and poison_chain = 1 to
 * set one post-addition ordering counter, after each call's reset, to a value
 * no task writes, so that its waiters time out.  FMM_ERR_INVALID unless
 * 0 < wait_timeout_s <= 3600. */
fmm_status_t fmm_noalloc_set_debug(double wait_timeout_s, int poison_chain);

/* Testing only (no counterpart in the paper): make the k-th next allocation
 * the library requests fail (k = 0: the next one; k < 0: none), counting every
 * device, page-locked host and plan-object allocation of fmm_plan_create*,
 * fmm_gemm_host, fmm_gemm_batched*, fmm_batch_graph_create and fmm_autotune.
 * The failing call returns FMM_ERR_OOM after releasing what it had taken. */
void fmm_debug_fail_allocation(int64_t k);

/* Testing only: the number of those allocations currently live (0 when no
 * plan, batch graph or call is outstanding). */
int64_t fmm_debug_live_allocations(void);

/* Describe a plan.  Host-only. */
fmm_status_t fmm_plan_get_info(const fmm_plan_t *plan, fmm_plan_info_t *info);

/* Device workspace owned by the plan, in bytes (0 for NULL). */
size_t fmm_plan_workspace_bytes(const fmm_plan_t *plan);

/* Release the plan and its device memory.  NULL is a no-op.  The caller must
 * ensure no GPU work using the plan is still pending. */
void fmm_plan_destroy(fmm_plan_t *plan);

#ifdef __cplusplus
}
#endif

#endif /* FMM_H_ */
