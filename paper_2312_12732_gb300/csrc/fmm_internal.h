// Internal declarations shared by the host planner and the CUDA kernels of the
// fast-matrix-multiplication library.  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace fmm {

// CTA tile of the FP64 leaf kernel: kBM rows x kBN (or 64) columns of a
// product tile, K slab kBK.
constexpr int kBM = 128;
constexpr int kBN = 128;
constexpr int kBK = 16;
// Upper bound on the number of blocks combined into one operand (nonzeros of a
// flattened U or V column) and on the destinations of one product (nonzeros
// of a flattened W column).
constexpr int kMaxTerms = 256;

// Device error codes written to the plan's error word.
enum : int { kDevOk = 0, kDevTimeout = 1 };

// Geometry and coefficient tables of one plan, resident in device memory.
// "Core" tasks compute one kBM x kBN tile of one leaf product; peel tasks fix
// up the trailing n - n_core rows/columns.
struct F64Geom {
    long long n;           // full problem size
    long long m;           // leaf block size
    long long n_core;      // P * m
    long long ld_src_a;    // leading dimension of the core-task operand sources
    long long ld_src_b;
    long long sub_stride_a;  // elements between consecutive materialized sub-problems
    long long sub_stride_b;
    int P;                 // blocks per side of C (p^depth)
    int P_src;             // blocks per side of a core-task source (p^(depth - materialized))
    int R_src;             // products per sub-problem (R^(depth - materialized))
    int nsub;              // sub-problems (R^materialized)
    int sub_begin;         // first sub-problem of a sharded plan (core task 0 belongs to it)
    int tiles_m, tiles_n;  // tiles per leaf block
    int bn;                // tile columns: 128 or 64 (0 means 128)
    // CSC over products: U/V columns are indexed by the sub-problem-local
    // product, W columns by the global product s * R_src + r.
    const int *u_ptr;
    const int2 *u_ent;  // {source block, coefficient}
    const int *v_ptr;
    const int2 *v_ent;
    const int *w_ptr;
    const int4 *w_ent;  // {C block, coefficient, position among the row's nonzeros, 0}
    const int *w_row_nnz;
    long long tasks_core, tasks_right, tasks_bottom, tasks_rankq;
    int rb_tm, rb_tn;  // right-border tiling (n_core x q)
    int bb_tm, bb_tn;  // bottom-border tiling (q x n)
    // Stored leaf products (post-additions in separate passes): when pout is
    // set, core task r stores P_r = S_r T_r unscaled at pout + r m^2 (leading
    // dimension m) instead of adding it into C.
    double *pout;
    // 1: rank-q tasks add into C without waiting on ordering counters (C's
    // core blocks are complete before the launch that runs them).
    int rankq_free;
    int pad_;
};

struct F64Problem {
    const F64Geom *g;    // device pointer
    const double *A;     // original operands (ld = n)
    const double *B;
    const double *SA;    // sources of core tasks (A itself, or materialized S)
    const double *SB;
    double *C;           // output (ld = n)
    unsigned *chain;     // [P*P][tiles] post-add ordering counters
    long long task_begin;
    // C = alpha A B + beta C (alpha = 0 never reaches a kernel).  Core tasks
    // apply alpha times the plan's coefficient scale (a rational algorithm's
    // 1 / denominators) to every W coefficient; peel tasks apply alpha_peel.
    double alpha;
    double alpha_peel;
    double beta;         // beta = 0: C is written without being read
};

template <int MAXP>
struct F64Launch {
    int nprobs;
    long long total_tasks;
    unsigned long long *task_counter;
    int *error;
    long long timeout_ns;
    // Interleaved order (grouped launches, interleave = 1): problems sorted by
    // task count, descending, are visited round-robin by local task index, so
    // that concurrently running tasks mostly belong to different problems.
    // Segment q (q = nprobs .. 1 active problems) starts at global index
    // seg_start[q - 1] and covers rounds [seg_round[q - 1], ...); order[j] is
    // the problem at sorted position j.  Each problem's own order is kept, so
    // every post-addition wait still points at a lower global index.
    int interleave;
    long long seg_start[MAXP];
    int seg_round[MAXP];
    short order[MAXP];
    F64Problem probs[MAXP];
};

constexpr int kMaxBatchPerLaunch = 256;

// Emulated-FP64 leaf (fmm_ozaki.cu): balanced digits of kOzDigitBits bits
// stored as e4m3, up to kOzMaxSlices slices per operand.
constexpr int kOzDigitBits = 5;
constexpr int kOzMaxSlices = 12;

struct OzParams {
    const unsigned char *sa;  // left slices  [R][s][Mp][Kp] (row r of S_r, K contiguous)
    const unsigned char *sb;  // right slices [R][s][Mp][Kp] (column j of T_r, K contiguous)
    const int *mxa;           // [R][Mp] largest biased exponent of each row of S_r
    const int *mxb;           // [R][Mp] ... of each column of T_r
    double *C;                // C (the mma.sync engine adds into it directly)
    long long ldc;
    double *pout;             // [R][m][m] leaf products P_r (tcgen05 engines), leading dimension m
    long long m;              // leaf size
    int Mp, Kp;               // padded to multiples of 128
    int s;                    // slices per operand
    int L;                    // right shift keeping the int64 recombination in range
    int kparts;               // CTA-pair engine: K pieces per slice pair, each a diagonal group of its own
    int tiles_m, tiles_n;
    int R;                    // leaf products
    int P;                    // C blocks per side
    const int *w_ptr;
    const int4 *w_ent;
    unsigned *chain;
    long long tasks;
    unsigned long long *task_counter;
    int *error;
    long long timeout_ns;
    double alpha, beta;       // C = alpha A B + beta C (the mma.sync engine's epilogue)
};

// Exponents and slices of every row (by_rows) or column of the nmat matrices
// X + i * mat_stride (rows x cols, leading dimension ld); mx receives the
// largest biased exponent of each line ([mat][pitch]).
cudaError_t launch_ozaki_slices(const double *X, long long ld, long long mat_stride, int nmat, int rows, int cols,
                                bool by_rows, int *mx, int pitch, int s, int Mp, int Kp, unsigned char *out,
                                cudaStream_t st);
cudaError_t launch_ozaki_gemm(const OzParams &P, int grid, cudaStream_t s);
int ozaki_ctas_per_sm();
size_t ozaki_smem_bytes();
// tcgen05 slice GEMM (fmm_ozaki_tc.cu): map_a / map_b are 2-D uint8 tensor
// maps over the slice buffers ([rows][Kp], 128 x 128 boxes, 128B swizzle).
cudaError_t launch_ozaki_tc(const CUtensorMap &map_a, const CUtensorMap &map_b, const OzParams &P, int grid,
                            cudaStream_t s);
// The same slice GEMM on CTA pairs (tcgen05 cta_group::2): `ctas` CTAs in
// clusters of 2 (one pair each).  map_a has 128-row boxes over the left
// slices, map_bh 64-row boxes over the right slices; each CTA loads its own
// boxes.  P.tasks counts (product, tile-row pair, two tile columns).
cudaError_t launch_ozaki_tc_pair(const CUtensorMap &map_a, const CUtensorMap &map_bh, const OzParams &P, int ctas,
                                 cudaStream_t s);
// Largest number of co-resident CTA pairs of the pair kernel (0 if it cannot run).
int ozaki_tc_max_pairs();
// C_l = alpha sum_r W[l][r] P_r + beta C_l for the P x P blocks of side m of
// C (leading dimension ldc), in ascending r: wl_ptr / wl_ent list, per block
// l, the products (r, coefficient) in ascending r.  beta = 0 writes C without
// reading it.  The peel tasks that follow add into C without ordering waits.
cudaError_t launch_ozaki_postadd(const double *pout, long long m, int P, const int *wl_ptr, const int2 *wl_ent,
                                 double *C, long long ldc, double alpha, double beta, cudaStream_t s);
// One pass of level-by-level post-additions of a plan whose leaf products
// are stored (fmm_postadd.cu).  The products are indexed by the
// digits (r_1, ..., r_K) of the Kronecker factors of W over all recursion
// levels, outermost first, and C blocks by (q_1, ..., q_K), q_k = i_k p_k +
// j_k.  A pass sums the innermost factor not yet summed (or the two innermost
// when both are 2 x 2 with at most 8 products): input block
// ((x R_a + r_a) R_b + r_b) ns + s, output block ((x Q_a + q_a) Q_b + q_b) ns + s
// for prefix x < np and suffix s < ns, each block m x m contiguous.  A
// single-factor pass has R_a = Q_a = 1.  The last pass (np = 1) writes C block
// c_blk[o] = (block row, block column) of output o as alpha sum + beta C.
struct LevelPass {
    const double *in;
    double *out;          // intermediate blocks, or C (leading dimension ldc) in the last pass
    long long m, mm, ldc;
    int np, ns;
    int ra, qa, rb, qb;
    // single pass: columns r of W_b, entries {q, coefficient low word, high word, flags}
    // (bit 0: first term of row q, bit 1: coefficient +-1); pair pass: rows q of W_b,
    // entries {r, low word, high word, 0} ascending r
    const int *b_ptr;
    const int4 *b_ent;
    // pair pass: columns r of W_a, entries {q, low word, high word, flags}
    const int *a_ptr;
    const int4 *a_ent;
    const int2 *c_blk;
    double alpha, beta;
    int last;
    int unit_b;           // pair pass: every coefficient of W_b is +-1
    int chunk;            // positions per work unit (a multiple of 128; set by the launcher)
    int store;            // last pass, set by the launcher: 1 C = s, 2 alpha s, 3 fma(alpha, s, C), 4 fma(alpha, s, beta C)
};
cudaError_t launch_level_pass(const LevelPass &a, cudaStream_t s);
constexpr int kLevelMaxQ = 64;  // blocks of one single-factor pass (p <= 8)

// C = beta C over `count` contiguous doubles; beta = 0 stores zeros without
// reading C (fmm_materialize.cu).
cudaError_t launch_scale_c(double *C, long long count, double beta, cudaStream_t s);

// Double-complex planes (fmm_complex.cu); X and C are interleaved (re, im)
// arrays of `count` complex entries, 16-byte aligned.
// re, im (and sum = re + im when not null) <- X.
cudaError_t launch_split_complex(const double *X, long long count, double *re, double *im, double *sum,
                                 cudaStream_t s);
// C <- (re, im).
cudaError_t launch_join_complex(const double *re, const double *im, double *C, long long count, cudaStream_t s);
// Single precision (fmm_complex.cu): out <- (double) X; out <- round-to-nearest
// (float) X; C <- beta C on `count` floats (beta = 0: zeros, C not read).
cudaError_t launch_f32_to_f64(const float *X, long long count, double *out, cudaStream_t s);
cudaError_t launch_f64_to_f32(const double *X, long long count, float *out, cudaStream_t s);
cudaError_t launch_scale_f32(float *C, long long count, float beta, cudaStream_t s);
// C <- alpha (T1 - T2, (T3 - T1) - T2) + beta C (beta = 0: C not read).
cudaError_t launch_gauss_join(const double *T1, const double *T2, const double *T3, double *C, long long count,
                              double alpha, double beta, cudaStream_t s);

// Kernel launchers (fmm_f64.cu).  Return cudaSuccess or the launch error.
// bn selects the tile configuration (128 or 64 columns).
cudaError_t launch_f64_single(const F64Launch<1> &L, int grid, cudaStream_t s, int bn = kBN);
cudaError_t launch_f64_batch(const F64Launch<kMaxBatchPerLaunch> &L, int grid, cudaStream_t s, int bn = kBN);
int f64_kernel_ctas_per_sm(int bn = kBN);  // resident CTAs per SM of the leaf kernel (0 on error)
size_t f64_kernel_smem_bytes(int bn = kBN);

// Pre-addition pass for one materialized recursion level (fmm_f64.cu).
// Input matrix c (c < n_in) starts at in + c * in_stride with leading
// dimension ld_in and is split into p x p blocks of size b_out; output
// c * R + s is the b_out x b_out matrix sum_e coef_e * block(row_e, col_e)
// over the CSC column s (s < R) of the one-level coefficient matrix, entries
// {block row, block col, low word, high word of coef_e as a double}, stored
// densely at out + (c * R + s) * b_out^2.  unit: every coefficient is +-1.
cudaError_t launch_materialize_level(const double *in, long long ld_in, long long in_stride, int n_in,
                                     long long b_out, int p, int R, const int *ptr, const int4 *ent, bool unit,
                                     double *out, cudaStream_t s);
// Two consecutive steps with 2 x 2 block grids (at most 8 products each) in
// one pass; out receives n_in * R1 * R2 matrices of side b2 (= input side / 4).
// unit: every coefficient of both steps is +-1.
cudaError_t launch_materialize_two_steps(const double *in, long long ld_in, long long in_stride, int n_in,
                                         long long b2, int R1, const int *ptr1, const int4 *ent1, int R2,
                                         const int *ptr2, const int4 *ent2, bool unit, double *out,
                                         cudaStream_t s);

// Calibration (fmm_calib.cu): FP64 throughput of DMMA (mma.sync m16n8k4) and
// DFMA on the current device, in TFLOP/s, timed with CUDA events on `s`.
cudaError_t measure_fp64_peaks(cudaStream_t s, double *dmma_tflops, double *dfma_tflops);
// ... and of mma.sync m16n8k32 e4m3 with FP32 accumulation (the emulated leaf's instruction).
cudaError_t measure_e4m3_peak(cudaStream_t s, double *tflops);

}  // namespace fmm
