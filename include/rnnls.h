/*
 * rnnls.h -- C ABI of the GB300 RandomizedNNLS library (librnnls.so).
 *
 * Implements the method of Boutsidis & Drineas, "Random Projections for the
 * Nonnegative Least-Squares Problem": given a tall A (n x d, n >> d), a
 * target b and a sample size r, build the small problem
 *     SA = H~ D A,  Sb = H~ D b                         (Alg. 1 steps 1-4)
 * with D a random +-1 diagonal and H~ the randomly sampled, rescaled rows of
 * the normalised Walsh-Hadamard matrix H_n (Sec. 2), and return
 *     x~ = argmin_{x >= 0} ||SA x - Sb||^2              (Alg. 1 step 5)
 * computed by the Lawson-Hanson active-set method (Sec. 2.2) on the
 * quadratic-programming form Q = SA'SA, q = SA'Sb (Sec. 3.4).
 *
 * Conventions shared by every entry point
 *   - Matrices are column-major with an explicit leading dimension.
 *   - Pointers named A, b, SA, Sb, idx, x, info, SB, X are DEVICE pointers
 *     (cudaMalloc'd or torch-allocated memory of the context's device)
 *     unless the entry point's comment says HOST.  The caller owns every
 *     buffer; the library never frees or retains caller pointers.
 *   - The library owns only the context and its workspace (device memory
 *     grown on demand by cudaMalloc and freed by rnnls_destroy).
 *   - All work is enqueued on the context's stream and is asynchronous
 *     unless stated; results are valid once that stream is synchronised.
 *   - Rows n_raw..n-1, where n is the next power of two >= n_raw, are the
 *     zero padding of Sec. 2; they are never read or stored.
 *   - Return value: RNNLS_OK or an error code below.  Argument errors are
 *     detected on the host before anything is enqueued.  Per-solve
 *     outcomes (singular, iteration cap) are reported in rnnls_info.
 *   - A call that takes a context makes the context's device current while
 *     it runs and gives the calling thread's current device back before it
 *     returns; rnnls_sketch_noalloc runs on the current device.
 *   - A context is used by one host thread at a time (its workspace and
 *     staging buffer are reused call after call); use one context per
 *     thread or stream for concurrent work.  Different contexts may share a
 *     device and run concurrently.
 *
 * Randomness (the paper leaves the generator unspecified, Alg. 1 steps 2
 * and 4): Philox4x64-10 (Salmon et al., SC'11) keyed by (seed, instance),
 * counter (j, stream, 0, 0).
 *   D_ii  : bit (i mod 64) of word (i / 64) of stream 0; set bit -> -1.
 *   iid   : draw k (k < r) is row (word k of stream 2) >> (64 - log2 n).
 *   Bernoulli (Alg. 1 step 2): row i kept iff word i of stream 1 is below
 *           r * 2^(64 - log2 n), i.e. with probability exactly r/n; every
 *           row when r >= n.  Kept rows are listed in increasing order.
 *   Word w of a stream is word (w mod 4) of block j = w / 4.
 * Scale of every kept row: 1/sqrt(r), the normalisation 1/sqrt(n) of H_n
 * times sqrt(n/r) of S (Alg. 1 step 2); 1/sqrt(n) in Bernoulli mode with
 * r >= n (Alg. 2 with p_i = 1/n).
 */
#ifndef RNNLS_H
#define RNNLS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define RNNLS_OK 0
#define RNNLS_EINVAL 1       /* bad argument (null pointer, size, stride, flag) */
#define RNNLS_ECAPACITY 2    /* sampled rows exceed the caller's capacity */
#define RNNLS_ENONFINITE 3   /* NaN or Inf in the Gram matrix of the sketch */
#define RNNLS_ESINGULAR 4    /* passive-set system numerically singular */
#define RNNLS_EMAXITER 5     /* Lawson-Hanson iteration cap reached */
#define RNNLS_ETIMEOUT 6     /* reserved: a sketch block whose bounded wait on a tensor copy
                                gives up writes NaN in its part of SA/Sb instead, which
                                the solve reports as RNNLS_ENONFINITE */
#define RNNLS_ECUDA 7        /* a CUDA runtime call failed */
#define RNNLS_ENOMEM 8       /* workspace allocation failed */
#define RNNLS_EUNSUPPORTED 9 /* size outside what this build handles */

/* ---- flags --------------------------------------------------------------- */
#define RNNLS_SAMPLE_IID 0u       /* r uniform draws with replacement (default) */
#define RNNLS_SAMPLE_BERNOULLI 1u /* each row kept with probability r/n (Alg. 1 step 2) */
#define RNNLS_SAMPLE_MASK 1u
/* Precision of the FP32 sketch's Hadamard passes (rnnls_sketch,
 * rnnls_sketch_batched_ex).  RNNLS_PREC_FP32 (default): both 64-point
 * factors of each 4096-row chunk's transform in FP32 registers.
 * RNNLS_PREC_BF16X2: the first factor (row-index bits 0-4 and 11) runs on
 * the tensor cores as a product with H_64, whose +-1 entries are exact in
 * BF16: each value x (signs of D applied) is split into hi = bf16(x) and
 * lo = bf16(x - hi) (|x - hi - lo| <= 2^-18 |x|), and (hi + lo) H_64 is
 * accumulated in FP32 (Sec. 3.4's O(nd log r) preconditioning step, the
 * split-precision form).  Relative Frobenius error vs FP64 about 1e-6
 * (bound used by the tests: 5e-4).  Rows are the same as in FP32 mode.  For
 * padded n <= 8192 (whole column in shared memory) the flag has no effect. */
#define RNNLS_PREC_FP32 0u
#define RNNLS_PREC_BF16X2 2u
#define RNNLS_PREC_MASK 2u

typedef struct rnnls_ctx rnnls_ctx;

/* Outcome of one Lawson-Hanson solve (written by the device). */
typedef struct rnnls_info {
  int32_t status;        /* RNNLS_OK, RNNLS_ESINGULAR, RNNLS_EMAXITER or RNNLS_ENONFINITE */
  int32_t outer_iters;   /* accepted additions to the passive set */
  int32_t inner_iters;   /* passive-set solves inside the interpolation loop */
  int32_t passive_count; /* |P| at exit = number of positive entries of x */
  double tol;            /* dual tolerance used: 10 eps ||SA||_1 max(r, d) ||Sb||_2 */
  double dual_max;       /* max over j not in P of w_j = (SA'(Sb - SA x))_j at exit */
  double objective;      /* ||SA x - Sb||^2 at exit */
  int32_t accurate_mode; /* 0: the FP32 iterations' end point passed its float-float
                            check; 1: a refined passive solve there had z_j <= 0, or
                            2: a float-float dual there exceeded tol, and the solve
                            continued with every step refined (see rnnls_solve) */
  int32_t reserved;      /* zero */
} rnnls_info;

/* One problem of a batched solve.  All pointers are device pointers. */
typedef struct rnnls_problem {
  const float *SA; /* r x d, column-major, leading dimension ldsa >= r */
  int64_t ldsa;
  const float *Sb; /* r */
  int64_t r;
  int64_t d;
  double *x;         /* out: d */
  rnnls_info *info;  /* out: nullable */
} rnnls_problem;

/* Launch-shape choices of one context (not part of the method: none of them
 * changes what is computed beyond FP32 summation order).  0 in a field means
 * the built-in default; rnnls_set_tuning validates the ranges.
 *   sketch_sms           SMs the large-n sketch may occupy (default all;
 *                        the same value as rnnls_set_sketch_sms)
 *   full_step_min_slots  sampled rows per sketch thread from which the four
 *                        chunks of a step are first combined by H_4 (a
 *                        16384-point transform per step) so that each row
 *                        reads one word instead of four (default 48; rows
 *                        per thread below 48 live in registers and never use
 *                        the pass; 48..1024, above 128 meaning never)
 *   gram_min_chunks      least 32-row chunks per tensor-core Gram CTA of a
 *                        single problem (default 8; 1..65536)
 *   gram_max_splits      most K-splits of one Gram tile (default 32; 1..1024)
 *   batch_gram_chunks    most 32-row chunks per Gram CTA in batched solves
 *                        (default 128; 1..65536)
 *   batch_step_cost      the batched sketch's cost of a step's transform in
 *                        the units of one sampled row per thread, used to
 *                        cut the block ranges (default 114; 1..100000) */
typedef struct rnnls_tuning {
  int32_t sketch_sms;
  int32_t full_step_min_slots;
  int32_t gram_min_chunks;
  int32_t gram_max_splits;
  int32_t batch_gram_chunks;
  int32_t batch_step_cost;
  int32_t lh_warp_max_d;  /* Lawson-Hanson problems with d up to this run as one-warp
                             blocks, larger ones as 256-thread blocks (0: none) */
  int32_t reserved;       /* zero */
} rnnls_tuning;

/* Create a context on CUDA device `device` that enqueues on `stream`
 * (a cudaStream_t, borrowed, may be NULL for the legacy default stream).
 * Errors: EINVAL (ctx null), ECUDA (device unusable). */
int rnnls_create(rnnls_ctx **ctx, int device, void *stream);

/* Free the context and its workspace (synchronises its stream first).
 * Errors: EINVAL (ctx null). */
int rnnls_destroy(rnnls_ctx *ctx);

/* Replace the stream the context enqueues on (borrowed; the caller orders
 * work already enqueued on the old stream).  Errors: EINVAL (ctx null). */
int rnnls_set_stream(rnnls_ctx *ctx, void *stream);

/* Cap the number of SMs the large-n sketch kernel of this context occupies
 * (one resident block per SM); 0 (the default) means every SM.  Leaving a
 * few SMs free lets solves enqueued on other streams run beside a sketch
 * instead of waiting for it.  Results do not depend on the cap.
 * Errors: EINVAL (ctx null or sms < 0). */
int rnnls_set_sketch_sms(rnnls_ctx *ctx, int sms);

/* Set / read the context's launch-shape choices (rnnls_tuning).  Later
 * calls on the context use them.  Errors: EINVAL (null pointer, a field
 * out of range, reserved not zero). */
int rnnls_set_tuning(rnnls_ctx *ctx, const rnnls_tuning *t);
int rnnls_get_tuning(rnnls_ctx *ctx, rnnls_tuning *t);

/* Scheduling aid (not part of the method): `event` (a cudaEvent_t, borrowed;
 * NULL to stop) is recorded on the context stream by every FP32 sketch call
 * once its row sampling and plan launches are enqueued, before the transform
 * launch (at the start of the call for n <= 8192, which has no plan).  Work
 * on other streams that waits on it starts after the plan, so it does not
 * delay the plan launch, and runs beside the transform.  Errors: EINVAL
 * (ctx null). */
int rnnls_set_plan_event(rnnls_ctx *ctx, void *event);

/* Sketch of Alg. 1 steps 1-4 for FP32 data:
 *   SA[k, j] = s * sum_i H_n[idx[k], i] D_ii A[i, j]   (k < r_out, j < d)
 *   Sb[k]    = s * sum_i H_n[idx[k], i] D_ii b[i]
 * with s the row scale above and H_n unnormalised (entries +-1).
 * A: n_raw x d, leading dimension lda >= n_raw.  b: n_raw.
 * SA: cap x d, leading dimension ldsa >= cap.  Sb: cap.  idx: cap int32
 * (nullable): the sampled rows, draw order (iid) or increasing (Bernoulli).
 * cap must be >= r in iid mode; in Bernoulli mode a count above cap
 * returns ECAPACITY (size cap as r + 6 sqrt(r) + 16, or n when r >= n).
 * r_out (HOST, nullable) receives the number of rows; in Bernoulli mode
 * this synchronises the stream.  Requires n_raw >= 1, d >= 1, r >= 1,
 * n_raw <= 2^28.  A and b need not be 16-byte aligned (aligned is faster).
 * Accuracy: FP32 accumulation; relative Frobenius error vs FP64 about
 * 1e-7 * sqrt(log2 n).  Errors: EINVAL (null A, b, SA or Sb; a size < 1;
 * lda < n_raw; ldsa < cap; unknown flags; cap < r in iid mode; nothing is
 * enqueued then), EUNSUPPORTED (n_raw > 2^28, d > 2^20, r > 2^30),
 * ECAPACITY, ENOMEM, ECUDA.  flags: one RNNLS_SAMPLE_* value, or'ed with
 * one RNNLS_PREC_* value (in RNNLS_PREC_BF16X2 mode a sketch with more than
 * 24,576 rows per plan group is formed in several passes over A, each for
 * a share of the rows). */
int rnnls_sketch(rnnls_ctx *ctx, const float *A, int64_t lda, const float *b, int64_t n_raw, int64_t d,
                 int64_t r, uint64_t seed, uint64_t instance, uint32_t flags, float *SA, int64_t ldsa, float *Sb,
                 int32_t *idx, int64_t cap, int64_t *r_out);

/* Sketch shared by several targets (the multiple right-hand-side problem
 * min_{x_t >= 0} ||A x_t - B[:, t]||, which Sec. 5 lists as an extension;
 * one S H D is applied to X = [A | B]):
 *   SA[k, j] = s * sum_i H_n[idx[k], i] D_ii A[i, j]      (j < d)
 *   SB[k, t] = s * sum_i H_n[idx[k], i] D_ii B[i, t]      (t < nrhs)
 * iid sampling (r rows, s = 1/sqrt(r)), the same rows and signs as
 * rnnls_sketch with the same seed and instance (which is the nrhs = 1 case).
 * A: n_raw x d, lda >= n_raw.  B: n_raw x nrhs, ldb >= n_raw.  SA: r x d,
 * ldsa >= r.  SB: r x nrhs, ldsb >= r.  idx: r int32 (nullable).  All device,
 * column-major, caller-owned.  Errors: EINVAL (null pointer, a size < 1, a
 * leading dimension too small), EUNSUPPORTED (n_raw > 2^28 or
 * d + nrhs > 2^20), ENOMEM, ECUDA. */
int rnnls_sketch_multi(rnnls_ctx *ctx, const float *A, int64_t lda, const float *B, int64_t ldb, int64_t n_raw,
                       int64_t d, int64_t nrhs, int64_t r, uint64_t seed, uint64_t instance, float *SA, int64_t ldsa,
                       float *SB, int64_t ldsb, int32_t *idx);

/* Part of the sketch contributed by rows row0 .. row0 + rows - 1 of the
 * full problem (A: n_raw x d, b: n_raw).  H_n = H_G (x) H_{n/G} for any
 * split into row blocks, so with P_g this function's output for block g,
 *   sum_g P_g = the output of rnnls_sketch (iid mode, same seed/instance),
 * which lets each GPU sketch only the rows it holds and one sum-reduce of
 * r x (d + 1) floats finish the sketch.  A and b hold ONLY the shard's rows
 * that carry data, v = min(rows, n_raw - row0) of them (A: v x d,
 * lda >= max(v, 1); b: v); the shard's rows past n_raw are zero.
 * n_raw is the full problem's row count (it fixes the padding, the sampled
 * rows and D).  row0 must be a multiple of 16384 and below the padded n;
 * rows >= 1.  SA: r x d (ldsa >= r), Sb: r, idx: r (nullable; the full
 * problem's sampled rows, the same in every shard).  row0 = 0 with
 * rows >= n_raw is exactly rnnls_sketch; other shards need n > 8192
 * (EUNSUPPORTED otherwise).  Errors: EINVAL, EUNSUPPORTED, ENOMEM, ECUDA. */
int rnnls_sketch_shard(rnnls_ctx *ctx, const float *A, int64_t lda, const float *b, int64_t n_raw, int64_t row0,
                       int64_t rows, int64_t d, int64_t r, uint64_t seed, uint64_t instance, float *SA, int64_t ldsa,
                       float *Sb, int32_t *idx);

/* One instance of a batched sketch (rnnls_sketch_batched): the arguments
 * of rnnls_sketch in iid mode with cap = r (all device pointers; idx must not
 * be null). */
typedef struct rnnls_sketch_job {
  const float *A;
  int64_t lda;
  const float *b;
  int64_t n_raw;
  int64_t d;
  int64_t r;
  uint64_t seed;
  uint64_t instance;
  float *SA;
  int64_t ldsa;
  float *Sb;
  int32_t *idx;
} rnnls_sketch_job;

/* The sketches of `count` independent instances of Alg. 1 (uneven sizes),
 * each exactly as rnnls_sketch in iid mode would give it (up to the FP32
 * summation order), computed together: one launch draws every instance's
 * rows, one makes every plan, and one persistent kernel walks all the
 * instances' chunk groups.  `jobs` is a HOST array (count = 0 enqueues
 * nothing); each job's pointers are device pointers with the layouts of
 * rnnls_sketch (ldsa >= r, lda >= n_raw).
 * Errors: EINVAL (a null pointer or a bad size in any job; nothing is
 * enqueued then), EUNSUPPORTED (n_raw > 2^28), ENOMEM, ECUDA. */
int rnnls_sketch_batched(rnnls_ctx *ctx, const rnnls_sketch_job *jobs, int64_t count);

/* rnnls_sketch_batched with a precision flag (RNNLS_PREC_FP32 or
 * RNNLS_PREC_BF16X2, see above; the same rows in both).  Errors: those of
 * rnnls_sketch_batched, and EINVAL for any other flag bit. */
int rnnls_sketch_batched_ex(rnnls_ctx *ctx, const rnnls_sketch_job *jobs, int64_t count, uint32_t flags);

/* rnnls_sketch for a sparse A held by columns (compressed sparse column),
 * the form of the paper's term-document data (Sec. 4.1, 4.2): the same iid
 * rows, signs and 1/sqrt(r) scale, so SA and Sb equal rnnls_sketch's of
 * the dense A to FP32 rounding.  Column j's non-zeros are rowidx[p], val[p]
 * for colptr[j] <= p < colptr[j + 1] (int64 offsets, colptr[0] = 0, row
 * indices ascending within a column and in [0, n_raw); entries that break
 * the order are skipped); b is dense (n_raw).  All pointers are device
 * pointers; rowidx and val may be null when every column is empty.
 * The transform still runs over every row (n log2(4096) additions per
 * column); the read of A is 8 bytes per non-zero.  Limits: padded n >= 4096
 * (n_raw > 2048) and r <= 16384 (EUNSUPPORTED otherwise), iid rows only.
 * idx (nullable) receives the r sampled rows.  Scratch lives in the
 * context.  Errors: EINVAL (null colptr, b, SA or Sb; a size < 1;
 * ldsa < r), EUNSUPPORTED, ENOMEM, ECUDA. */
int rnnls_sketch_csc(rnnls_ctx *ctx, const int64_t *colptr, const int32_t *rowidx, const float *val, const float *b,
                     int64_t n_raw, int64_t d, int64_t r, uint64_t seed, uint64_t instance, float *SA, int64_t ldsa,
                     float *Sb, int32_t *idx);

/* The same sketch in FP64 throughout (for FP64 inputs), with the same
 * arguments, sampling, scale and errors as rnnls_sketch; every sum is
 * formed in FP64. */
int rnnls_sketch_f64(rnnls_ctx *ctx, const double *A, int64_t lda, const double *b, int64_t n_raw, int64_t d,
                     int64_t r, uint64_t seed, uint64_t instance, uint32_t flags, double *SA, int64_t ldsa,
                     double *Sb, int32_t *idx, int64_t cap, int64_t *r_out);

/* Small NNLS of Alg. 1 step 5:  x = argmin_{x >= 0} ||SA x - Sb||^2,
 * SA r x d (ldsa >= r), Sb r, FP32 device data; x (device, FP64, d) and
 * info (device, nullable).  Lawson-Hanson rules: start at x = 0 (Sec. 4.1);
 * add argmax_j w_j (ties to the smallest j) while it exceeds info->tol;
 * a candidate whose passive solve gives z_t <= 0 or a dependent column
 * (pivot^2 <= 1e-13 Q_tt) is rejected for that selection; interpolate with
 * alpha = min x_j/(x_j - z_j) (ties to the smallest j) and drop x_j <= 0;
 * caps 3d additions and 30d interpolation solves (EMAXITER).
 * Q = SA'SA and q = SA'Sb are formed as rnnls_gram forms them (tensor
 * cores, exact slice products).  The iterations run in FP32 (an inverse of
 * the equilibrated passive block, FP32 duals); their end point is checked
 * in float-float (a refined passive solve must be positive, the float-float
 * dual must not exceed tol off the passive set).  If a check fails the
 * solve continues from that point with every passive solve refined and the
 * dual in float-float, so every decision is taken on refined values;
 * info->accurate_mode records which check sent it there.  Requires 1 <= d <= 1024 (for d
 * above about 230 the passive-block inverse is kept in the context's
 * workspace instead of shared memory),
 * r >= 1.  A return of RNNLS_OK means the work was enqueued; the solve's
 * own outcome is info->status (RNNLS_ENONFINITE with x = 0 when SA or Sb
 * holds a NaN or an infinity).  Errors: EINVAL (null SA, Sb or x; r < 1;
 * d < 1; ldsa < r), EUNSUPPORTED (d > 1024), ENOMEM, ECUDA. */
int rnnls_solve(rnnls_ctx *ctx, const float *SA, int64_t ldsa, const float *Sb, int64_t r, int64_t d, double *x,
                rnnls_info *info);

/* The same solve for FP64 sketches (same rules, limits and errors; the
 * Gram is summed in FP64). */
int rnnls_solve_f64(rnnls_ctx *ctx, const double *SA, int64_t ldsa, const double *Sb, int64_t r, int64_t d,
                    double *x, rnnls_info *info);

/* Sketch moments of Sec. 3.4 (the quadratic-programming form of the small
 * problem): Q = X'X for X = [SA | Sb], i.e. Q~ = SA'SA in the leading d x d
 * block, q~ = SA'Sb in row and column d, ||Sb||^2 at (d, d).
 * SA: r x d FP32 column-major (ldsa >= r), Sb: r, device.  Q: device FP64,
 * (d + 1) x (d + 1) row-major (symmetric, every entry written).  colabs:
 * device FP64, d entries sum_k |SA_kj| (nullable).
 * Arithmetic: each column j is scaled by the power of two that brings its
 * largest magnitude into [64, 128) and cut into six 8-bit integer slices
 * (exact in BF16); the slice products are summed exactly on the tcgen05
 * tensor cores (FP32 accumulators drained before their integer sums reach
 * 2^24) and the drained sums are added in float-float arithmetic.  The
 * error is below about 2^-40 max_k|SA_ki| max_k|SA_kj| per row, plus the
 * float-float rounding (about 2^-44 relative).  Data must stay in the FP32
 * exponent range (Gram entries between about 1e-30 and 1e30).  A NaN or
 * an infinity in a column makes that column's entries of Q NaN.
 * Errors: EINVAL (null ctx, SA, Sb or Q; r < 1; d < 1; ldsa < r),
 * EUNSUPPORTED (d > 1024), ENOMEM, ECUDA. */
int rnnls_gram(rnnls_ctx *ctx, const float *SA, int64_t ldsa, const float *Sb, int64_t r, int64_t d, double *Q,
               double *colabs);

/* The small NNLS problem of Alg. 1 step 5 by an iterative method on the
 * quadratic-programming form of Sec. 3.4 (min x'Qx - 2q'x over x >= 0 with
 * Q = SA'SA, q = SA'Sb formed as rnnls_gram forms them), for d beyond the
 * active-set solve's limit: accelerated projected gradient (FISTA) with
 * gradient-based restarts on the diagonally equilibrated problem
 * (y = x / D, D = diag(Q)^-1/2), each iteration one O(d^2) product with Q~
 * (float-float) spread over all SMs in one cooperative launch.
 * Stops when the equilibrated gradient map is small:
 *   max_j L |z_j - max(0, z_j - g_j / L)| <= tol * max_j |D_j q_j|
 * (L >= the largest eigenvalue of DQD), or after max_iter iterations.
 * The result approaches the unique minimiser (SA of full column rank) at a
 * rate that depends on cond(DQD); it is not the exact active set of
 * rnnls_solve, but within the stated residual of it.
 * SA: r x d FP32 column-major (ldsa >= r), Sb: r, device; x: device FP64 d;
 * info (device, nullable): status (OK, EMAXITER, ENONFINITE, ETIMEOUT when
 * the launch's grid barrier gave up), outer_iters = iterations,
 * inner_iters = restarts, passive_count = positive entries, tol = the
 * residual threshold used, dual_max = max of q - Qx over the zero entries,
 * objective = ||SA x - Sb||^2.  Requires 1 <= d <= 8192 (EUNSUPPORTED
 * above), tol > 0, max_iter >= 1.  Errors: EINVAL, EUNSUPPORTED, ENOMEM,
 * ECUDA. */
int rnnls_solve_pg(rnnls_ctx *ctx, const float *SA, int64_t ldsa, const float *Sb, int64_t r, int64_t d, double *x,
                   rnnls_info *info, double tol, int max_iter);

/* The small NNLS problems of Alg. 1 step 5 for nrhs targets that share one
 * sketch (rnnls_sketch_multi): X[:, t] = argmin_{x >= 0} ||SA x - SB[:, t]||_2
 * for t < nrhs, each by the Lawson-Hanson method of rnnls_solve with the
 * same rules and tolerance; the Gram of SA is formed once for all targets.
 * SA: r x d (ldsa >= r), SB: r x nrhs (ldsb >= r), FP32, device.  X: device
 * FP64 d x nrhs, column-major, ldx >= d.  infos: device, nrhs entries
 * (nullable).  Requires 1 <= d <= 1024 (EUNSUPPORTED otherwise).  Errors:
 * EINVAL, EUNSUPPORTED, ENOMEM, ECUDA; each target's own outcome is
 * infos[t].status. */
int rnnls_solve_multi(rnnls_ctx *ctx, const float *SA, int64_t ldsa, const float *SB, int64_t ldsb, int64_t r,
                      int64_t d, int64_t nrhs, double *X, int64_t ldx, rnnls_info *infos);

/* Many independent small NNLS problems in one launch sequence (one
 * Lawson-Hanson block per problem, uneven d and r allowed, each d <= 1024).
 * `probs` is a HOST array of `count` descriptors whose pointers are device
 * pointers; flags must be 0.  count = 0 enqueues nothing.  Each problem's
 * own outcome is its info->status.  Errors: EINVAL (a null pointer, a bad
 * size in any problem, nonzero flags; nothing is enqueued then),
 * EUNSUPPORTED (a d above 1024), ENOMEM, ECUDA. */
int rnnls_solve_batched(rnnls_ctx *ctx, const rnnls_problem *probs, int64_t count, uint32_t flags);

/* rnnls_solve_batched with the descriptor array in DEVICE memory (count
 * rnnls_problem entries, device pointers inside), as a scheduler that
 * builds its batches on the GPU or inside a CUDA graph would hold it.  The
 * host cannot read the descriptors, so it passes bounds: every problem must
 * have 1 <= r <= max_r and 1 <= d <= max_d (max_d <= 1024).  A kernel plans
 * the batch on the device (tiles, K-splits, offsets) and every problem gets
 * a workspace slot of the bounds' size; a descriptor outside the bounds or
 * with a null pointer is not solved and its info (when given) gets status
 * RNNLS_EINVAL.  Results equal rnnls_solve_batched's.  Errors: EINVAL
 * (null ctx, null array with count > 0, count < 0, a bound < 1, flags != 0),
 * EUNSUPPORTED (max_d > 1024), ENOMEM, ECUDA. */
int rnnls_solve_batched_device(rnnls_ctx *ctx, const rnnls_problem *d_probs, int64_t count, int64_t max_r,
                               int64_t max_d, uint32_t flags);

/* Repeated RandomizedNNLS (the footnote to Theorem 1 in Sec. 1: a few
 * independent repetitions raise the success probability of the (1 + eps)
 * bound from 1/2 to at least 1 - 2^-k).  Run j (j < k) is Alg. 1 exactly as
 * rnnls_sketch (iid rows, seed, instance instance0 + j) followed by
 * rnnls_solve; the answer is the run with the smallest full residual
 * ||A x_j - b||^2 among the runs whose solve ended with status OK (ties to
 * the smallest j; run 0 when none did).  The residuals are evaluated in one
 * pass over A: row dot products in FP32 on FP32 copies of x_j, squared row
 * residuals summed in FP64.
 * A: n_raw x d FP32 column-major (lda >= n_raw), b: n_raw, device.
 * Outputs (device, caller-owned): x (FP64, d) the kept run's solution;
 * resid (FP64, k, nullable) every run's residual; best (int32, 1, nullable)
 * the kept run's j; info (nullable) the kept run's solve info.
 * Requires 1 <= k <= 16 and d <= 256 (EUNSUPPORTED otherwise).  Scratch (k
 * sketches, k solutions) lives in the context and is reused by the next
 * call.  Errors: EINVAL (null pointer, a size < 1, lda < n_raw),
 * EUNSUPPORTED, ENOMEM, ECUDA. */
int rnnls_solve_boosted(rnnls_ctx *ctx, const float *A, int64_t lda, const float *b, int64_t n_raw, int64_t d,
                        int64_t r, uint64_t seed, uint64_t instance0, int k, double *x, double *resid, int32_t *best,
                        rnnls_info *info);

/* Objective of Definition 1 on the full data: out[0] = ||A x - b||^2 with
 * A n x d (lda >= n) and b FP32, x FP64 (device), accumulated in FP64.
 * out: device double.  Errors: EINVAL (a null pointer, n < 1, d < 1,
 * lda < n), ENOMEM, ECUDA. */
int rnnls_residual(rnnls_ctx *ctx, const float *A, int64_t lda, const float *b, int64_t n, int64_t d,
                   const double *x, double *out);

/* Launch profiling (tracing aid, not part of the method).  Between
 * rnnls_profile_begin and rnnls_profile_end the context records a CUDA
 * event pair on its stream around each of its kernel launches (at most
 * max_launches).  rnnls_profile_end synchronises the stream and writes one
 * entry per kernel kind (HOST array `out` of capacity max_out): the kernel
 * name, its launch count and the summed event time in milliseconds.
 * *n_out receives the number of entries written.  Errors: EINVAL (null
 * context or out, max_launches < 1), ENOMEM, ECUDA. */
typedef struct rnnls_kernel_time {
  char name[32];
  int64_t launches;
  double total_ms;
} rnnls_kernel_time;

int rnnls_profile_begin(rnnls_ctx *ctx, int max_launches);
int rnnls_profile_end(rnnls_ctx *ctx, rnnls_kernel_time *out, int max_out, int *n_out);

/* rnnls_sketch without any memory allocation (the paper has no counterpart:
 * this is a deployment convenience).  For callers that cannot call
 * cudaMalloc when they need a sketch -- a frozen or fully reserved memory
 * pool, a real-time loop that must not enter the allocator (it may
 * synchronise the device), a host that only hands out registered buffers.
 * Computes exactly what rnnls_sketch computes in iid mode (r uniform row
 * draws, same Philox streams and scale), enqueued on `stream` (a
 * cudaStream_t, NULL = legacy default stream) of the current device.
 * Inputs and outputs are the caller's, as in rnnls_sketch (idx nullable);
 * all scratch lives in one 8 MiB array compiled into the library, which
 * every GPU on which this entry point has been called holds until the
 * process exits.
 * Set-up: the first call on a device (and the first call after the current
 * context changed, e.g. after cudaDeviceReset) looks up that device's
 * address of the array (cudaGetSymbolAddress) with the device current.
 * With lazy module loading the driver also reserves the array and the
 * kernels' code on that device at this first call, so make one first
 * (warm-up) call while device memory is still free, and before any stream
 * capture; later calls allocate nothing.  Every call shares the array and
 * overwrites all of the scratch it reads (nothing needs clearing), so calls
 * whose work overlaps on the GPU (other streams, other threads) race:
 * serialise them.
 * Limits: 1 <= r <= 16384 (RNNLS_EUNSUPPORTED above), n_raw <= 2^28;
 * large column counts get fewer chunk groups (less parallelism) so that the
 * partial sums fit.  Calls no cudaMalloc, cudaFree or allocating library
 * routine.  Errors: EINVAL (null pointer, bad size or stride),
 * EUNSUPPORTED (r above the limit, n_raw above 2^28, a current device
 * ordinal of 64 or more), ECUDA (the set-up's address lookup or a launch
 * failed). */
int rnnls_sketch_noalloc(void *stream, const float *A, int64_t lda, const float *b, int64_t n_raw, int64_t d,
                         int64_t r, uint64_t seed, uint64_t instance, float *SA, int64_t ldsa, float *Sb,
                         int32_t *idx);

/* Human-readable text of a status code (static storage). */
const char *rnnls_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* RNNLS_H */
