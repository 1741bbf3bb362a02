// kernels.h -- host-side launchers shared between the translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace rnnls {

// ---- sampling (sample.cu) -------------------------------------------------
// idx[k] = top L bits of word k of stream 2, k < r.
int launch_sample_iid(cudaStream_t s, uint64_t seed, uint64_t inst, int L, int64_t r, int32_t *idx);
// Bernoulli rows in increasing order; count written to *d_count (device);
// rows beyond cap are dropped (the count still reports the true total).
size_t bernoulli_ws_bytes(int64_t n);
int launch_sample_bernoulli(cudaStream_t s, uint64_t seed, uint64_t inst, int L, int64_t r, int32_t *idx,
                            int64_t cap, int64_t *d_count, void *ws);

// ---- combine plan (sample.cu) ----------------------------------------------
// Chunk size of the large-n sketch: 2^kLogM rows.
constexpr int kLogM = 12;
constexpr int kM = 1 << kLogM;
constexpr int kThreads = 256;                 // threads of a sketch block
constexpr int kWorkers = 4;                   // chunks transformed together
constexpr int kMaxSlots = 128;                // plan rows per sketch thread (TMEM columns)
constexpr int kPlanMaxRows = kThreads * kMaxSlots;  // rows per plan group

struct plan_t {
  uint32_t *pk;   // [kgroups][slots][kThreads]
  int32_t *k;     // [kgroups][slots][kThreads]
  int slots;
  int kgroups;
  int64_t rows_per_group;
};
size_t plan_ws_bytes(int slots, int kgroups);
// The plan of the sampled rows; with a sign table the same launch also
// writes the first sign_words sign words of D.  gen_L = 0: the rows are
// read from idx (drawn before); gen_L > 0: the launch draws the r iid rows
// of an n = 2^gen_L problem itself and writes them to idx.
int launch_build_plan(cudaStream_t s, int32_t *idx, int64_t r, const int64_t *d_count, plan_t plan,
                      uint64_t *sign_table, int64_t sign_words, int64_t sign_block0, uint64_t seed, uint64_t inst,
                      int gen_L = 0);

// Many instances' rows and plans in one launch each (iid rows; a sign table
// per instance, its words counted from the instance's first chunk).
struct plan_job {
  int32_t *idx;
  int64_t r;
  uint32_t *pk;
  int32_t *k;
  int slots, kgroups, L;
  int64_t rows_per_group;
  uint64_t seed, inst;
  uint64_t *signs;
  int64_t sign_words;
};
int64_t sample_blocks(int64_t r);
int64_t plan_blocks(const plan_job &j);
int launch_plan_batched(cudaStream_t s, const plan_job *d_jobs, const int64_t *d_first_sample,
                        const int64_t *d_first_plan, int count, int64_t sample_total, int64_t plan_total);

// ---- sketch (sketch.cu) ------------------------------------------------------
// Columns of X = [A | B]: d columns of A, then nb columns of B (nb = 1: the
// target b).  A row shard (rows chunk0 * 2^12 ... of the full problem, A and
// B holding only those rows) gives its additive part of the full sketch.
struct sketch_args_f32 {
  const float *A;
  int64_t lda;
  const float *b;     // B (nb columns, leading dimension ldb)
  int64_t ldb;
  int nb;
  int64_t n_raw;      // rows of A / B with data (of the shard)
  int d;
  int L;              // log2 of the padded row count of the full problem
  int64_t chunk0;     // full-problem index of the first 2^12-row chunk (multiple of 4)
  int64_t r;          // rows (iid) or capacity bound (Bernoulli)
  const int64_t *d_count;  // device row count (Bernoulli) or null
  uint64_t seed, inst;
  float scale;
  float *SA;
  int64_t ldsa;
  float *Sb;          // SB (nb columns, leading dimension ldsb)
  int64_t ldsb;
  int32_t *idx;
  int gen_iid;  // 1: the sketch draws the iid rows itself (idx is output only)
  int tc = 0;   // 1: split-precision mode (pass 1 on the tensor cores, RNNLS_PREC_BF16X2)
};
int sketch_f32(rnnls_ctx *ctx, const sketch_args_f32 &a, int num_sms);
// many instances (iid rows, FP32): rows, plans and sketches of all in one launch each
int sketch_batched_f32(rnnls_ctx *ctx, const rnnls_sketch_job *jobs, int64_t count, int tc = 0);
// sketch_f32 with caller-provided scratch (no allocation; see noalloc.cu)
int sketch_f32_scratch(cudaStream_t s, const sketch_args_f32 &a, int num_sms, void *scratch, size_t bytes);

struct sketch_args_f64 {
  const double *A;
  int64_t lda;
  const double *b;
  int64_t n_raw;
  int d;
  int L;
  int64_t r;
  const int64_t *d_count;
  uint64_t seed, inst;
  double scale;
  double *SA;
  int64_t ldsa;
  double *Sb;
  const int32_t *idx;
};
int sketch_f64(rnnls_ctx *ctx, const sketch_args_f64 &a);

// ---- tensor-core Gram (gram_tc.cu) --------------------------------------------
// Q = X'X for X = [S | s_0 .. s_{nb-1}] (m rows, c = d + nb columns), exact
// to about 2^-40 of the column maxima's products per row, written as FP64
// (Qd) and float pairs (Qhi + Qlo), c x c row-major, plus colabs[g] =
// sum_k |S_kg| for g < d.  multi = 1: products between two different target
// columns are not needed (tiles holding none of them and no diagonal entry
// are skipped).
constexpr int kGramTileM = 128;
constexpr int kGramTileN = 64;
struct gram_tc_job {
  const float *S, *s;
  int64_t lds, ldt, m;
  int d, nb, c, multi;
  int tiles, splits, vec4;
  int64_t chunks_per_split;  // 32-row chunks per K-split
  float *colscale;           // [2c] the two factors of 2^(7 - E_g)
  float *colunscale;         // [c] 2^(E_g - 7)
  double *part;              // [splits][tiles][128 * 64] partial tiles (splits > 1)
  unsigned int *counters;    // [tiles] zeroed completion counters
  double *Qd;
  float *Qhi, *Qlo;
  double *colabs;
};
// Tile (mt, nt) = rows 128 mt.., columns 64 nt.. of Q; kept when it holds an
// entry on or above the diagonal (and, with multi, a row of S or a diagonal
// entry).
__host__ __device__ inline bool gram_tc_tile_needed(int mt, int nt, int c, int d, int multi) {
  const int i0 = mt * kGramTileM, j0 = nt * kGramTileN;
  if (i0 >= c || j0 >= c) return false;
  const int i1 = i0 + kGramTileM < c ? i0 + kGramTileM : c;
  const int j1 = j0 + kGramTileN < c ? j0 + kGramTileN : c;
  if (j1 - 1 < i0) return false;
  if (multi && i0 >= d) return j0 < i1 && j1 > i0;
  return true;
}
__host__ __device__ inline void gram_tc_tile_at(int t, int c, int d, int multi, int &mt, int &nt) {
  for (int a = 0; a * kGramTileM < c; ++a)
    for (int b = 0; b * kGramTileN < c; ++b)
      if (gram_tc_tile_needed(a, b, c, d, multi)) {
        if (t == 0) {
          mt = a;
          nt = b;
          return;
        }
        --t;
      }
  mt = nt = 0;
}
__host__ __device__ inline int gram_tc_tile_count(int c, int d, int multi) {
  int n = 0;
  for (int mt = 0; mt * kGramTileM < c; ++mt)
    for (int nt = 0; nt * kGramTileN < c; ++nt) n += gram_tc_tile_needed(mt, nt, c, d, multi) ? 1 : 0;
  return n;
}
// K-splits of a problem of m rows with `tiles` tiles (fields splits and
// chunks_per_split of gram_tc_job): about want_ctas CTAs, at least
// min_chunks chunks of 32 rows per CTA when the problem allows, at most
// max_splits splits, at most max_chunks_per_cta chunks per CTA.
__host__ __device__ inline void gram_tc_splits(int64_t m, int tiles, int want_ctas, int64_t max_chunks_per_cta,
                                               int min_chunks, int max_splits, int &splits_out, int64_t &cps_out) {
  const int64_t chunks = m > 32 ? (m + 31) / 32 : 1;
  int64_t splits = ((int64_t)want_ctas + tiles - 1) / tiles;
  if (splits < 1) splits = 1;
  const int64_t by_min = chunks / min_chunks > 1 ? chunks / min_chunks : 1;
  if (splits > max_splits) splits = max_splits;
  if (splits > by_min) splits = by_min;
  const int64_t by_max = (chunks + max_chunks_per_cta - 1) / max_chunks_per_cta;
  if (splits < by_max) splits = by_max;
  cps_out = (chunks + splits - 1) / splits;
  splits_out = (int)((chunks + cps_out - 1) / cps_out);
}
// Tiles and K-splits of one problem: about want_ctas CTAs, at most
// max_chunks_per_cta and (if the problem allows) at least min_chunks chunks
// of 32 rows each, at most max_splits splits (pointers left for gram_tc_carve).
gram_tc_job gram_tc_plan(const float *S, int64_t lds, const float *s, int64_t ldt, int nb, int64_t m, int d,
                         int multi, int want_ctas, int64_t max_chunks_per_cta, int min_chunks, int max_splits);
// the context's choices of the above (rnnls_tuning), defaults 8 and 32
inline int gram_min_chunks(const rnnls_ctx *ctx) { return tune_or(ctx->tune.gram_min_chunks, 8); }
inline int gram_max_splits(const rnnls_ctx *ctx) { return tune_or(ctx->tune.gram_max_splits, 32); }
size_t gram_tc_ws_bytes(const gram_tc_job &j);
void gram_tc_carve(gram_tc_job &j, ws_carver &wc, unsigned int *counters, double *Qd, float *Qhi, float *Qlo,
                   double *colabs);
// column statistics, then the Gram (two launches)
int gram_tc_launch_one(rnnls_ctx *ctx, const gram_tc_job &j);
int gram_tc_launch_batched(rnnls_ctx *ctx, const gram_tc_job *d_jobs, const int64_t *d_first_col,
                           const int64_t *d_first_cta, int count, int64_t cols, int64_t ctas);
// rnnls_gram: Q (FP64, (d+1) x (d+1)) and colabs (nullable) into caller buffers
int gram_f32(rnnls_ctx *ctx, const float *SA, int64_t ldsa, const float *Sb, int64_t r, int64_t d, double *Q,
             double *colabs);

// ---- solve (solve.cu) ----------------------------------------------------------
int solve_f32(rnnls_ctx *ctx, const float *SA, int64_t ldsa, const float *Sb, int64_t r, int64_t d, double *x,
              rnnls_info *info);
int solve_f64(rnnls_ctx *ctx, const double *SA, int64_t ldsa, const double *Sb, int64_t r, int64_t d, double *x,
              rnnls_info *info);
int solve_batched(rnnls_ctx *ctx, const rnnls_problem *probs, int64_t count);
// the same from a device-resident descriptor array (plan made on the device)
int solve_batched_device(rnnls_ctx *ctx, const rnnls_problem *d_probs, int64_t count, int64_t max_r, int64_t max_d);
// nrhs targets sharing one sketch SA: X (d x nrhs, leading dimension ldx), infos nrhs (nullable)
int solve_multi(rnnls_ctx *ctx, const float *SA, int64_t ldsa, const float *SB, int64_t ldsb, int64_t r, int64_t d,
                int64_t nrhs, double *X, int64_t ldx, rnnls_info *infos);
// repeated runs (rnnls_solve_boosted); k <= kBoostMaxK, d <= kBoostMaxD
constexpr int kBoostMaxK = 16;
constexpr int kBoostMaxD = 256;
int solve_boosted_f32(rnnls_ctx *ctx, const float *A, int64_t lda, const float *b, int64_t n_raw, int64_t d,
                      int64_t r, uint64_t seed, uint64_t instance0, int k, double *x, double *resid, int32_t *best,
                      rnnls_info *info);
// sketch of a sparse A in compressed columns (sparse.cu)
int sketch_csc_f32(rnnls_ctx *ctx, const int64_t *colptr, const int32_t *rowidx, const float *val, const float *b,
                   int64_t n_raw, int64_t d, int64_t r, uint64_t seed, uint64_t instance, float *SA, int64_t ldsa,
                   float *Sb, int32_t *idx);
// iterative solve on the quadratic-programming form (pg.cu); d <= kMaxSolvePgD
constexpr int64_t kMaxSolvePgD = 8192;
int solve_pg_f32(rnnls_ctx *ctx, const float *SA, int64_t ldsa, const float *Sb, int64_t r, int64_t d, double *x,
                 rnnls_info *info, double tol, int max_iter);
int residual_f32(rnnls_ctx *ctx, const float *A, int64_t lda, const float *b, int64_t n, int64_t d,
                 const double *x, double *out);

}  // namespace rnnls
