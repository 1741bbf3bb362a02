// boost.cu -- repeated RandomizedNNLS: k independent runs, best full residual kept.
//
// The footnote to Theorem 1 (Sec. 1) notes that a few repetitions raise the
// algorithm's success probability: each run meets the (1 + eps) residual
// bound with probability at least 1/2, so the best of k independent runs
// misses it with probability at most 2^-k.  Repetition j uses the
// randomness (seed, instance0 + j).  The k sketches go through one batched
// sketch (one launch each for the rows, the plans and the transforms), the
// k small problems through one batched solve; one pass over A then
// evaluates all k residuals ||A x_j - b||^2, and a one-block kernel keeps
// the smallest among the runs whose solve ended with status OK (ties to the
// smallest j; repetition 0 when none did).
#include <math.h>
#include <string.h>

#include <vector>

#include "kernels.h"

namespace rnnls {
namespace {

constexpr int kResThreads = 256;
// rows of A per thread in flight (more for few runs, where the pass is a
// plain stream over A)
__host__ __device__ constexpr int res_rows(int K) { return K <= 4 ? 8 : 4; }

// Partial sums of ||A x_j - b||^2 over this block's rows, for j < K.
// A: n x d column-major (lda >= n), b: n, X: d x K FP64 column-major (ldx).
// Row dot products run in FP32 (fused multiply-adds, columns in order) on
// FP32 copies of x_j; each row's squared residual is accumulated in FP64.
// partial: [block][K], summed in a fixed order by the select kernel.
template <int K>
__global__ void __launch_bounds__(kResThreads, K <= 8 ? 2 : 1) boost_residual_kernel(const float *__restrict__ A, int64_t lda,
                                                                     const float *__restrict__ b, int64_t n, int d,
                                                                     const double *__restrict__ X, int64_t ldx,
                                                                     double *__restrict__ partial) {
  __shared__ float xs[kBoostMaxD][K];
  __shared__ double red[kResThreads / 32][K];
  constexpr int kResRows = res_rows(K);
  for (int e = threadIdx.x; e < d * K; e += kResThreads) {
    const int c = e / K, j = e - c * K;
    xs[c][j] = (float)X[(int64_t)j * ldx + c];
  }
  __syncthreads();
  double acc[K];
#pragma unroll
  for (int j = 0; j < K; ++j) acc[j] = 0.0;
  const int64_t span = (int64_t)kResThreads * kResRows;
  for (int64_t base = (int64_t)blockIdx.x * span + threadIdx.x; base < n; base += (int64_t)gridDim.x * span) {
    float t[kResRows][K];
#pragma unroll
    for (int u = 0; u < kResRows; ++u)
#pragma unroll
      for (int j = 0; j < K; ++j) t[u][j] = 0.0f;
#pragma unroll 4
    for (int c = 0; c < d; ++c) {
      const float *col = A + (int64_t)c * lda;
      float a[kResRows];
#pragma unroll
      for (int u = 0; u < kResRows; ++u) {
        const int64_t i = base + (int64_t)u * kResThreads;
        a[u] = (i < n) ? __ldcs(col + i) : 0.0f;
      }
#pragma unroll
      for (int j = 0; j < K; ++j) {
        const float xv = xs[c][j];
#pragma unroll
        for (int u = 0; u < kResRows; ++u) t[u][j] = fmaf(a[u], xv, t[u][j]);
      }
    }
#pragma unroll
    for (int u = 0; u < kResRows; ++u) {
      const int64_t i = base + (int64_t)u * kResThreads;
      if (i < n) {
        const float bi = b[i];
#pragma unroll
        for (int j = 0; j < K; ++j) {
          const double rr = (double)(t[u][j] - bi);
          acc[j] = fma(rr, rr, acc[j]);
        }
      }
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    double v = acc[j];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][j] = v;
  }
  __syncthreads();
  if (threadIdx.x < K) {
    double v = 0.0;
    for (int w = 0; w < kResThreads / 32; ++w) v += red[w][threadIdx.x];
    partial[(int64_t)blockIdx.x * K + threadIdx.x] = v;
  }
}

// Residuals of the k runs (block partials summed in a fixed order), the kept
// run (smallest residual among status-OK runs, ties to the smallest j,
// run 0 if none), its x, index and info.
__global__ void boost_select_kernel(const double *__restrict__ partial, int nblk, int K, int k,
                                    const rnnls_info *__restrict__ infos, const double *__restrict__ X, int64_t ldx,
                                    int d, double *__restrict__ x_out, double *__restrict__ resid_out,
                                    int32_t *__restrict__ best_out, rnnls_info *__restrict__ info_out) {
  __shared__ double res[kBoostMaxK];
  __shared__ double red[32];
  __shared__ int best_s;
  const int tid = threadIdx.x;
  // run j's residual: thread t sums blocks t, t + blockDim.x, ..., then the
  // threads' sums are added in a fixed tree order
  for (int j = 0; j < k; ++j) {
    double v = 0.0;
    for (int q = tid; q < nblk; q += blockDim.x) v += partial[(int64_t)q * K + j];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
      res[j] = t;
    }
    __syncthreads();
  }
  if (tid == 0) {
    int best = -1;
    for (int j = 0; j < k; ++j) {
      const bool ok = infos[j].status == RNNLS_OK && isfinite(res[j]);
      if (ok && (best < 0 || res[j] < res[best])) best = j;
    }
    best_s = best < 0 ? 0 : best;
  }
  __syncthreads();
  const int best = best_s;
  for (int c = tid; c < d; c += blockDim.x) x_out[c] = X[(int64_t)best * ldx + c];
  if (resid_out && tid < k) resid_out[tid] = res[tid];
  if (tid == 0) {
    if (best_out) *best_out = best;
    if (info_out) *info_out = infos[best];
  }
}

int ensure_boost(rnnls_ctx *ctx, size_t bytes) {
  if (bytes <= ctx->boost_bytes) return RNNLS_OK;
  RNNLS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  if (ctx->boost) cudaFree(ctx->boost);
  ctx->boost = nullptr;
  ctx->boost_bytes = 0;
  const size_t want = align_up(bytes + bytes / 4, 1 << 16);
  if (cudaMalloc(&ctx->boost, want) != cudaSuccess) {
    cudaGetLastError();
    return RNNLS_ENOMEM;
  }
  ctx->boost_bytes = want;
  return RNNLS_OK;
}

template <int K>
void launch_residual(cudaStream_t s, int nblk, const float *A, int64_t lda, const float *b, int64_t n, int d,
                     const double *X, int64_t ldx, double *partial) {
  boost_residual_kernel<K><<<nblk, kResThreads, 0, s>>>(A, lda, b, n, d, X, ldx, partial);
}

}  // namespace

int solve_boosted_f32(rnnls_ctx *ctx, const float *A, int64_t lda, const float *b, int64_t n_raw, int64_t d,
                      int64_t r, uint64_t seed, uint64_t instance0, int k, double *x, double *resid, int32_t *best,
                      rnnls_info *info) {
  cudaStream_t s = ctx->stream;
  const int K = k <= 1 ? 1 : k <= 2 ? 2 : k <= 4 ? 4 : k <= 8 ? 8 : 16;
  const int64_t span = (int64_t)kResThreads * res_rows(K);
  const int nblk = (int)std::max<int64_t>(1, std::min<int64_t>(2 * (int64_t)ctx->num_sms, (n_raw + span - 1) / span));
  // scratch: k sketches (SA r x d, Sb, rows), X (d x K), infos, block partials
  const size_t b_sa = align_up((size_t)k * r * d * sizeof(float), 256);
  const size_t b_sb = align_up((size_t)k * r * sizeof(float), 256);
  const size_t b_idx = align_up((size_t)k * r * sizeof(int32_t), 256);
  const size_t b_x = align_up((size_t)K * d * sizeof(double), 256);
  const size_t b_info = align_up((size_t)k * sizeof(rnnls_info), 256);
  const size_t b_part = align_up((size_t)nblk * K * sizeof(double), 256);
  int st = ensure_boost(ctx, b_sa + b_sb + b_idx + b_x + b_info + b_part);
  if (st) return st;
  char *p = (char *)ctx->boost;
  float *SA = (float *)p;
  float *Sb = (float *)(p += b_sa);
  int32_t *idx = (int32_t *)(p += b_sb);
  double *X = (double *)(p += b_idx);
  rnnls_info *infos = (rnnls_info *)(p += b_x);
  double *partial = (double *)(p += b_info);
  // the residual kernel reads K columns of X: runs k .. K-1 are zero
  if (K > k) RNNLS_CUDA_TRY(cudaMemsetAsync(X + (size_t)k * d, 0, (size_t)(K - k) * d * sizeof(double), s));

  std::vector<rnnls_sketch_job> jobs((size_t)k);
  std::vector<rnnls_problem> probs((size_t)k);
  for (int j = 0; j < k; ++j) {
    rnnls_sketch_job &J = jobs[(size_t)j];
    memset(&J, 0, sizeof(J));
    J.A = A; J.lda = lda; J.b = b; J.n_raw = n_raw; J.d = d; J.r = r; J.seed = seed; J.instance = instance0 + j;
    J.SA = SA + (size_t)j * r * d; J.ldsa = r; J.Sb = Sb + (size_t)j * r; J.idx = idx + (size_t)j * r;
    rnnls_problem &P = probs[(size_t)j];
    P.SA = J.SA; P.ldsa = r; P.Sb = J.Sb; P.r = r; P.d = d; P.x = X + (size_t)j * d; P.info = infos + j;
  }
  st = sketch_batched_f32(ctx, jobs.data(), k);
  if (st) return st;
  st = solve_batched(ctx, probs.data(), k);
  if (st) return st;
  {
    prof_scope ps(ctx, K_BOOST_RES);
    switch (K) {
      case 1: launch_residual<1>(s, nblk, A, lda, b, n_raw, (int)d, X, d, partial); break;
      case 2: launch_residual<2>(s, nblk, A, lda, b, n_raw, (int)d, X, d, partial); break;
      case 4: launch_residual<4>(s, nblk, A, lda, b, n_raw, (int)d, X, d, partial); break;
      case 8: launch_residual<8>(s, nblk, A, lda, b, n_raw, (int)d, X, d, partial); break;
      default: launch_residual<16>(s, nblk, A, lda, b, n_raw, (int)d, X, d, partial); break;
    }
    if (cudaGetLastError() != cudaSuccess) return RNNLS_ECUDA;
  }
  {
    prof_scope ps(ctx, K_BOOST_SEL);
    boost_select_kernel<<<1, 256, 0, s>>>(partial, nblk, K, k, infos, X, d, (int)d, x, resid, best, info);
    if (cudaGetLastError() != cudaSuccess) return RNNLS_ECUDA;
  }
  return RNNLS_OK;
}

}  // namespace rnnls
