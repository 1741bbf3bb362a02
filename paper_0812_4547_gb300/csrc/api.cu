// api.cu -- the C ABI declared in include/rnnls.h: context, workspace,
// argument checks and dispatch to the sampling, sketch and solve kernels.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "kernels.h"

namespace rnnls {

int ensure_workspace(rnnls_ctx *ctx, size_t bytes) {
  if (bytes <= ctx->ws_bytes) return RNNLS_OK;
  // in-flight work on the context stream may still use the old buffer
  RNNLS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  if (ctx->ws) cudaFree(ctx->ws);
  ctx->ws = nullptr;
  ctx->ws_bytes = 0;
  const size_t want = align_up(bytes + bytes / 4, 1 << 20);
  if (cudaMalloc(&ctx->ws, want) != cudaSuccess) {
    cudaGetLastError();
    return RNNLS_ENOMEM;
  }
  ctx->ws_bytes = want;
  return RNNLS_OK;
}

int ensure_aux(rnnls_ctx *ctx, size_t bytes) {
  if (bytes <= ctx->aux_bytes) return RNNLS_OK;
  RNNLS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  if (ctx->aux) cudaFree(ctx->aux);
  ctx->aux = nullptr;
  ctx->aux_bytes = 0;
  const size_t want = align_up(bytes + bytes / 4, 1 << 16);
  if (cudaMalloc(&ctx->aux, want) != cudaSuccess) {
    cudaGetLastError();
    return RNNLS_ENOMEM;
  }
  ctx->aux_bytes = want;
  return RNNLS_OK;
}

int ensure_counters(rnnls_ctx *ctx, size_t n, unsigned int **out) {
  if (n > ctx->counters_len) {
    RNNLS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    if (ctx->counters) cudaFree(ctx->counters);
    ctx->counters = nullptr;
    ctx->counters_len = 0;
    const size_t want = align_up(n, 1024);
    if (cudaMalloc(&ctx->counters, want * sizeof(unsigned int)) != cudaSuccess) {
      cudaGetLastError();
      return RNNLS_ENOMEM;
    }
    RNNLS_CUDA_TRY(cudaMemset(ctx->counters, 0, want * sizeof(unsigned int)));
    ctx->counters_len = want;
  }
  *out = ctx->counters;
  return RNNLS_OK;
}

int ensure_pinned(rnnls_ctx *ctx, size_t bytes) {
  // the previous copy out of the staging buffer must be complete
  RNNLS_CUDA_TRY(cudaEventSynchronize(ctx->pinned_ready));
  if (bytes <= ctx->pinned_bytes) return RNNLS_OK;
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  ctx->pinned = nullptr;
  ctx->pinned_bytes = 0;
  const size_t want = align_up(bytes + bytes / 4, 4096);
  if (cudaMallocHost(&ctx->pinned, want) != cudaSuccess) {
    cudaGetLastError();
    return RNNLS_ENOMEM;
  }
  ctx->pinned_bytes = want;
  return RNNLS_OK;
}

const char *kernel_name(int kid) {
  static const char *names[K_COUNT] = {"sample_rows", "build_plan", "sketch_srht_f32", "sketch_small",
                                       "reduce_partials", "sketch_f64", "gram", "gram_reduce", "colabs",
                                       "lawson_hanson", "residual", "boost_residual", "boost_select",
                                       "colstats", "gram_tc", "projected_gradient",
                                       "sketch_csc"};
  return (kid >= 0 && kid < K_COUNT) ? names[kid] : "?";
}

}  // namespace rnnls

using namespace rnnls;

namespace {

// Makes a context's device current while an entry point runs and gives the
// caller's current device back when it returns (so that a call never moves
// the calling thread to another device).
struct device_guard {
  int prev = -1;
  cudaError_t set(int dev) {
    cudaError_t e = cudaGetDevice(&prev);
    if (e != cudaSuccess || prev == dev) {
      prev = -1;
      return e;
    }
    e = cudaSetDevice(dev);
    if (e != cudaSuccess) prev = -1;
    return e;
  }
  ~device_guard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

constexpr int64_t kMaxRows = (int64_t)1 << 28;
// Largest d of the small NNLS (beyond about 230 the passive-block inverse
// leaves shared memory for the workspace)
constexpr int64_t kMaxSolveD = 1024;

// Device layout of the auxiliary buffer: [count (int64) | sampled rows (int32)].
struct aux_view {
  int64_t *d_count;
  int32_t *idx;
  void *bern_ws;
};

int get_aux(rnnls_ctx *ctx, int64_t cap, int64_t n, bool need_idx, aux_view &v) {
  const size_t b_count = 256;
  const size_t b_idx = need_idx ? align_up((size_t)cap * sizeof(int32_t), 256) : 0;
  const size_t b_bern = bernoulli_ws_bytes(n);
  int st = ensure_aux(ctx, b_count + b_idx + b_bern);
  if (st) return st;
  char *base = (char *)ctx->aux;
  v.d_count = (int64_t *)base;
  v.idx = need_idx ? (int32_t *)(base + b_count) : nullptr;
  v.bern_ws = base + b_count + b_idx;
  return RNNLS_OK;
}

template <typename T>
int check_sketch_args(rnnls_ctx *ctx, const T *A, int64_t lda, const T *b, int64_t n_raw, int64_t d, int64_t r,
                      uint32_t flags, T *SA, int64_t ldsa, T *Sb, int64_t cap, uint32_t allowed = RNNLS_SAMPLE_MASK) {
  if (!ctx || !A || !b || !SA || !Sb) return RNNLS_EINVAL;
  if (n_raw < 1 || d < 1 || r < 1 || cap < 1) return RNNLS_EINVAL;
  if (lda < n_raw || ldsa < cap) return RNNLS_EINVAL;
  if (flags & ~allowed) return RNNLS_EINVAL;
  if ((flags & RNNLS_SAMPLE_MASK) == RNNLS_SAMPLE_IID && cap < r) return RNNLS_EINVAL;
  if (n_raw > kMaxRows || d > (1 << 20) || r > ((int64_t)1 << 30)) return RNNLS_EUNSUPPORTED;
  return RNNLS_OK;
}

// Sampling shared by both precisions; fills a.idx / count and the scale.
int sample_rows(rnnls_ctx *ctx, int L, int64_t r, uint64_t seed, uint64_t instance, uint32_t flags, int32_t *idx,
                int64_t cap, aux_view &av, double &scale) {
  const int64_t n = (int64_t)1 << L;
  const bool bern = (flags & RNNLS_SAMPLE_MASK) == RNNLS_SAMPLE_BERNOULLI;
  int st;
  prof_scope ps(ctx, K_SAMPLE);
  if (bern) {
    st = launch_sample_bernoulli(ctx->stream, seed, instance, L, r, idx, cap, av.d_count, av.bern_ws);
    scale = (r >= n) ? 1.0 / sqrt((double)n) : 1.0 / sqrt((double)r);
  } else {
    st = launch_sample_iid(ctx->stream, seed, instance, L, r, idx);
    scale = 1.0 / sqrt((double)r);
  }
  return st;
}

int read_count(rnnls_ctx *ctx, const aux_view &av, int64_t cap, int64_t *r_out) {
  int st = ensure_pinned(ctx, sizeof(int64_t));
  if (st) return st;
  RNNLS_CUDA_TRY(cudaMemcpyAsync(ctx->pinned, av.d_count, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
  RNNLS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  const int64_t cnt = *(int64_t *)ctx->pinned;
  *r_out = cnt < cap ? cnt : cap;
  return cnt > cap ? RNNLS_ECAPACITY : RNNLS_OK;
}

}  // namespace

extern "C" {

int rnnls_create(rnnls_ctx **out, int device, void *stream) {
  if (!out) return RNNLS_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return RNNLS_ECUDA;
  }
  device_guard dg;
  RNNLS_CUDA_TRY(dg.set(device));
  rnnls_ctx *ctx = new (std::nothrow) rnnls_ctx();
  if (!ctx) return RNNLS_ENOMEM;
  memset(ctx, 0, sizeof(*ctx));
  ctx->device = device;
  ctx->stream = (cudaStream_t)stream;
  if (cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaDeviceGetAttribute(&ctx->max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->pinned_ready, cudaEventDisableTiming) != cudaSuccess) {
    delete ctx;
    return RNNLS_ECUDA;
  }
  *out = ctx;
  return RNNLS_OK;
}

static void profile_free(rnnls_ctx *ctx) {
  if (ctx->prof_ev) {
    for (int i = 0; i < 2 * ctx->prof_cap; ++i) cudaEventDestroy(ctx->prof_ev[i]);
    delete[] ctx->prof_ev;
    delete[] ctx->prof_kid;
  }
  ctx->prof_ev = nullptr;
  ctx->prof_kid = nullptr;
  ctx->prof_cap = 0;
  ctx->prof_n = 0;
  ctx->prof_on = 0;
}

int rnnls_profile_begin(rnnls_ctx *ctx, int max_launches) {
  if (!ctx || max_launches < 1) return RNNLS_EINVAL;
  device_guard dg;
  RNNLS_CUDA_TRY(dg.set(ctx->device));
  if (ctx->prof_cap < max_launches) {
    RNNLS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    profile_free(ctx);
    ctx->prof_ev = new (std::nothrow) cudaEvent_t[2 * (size_t)max_launches];
    ctx->prof_kid = new (std::nothrow) int[(size_t)max_launches];
    if (!ctx->prof_ev || !ctx->prof_kid) {
      delete[] ctx->prof_ev;
      delete[] ctx->prof_kid;
      ctx->prof_ev = nullptr;
      ctx->prof_kid = nullptr;
      return RNNLS_ENOMEM;
    }
    for (int i = 0; i < 2 * max_launches; ++i) {
      if (cudaEventCreate(&ctx->prof_ev[i]) != cudaSuccess) {
        cudaGetLastError();
        ctx->prof_cap = i / 2;  // profile_free destroys the 2 * prof_cap events made so far ...
        if (i & 1) cudaEventDestroy(ctx->prof_ev[i - 1]);  // ... and this pair's first one here
        profile_free(ctx);
        return RNNLS_ECUDA;
      }
    }
    ctx->prof_cap = max_launches;
  }
  ctx->prof_n = 0;
  ctx->prof_on = 1;
  return RNNLS_OK;
}

int rnnls_profile_end(rnnls_ctx *ctx, rnnls_kernel_time *out, int max_out, int *n_out) {
  if (!ctx || !out || max_out < 1) return RNNLS_EINVAL;
  ctx->prof_on = 0;
  RNNLS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  double tot[K_COUNT] = {0};
  int64_t cnt[K_COUNT] = {0};
  for (int i = 0; i < ctx->prof_n; ++i) {
    float ms = 0.0f;
    RNNLS_CUDA_TRY(cudaEventElapsedTime(&ms, ctx->prof_ev[2 * i], ctx->prof_ev[2 * i + 1]));
    tot[ctx->prof_kid[i]] += ms;
    cnt[ctx->prof_kid[i]] += 1;
  }
  int n = 0;
  for (int k = 0; k < K_COUNT && n < max_out; ++k) {
    if (!cnt[k]) continue;
    memset(out[n].name, 0, sizeof(out[n].name));
    strncpy(out[n].name, kernel_name(k), sizeof(out[n].name) - 1);
    out[n].launches = cnt[k];
    out[n].total_ms = tot[k];
    ++n;
  }
  if (n_out) *n_out = n;
  ctx->prof_n = 0;
  return RNNLS_OK;
}

int rnnls_destroy(rnnls_ctx *ctx) {
  if (!ctx) return RNNLS_EINVAL;
  device_guard dg;
  dg.set(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  profile_free(ctx);
  if (ctx->ws) cudaFree(ctx->ws);
  if (ctx->aux) cudaFree(ctx->aux);
  if (ctx->boost) cudaFree(ctx->boost);
  if (ctx->counters) cudaFree(ctx->counters);
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  cudaEventDestroy(ctx->pinned_ready);
  delete ctx;
  return RNNLS_OK;
}

int rnnls_set_stream(rnnls_ctx *ctx, void *stream) {
  if (!ctx) return RNNLS_EINVAL;
  ctx->stream = (cudaStream_t)stream;
  return RNNLS_OK;
}

int rnnls_set_plan_event(rnnls_ctx *ctx, void *event) {
  if (!ctx) return RNNLS_EINVAL;
  ctx->plan_event = (cudaEvent_t)event;
  return RNNLS_OK;
}

int rnnls_set_sketch_sms(rnnls_ctx *ctx, int sms) {
  if (!ctx || sms < 0) return RNNLS_EINVAL;
  ctx->sketch_sms = sms;
  ctx->tune.sketch_sms = sms;
  return RNNLS_OK;
}

int rnnls_set_tuning(rnnls_ctx *ctx, const rnnls_tuning *t) {
  if (!ctx || !t) return RNNLS_EINVAL;
  auto in = [](int v, int lo, int hi) { return v == 0 || (v >= lo && v <= hi); };
  if (t->sketch_sms < 0 || !in(t->full_step_min_slots, 48, 1024) || !in(t->gram_min_chunks, 1, 65536) ||
      !in(t->gram_max_splits, 1, 1024) || !in(t->batch_gram_chunks, 1, 65536) ||
      !in(t->batch_step_cost, 1, 100000) || !in(t->lh_warp_max_d, 1, 1024) ||
      t->reserved != 0)
    return RNNLS_EINVAL;
  ctx->tune = *t;
  ctx->sketch_sms = t->sketch_sms;
  return RNNLS_OK;
}

int rnnls_get_tuning(rnnls_ctx *ctx, rnnls_tuning *t) {
  if (!ctx || !t) return RNNLS_EINVAL;
  *t = ctx->tune;
  t->sketch_sms = ctx->sketch_sms;
  return RNNLS_OK;
}

int rnnls_sketch(rnnls_ctx *ctx, const float *A, int64_t lda, const float *b, int64_t n_raw, int64_t d, int64_t r,
                 uint64_t seed, uint64_t instance, uint32_t flags, float *SA, int64_t ldsa, float *Sb, int32_t *idx,
                 int64_t cap, int64_t *r_out) {
  int st = check_sketch_args(ctx, A, lda, b, n_raw, d, r, flags, SA, ldsa, Sb, cap, RNNLS_SAMPLE_MASK | RNNLS_PREC_MASK);
  if (st) return st;
  device_guard dg;
  RNNLS_CUDA_TRY(dg.set(ctx->device));
  const int L = log2_ceil64(n_raw);
  const bool bern = (flags & RNNLS_SAMPLE_MASK) == RNNLS_SAMPLE_BERNOULLI;
  const int64_t rows = bern ? cap : r;
  aux_view av;
  st = get_aux(ctx, rows, (int64_t)1 << L, idx == nullptr, av);
  if (st) return st;
  int32_t *rows_idx = idx ? idx : av.idx;
  double scale = 0.0;
  // iid rows for the large-n path are drawn inside the sketch's plan kernel
  const bool fused_iid = !bern && ((int64_t)1 << L) > 8192;
  if (fused_iid) {
    scale = 1.0 / sqrt((double)r);
  } else {
    st = sample_rows(ctx, L, r, seed, instance, flags, rows_idx, rows, av, scale);
    if (st) return st;
  }
  sketch_args_f32 a;
  a.gen_iid = fused_iid ? 1 : 0;
  a.A = A;
  a.lda = lda;
  a.b = b;
  a.n_raw = n_raw;
  a.d = (int)d;
  a.L = L;
  a.r = rows;
  a.d_count = bern ? av.d_count : nullptr;
  a.seed = seed;
  a.inst = instance;
  a.scale = (float)scale;
  a.SA = SA;
  a.ldsa = ldsa;
  a.Sb = Sb;
  a.ldb = n_raw;
  a.nb = 1;
  a.ldsb = ldsa;
  a.chunk0 = 0;
  a.idx = rows_idx;
  a.tc = (flags & RNNLS_PREC_MASK) == RNNLS_PREC_BF16X2 ? 1 : 0;
  st = sketch_f32(ctx, a, ctx->num_sms);
  if (st) return st;
  if (r_out) {
    if (!bern) {
      *r_out = r;
    } else {
      st = read_count(ctx, av, cap, r_out);
      if (st) return st;
    }
  }
  return RNNLS_OK;
}

int rnnls_sketch_multi(rnnls_ctx *ctx, const float *A, int64_t lda, const float *B, int64_t ldb, int64_t n_raw,
                       int64_t d, int64_t nrhs, int64_t r, uint64_t seed, uint64_t instance, float *SA, int64_t ldsa,
                       float *SB, int64_t ldsb, int32_t *idx) {
  if (!ctx || !A || !B || !SA || !SB) return RNNLS_EINVAL;
  if (n_raw < 1 || d < 1 || nrhs < 1 || r < 1 || lda < n_raw || ldb < n_raw || ldsa < r || ldsb < r)
    return RNNLS_EINVAL;
  if (n_raw > kMaxRows || d + nrhs > (1 << 20) || r > ((int64_t)1 << 30)) return RNNLS_EUNSUPPORTED;
  device_guard dg;
  RNNLS_CUDA_TRY(dg.set(ctx->device));
  const int L = log2_ceil64(n_raw);
  aux_view av;
  int st = get_aux(ctx, r, (int64_t)1 << L, idx == nullptr, av);
  if (st) return st;
  int32_t *rows_idx = idx ? idx : av.idx;
  const bool fused_iid = ((int64_t)1 << L) > 8192;
  double scale = 1.0 / sqrt((double)r);
  if (!fused_iid) {
    st = sample_rows(ctx, L, r, seed, instance, RNNLS_SAMPLE_IID, rows_idx, r, av, scale);
    if (st) return st;
  }
  sketch_args_f32 a;
  a.gen_iid = fused_iid ? 1 : 0;
  a.A = A;
  a.lda = lda;
  a.b = B;
  a.ldb = ldb;
  a.nb = (int)nrhs;
  a.n_raw = n_raw;
  a.d = (int)d;
  a.L = L;
  a.chunk0 = 0;
  a.r = r;
  a.d_count = nullptr;
  a.seed = seed;
  a.inst = instance;
  a.scale = (float)scale;
  a.SA = SA;
  a.ldsa = ldsa;
  a.Sb = SB;
  a.ldsb = ldsb;
  a.idx = rows_idx;
  return sketch_f32(ctx, a, ctx->num_sms);
}

int rnnls_sketch_shard(rnnls_ctx *ctx, const float *A, int64_t lda, const float *b, int64_t n_raw, int64_t row0,
                       int64_t rows, int64_t d, int64_t r, uint64_t seed, uint64_t instance, float *SA, int64_t ldsa,
                       float *Sb, int32_t *idx) {
  if (!ctx || !A || !b || !SA || !Sb) return RNNLS_EINVAL;
  if (n_raw < 1 || d < 1 || r < 1 || rows < 1 || row0 < 0 || ldsa < r) return RNNLS_EINVAL;
  if (lda < std::max<int64_t>(1, std::min<int64_t>(rows, n_raw - row0))) return RNNLS_EINVAL;
  if (n_raw > kMaxRows || d > (1 << 20) || r > ((int64_t)1 << 30)) return RNNLS_EUNSUPPORTED;
  const int L = log2_ceil64(n_raw);
  const int64_t n = (int64_t)1 << L;
  const int64_t group_rows = 4 * (int64_t)kM;  // shards start on a group of four chunks
  if (row0 % group_rows != 0 || row0 >= n) return RNNLS_EINVAL;
  // the whole problem in one piece: the plain sketch (also covers n <= 2^13)
  if (row0 == 0 && rows >= n_raw)
    return rnnls_sketch(ctx, A, lda, b, n_raw, d, r, seed, instance, RNNLS_SAMPLE_IID, SA, ldsa, Sb, idx, r, nullptr);
  if (n <= 8192) return RNNLS_EUNSUPPORTED;
  device_guard dg;
  RNNLS_CUDA_TRY(dg.set(ctx->device));
  aux_view av;
  int st = get_aux(ctx, r, n, idx == nullptr, av);
  if (st) return st;
  sketch_args_f32 a;
  a.gen_iid = 1;
  a.A = A;
  a.lda = lda;
  a.b = b;
  a.ldb = lda;
  a.nb = 1;
  // rows of this shard that hold data; the rest (and the padding) are zero
  a.n_raw = std::max<int64_t>(0, std::min<int64_t>(rows, n_raw - row0));
  a.d = (int)d;
  a.L = L;
  a.chunk0 = row0 / kM;
  a.r = r;
  a.d_count = nullptr;
  a.seed = seed;
  a.inst = instance;
  a.scale = (float)(1.0 / sqrt((double)r));
  a.SA = SA;
  a.ldsa = ldsa;
  a.Sb = Sb;
  a.ldsb = ldsa;
  a.idx = idx ? idx : av.idx;
  if (a.n_raw == 0) {
    // no data in this shard: its part is zero (the rows are still drawn)
    RNNLS_CUDA_TRY(cudaMemset2DAsync(SA, (size_t)ldsa * sizeof(float), 0, (size_t)r * sizeof(float), (size_t)d,
                                     ctx->stream));
    RNNLS_CUDA_TRY(cudaMemsetAsync(Sb, 0, (size_t)r * sizeof(float), ctx->stream));
    double scale = 0.0;
    return sample_rows(ctx, L, r, seed, instance, RNNLS_SAMPLE_IID, a.idx, r, av, scale);
  }
  return sketch_f32(ctx, a, ctx->num_sms);
}

int rnnls_sketch_batched(rnnls_ctx *ctx, const rnnls_sketch_job *jobs, int64_t count) {
  return rnnls_sketch_batched_ex(ctx, jobs, count, 0u);
}

int rnnls_sketch_batched_ex(rnnls_ctx *ctx, const rnnls_sketch_job *jobs, int64_t count, uint32_t flags) {
  if (!ctx || (!jobs && count > 0) || count < 0 || (flags & ~RNNLS_PREC_MASK)) return RNNLS_EINVAL;
  for (int64_t i = 0; i < count; ++i) {
    const rnnls_sketch_job &j = jobs[i];
    if (!j.A || !j.b || !j.SA || !j.Sb || !j.idx) return RNNLS_EINVAL;
    if (j.n_raw < 1 || j.d < 1 || j.r < 1 || j.lda < j.n_raw || j.ldsa < j.r) return RNNLS_EINVAL;
    if (j.n_raw > kMaxRows || j.d > (1 << 20) || j.r > ((int64_t)1 << 30)) return RNNLS_EUNSUPPORTED;
  }
  if (count == 0) return RNNLS_OK;
  device_guard dg;
  RNNLS_CUDA_TRY(dg.set(ctx->device));
  return sketch_batched_f32(ctx, jobs, count, (flags & RNNLS_PREC_MASK) == RNNLS_PREC_BF16X2 ? 1 : 0);
}

int rnnls_sketch_f64(rnnls_ctx *ctx, const double *A, int64_t lda, const double *b, int64_t n_raw, int64_t d,
                     int64_t r, uint64_t seed, uint64_t instance, uint32_t flags, double *SA, int64_t ldsa, double *Sb,
                     int32_t *idx, int64_t cap, int64_t *r_out) {
  int st = check_sketch_args(ctx, A, lda, b, n_raw, d, r, flags, SA, ldsa, Sb, cap);
  if (st) return st;
  device_guard dg;
  RNNLS_CUDA_TRY(dg.set(ctx->device));
  const int L = log2_ceil64(n_raw);
  const bool bern = (flags & RNNLS_SAMPLE_MASK) == RNNLS_SAMPLE_BERNOULLI;
  const int64_t rows = bern ? cap : r;
  aux_view av;
  st = get_aux(ctx, rows, (int64_t)1 << L, idx == nullptr, av);
  if (st) return st;
  int32_t *rows_idx = idx ? idx : av.idx;
  double scale = 0.0;
  st = sample_rows(ctx, L, r, seed, instance, flags, rows_idx, rows, av, scale);
  if (st) return st;
  sketch_args_f64 a;
  a.A = A;
  a.lda = lda;
  a.b = b;
  a.n_raw = n_raw;
  a.d = (int)d;
  a.L = L;
  a.r = rows;
  a.d_count = bern ? av.d_count : nullptr;
  a.seed = seed;
  a.inst = instance;
  a.scale = scale;
  a.SA = SA;
  a.ldsa = ldsa;
  a.Sb = Sb;
  a.idx = rows_idx;
  st = sketch_f64(ctx, a);
  if (st) return st;
  if (r_out) {
    if (!bern) {
      *r_out = r;
    } else {
      st = read_count(ctx, av, cap, r_out);
      if (st) return st;
    }
  }
  return RNNLS_OK;
}

int rnnls_solve(rnnls_ctx *ctx, const float *SA, int64_t ldsa, const float *Sb, int64_t r, int64_t d, double *x,
                rnnls_info *info) {
  if (!ctx || !SA || !Sb || !x || r < 1 || d < 1 || ldsa < r) return RNNLS_EINVAL;
  if (d > kMaxSolveD) return RNNLS_EUNSUPPORTED;
  device_guard dg;
  RNNLS_CUDA_TRY(dg.set(ctx->device));
  return solve_f32(ctx, SA, ldsa, Sb, r, d, x, info);
}

int rnnls_gram(rnnls_ctx *ctx, const float *SA, int64_t ldsa, const float *Sb, int64_t r, int64_t d, double *Q,
               double *colabs) {
  if (!ctx || !SA || !Sb || !Q || r < 1 || d < 1 || ldsa < r) return RNNLS_EINVAL;
  if (d > kMaxSolveD) return RNNLS_EUNSUPPORTED;
  device_guard dg;
  RNNLS_CUDA_TRY(dg.set(ctx->device));
  return gram_f32(ctx, SA, ldsa, Sb, r, d, Q, colabs);
}

int rnnls_solve_pg(rnnls_ctx *ctx, const float *SA, int64_t ldsa, const float *Sb, int64_t r, int64_t d, double *x,
                   rnnls_info *info, double tol, int max_iter) {
  if (!ctx || !SA || !Sb || !x || r < 1 || d < 1 || ldsa < r || !(tol > 0.0) || max_iter < 1) return RNNLS_EINVAL;
  if (d > kMaxSolvePgD) return RNNLS_EUNSUPPORTED;
  device_guard dg;
  RNNLS_CUDA_TRY(dg.set(ctx->device));
  return solve_pg_f32(ctx, SA, ldsa, Sb, r, d, x, info, tol, max_iter);
}

int rnnls_sketch_csc(rnnls_ctx *ctx, const int64_t *colptr, const int32_t *rowidx, const float *val, const float *b,
                     int64_t n_raw, int64_t d, int64_t r, uint64_t seed, uint64_t instance, float *SA, int64_t ldsa,
                     float *Sb, int32_t *idx) {
  if (!ctx || !colptr || !b || !SA || !Sb || n_raw < 1 || d < 1 || r < 1 || ldsa < r) return RNNLS_EINVAL;
  if (n_raw > ((int64_t)1 << 31) - 1 || d > (1 << 20)) return RNNLS_EUNSUPPORTED;
  device_guard dg;
  RNNLS_CUDA_TRY(dg.set(ctx->device));
  return sketch_csc_f32(ctx, colptr, rowidx, val, b, n_raw, d, r, seed, instance, SA, ldsa, Sb, idx);
}

int rnnls_solve_batched_device(rnnls_ctx *ctx, const rnnls_problem *d_probs, int64_t count, int64_t max_r,
                               int64_t max_d, uint32_t flags) {
  if (!ctx || (!d_probs && count > 0) || count < 0 || max_r < 1 || max_d < 1 || flags != 0) return RNNLS_EINVAL;
  if (max_d > kMaxSolveD || count > ((int64_t)1 << 31) - 1) return RNNLS_EUNSUPPORTED;
  device_guard dg;
  RNNLS_CUDA_TRY(dg.set(ctx->device));
  return solve_batched_device(ctx, d_probs, count, max_r, max_d);
}

int rnnls_solve_f64(rnnls_ctx *ctx, const double *SA, int64_t ldsa, const double *Sb, int64_t r, int64_t d,
                    double *x, rnnls_info *info) {
  if (!ctx || !SA || !Sb || !x || r < 1 || d < 1 || ldsa < r) return RNNLS_EINVAL;
  if (d > kMaxSolveD) return RNNLS_EUNSUPPORTED;
  device_guard dg;
  RNNLS_CUDA_TRY(dg.set(ctx->device));
  return solve_f64(ctx, SA, ldsa, Sb, r, d, x, info);
}

int rnnls_solve_batched(rnnls_ctx *ctx, const rnnls_problem *probs, int64_t count, uint32_t flags) {
  if (!ctx || (!probs && count > 0) || count < 0 || flags != 0) return RNNLS_EINVAL;
  for (int64_t i = 0; i < count; ++i) {
    const rnnls_problem &p = probs[i];
    if (!p.SA || !p.Sb || !p.x || p.r < 1 || p.d < 1 || p.ldsa < p.r) return RNNLS_EINVAL;
    if (p.d > kMaxSolveD) return RNNLS_EUNSUPPORTED;
  }
  if (count == 0) return RNNLS_OK;
  device_guard dg;
  RNNLS_CUDA_TRY(dg.set(ctx->device));
  return solve_batched(ctx, probs, count);
}

int rnnls_solve_multi(rnnls_ctx *ctx, const float *SA, int64_t ldsa, const float *SB, int64_t ldsb, int64_t r,
                      int64_t d, int64_t nrhs, double *X, int64_t ldx, rnnls_info *infos) {
  if (!ctx || !SA || !SB || !X) return RNNLS_EINVAL;
  if (r < 1 || d < 1 || nrhs < 1 || ldsa < r || ldsb < r || ldx < d) return RNNLS_EINVAL;
  if (d > kMaxSolveD) return RNNLS_EUNSUPPORTED;
  device_guard dg;
  RNNLS_CUDA_TRY(dg.set(ctx->device));
  return solve_multi(ctx, SA, ldsa, SB, ldsb, r, d, nrhs, X, ldx, infos);
}

int rnnls_residual(rnnls_ctx *ctx, const float *A, int64_t lda, const float *b, int64_t n, int64_t d,
                   const double *x, double *out) {
  if (!ctx || !A || !b || !x || !out || n < 1 || d < 1 || lda < n) return RNNLS_EINVAL;
  device_guard dg;
  RNNLS_CUDA_TRY(dg.set(ctx->device));
  return residual_f32(ctx, A, lda, b, n, d, x, out);
}

int rnnls_solve_boosted(rnnls_ctx *ctx, const float *A, int64_t lda, const float *b, int64_t n_raw, int64_t d,
                        int64_t r, uint64_t seed, uint64_t instance0, int k, double *x, double *resid, int32_t *best,
                        rnnls_info *info) {
  if (!ctx || !A || !b || !x || n_raw < 1 || d < 1 || r < 1 || lda < n_raw || k < 1) return RNNLS_EINVAL;
  if (k > kBoostMaxK || d > kBoostMaxD || n_raw > kMaxRows || r > ((int64_t)1 << 30)) return RNNLS_EUNSUPPORTED;
  device_guard dg;
  RNNLS_CUDA_TRY(dg.set(ctx->device));
  return solve_boosted_f32(ctx, A, lda, b, n_raw, d, r, seed, instance0, k, x, resid, best, info);
}

const char *rnnls_strerror(int status) {
  switch (status) {
    case RNNLS_OK: return "ok";
    case RNNLS_EINVAL: return "invalid argument";
    case RNNLS_ECAPACITY: return "sampled rows exceed the output capacity";
    case RNNLS_ENONFINITE: return "non-finite value in the sketch's Gram matrix";
    case RNNLS_ESINGULAR: return "passive-set system numerically singular";
    case RNNLS_EMAXITER: return "Lawson-Hanson iteration cap reached";
    case RNNLS_ETIMEOUT: return "bounded device wait gave up";
    case RNNLS_ECUDA: return "CUDA runtime error";
    case RNNLS_ENOMEM: return "workspace allocation failed";
    case RNNLS_EUNSUPPORTED: return "size outside what this build supports";
    default: return "unknown status";
  }
}

}  // extern "C"
