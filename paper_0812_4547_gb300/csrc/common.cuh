// common.cuh -- shared device helpers of the GB300 RandomizedNNLS library.
//
// Philox4x64-10 (Salmon, Moraes, Dror & Shaw, SC'11) for the +-1 diagonal D
// (Alg. 1 step 4) and the row sampling S (Alg. 1 step 2); compensated
// single-precision pair arithmetic ("float-float", Dekker 1971 / Knuth
// TwoSum) used where the solve needs more than FP32 and GB300's FP64 rate is
// too low; context and workspace bookkeeping.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rnnls.h"

#define RNNLS_CUDA_TRY(expr)                      \
  do {                                            \
    cudaError_t _e = (expr);                      \
    if (_e != cudaSuccess) return RNNLS_ECUDA;    \
  } while (0)

namespace rnnls {

// ---------------------------------------------------------------------------
// Philox4x64-10.  key = (seed, instance); counter = (j, stream, 0, 0).
// ---------------------------------------------------------------------------
constexpr uint64_t kStreamSigns = 0;
constexpr uint64_t kStreamBernoulli = 1;
constexpr uint64_t kStreamIid = 2;

struct u64x4 {
  uint64_t w[4];
};

__device__ __forceinline__ u64x4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t k0, uint64_t k1) {
  // multipliers and Weyl increments of the 4x64 variant (SC'11, Table 2)
  const uint64_t m0 = 0xD2E7470EE14C6C93ull, m1 = 0xCA5A826395121157ull;
  const uint64_t w0 = 0x9E3779B97F4A7C15ull, w1 = 0xBB67AE8584CAA73Bull;
  uint64_t x0 = c0, x1 = c1, x2 = 0, x3 = 0;
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint64_t h0 = __umul64hi(m0, x0), l0 = m0 * x0;
    const uint64_t h1 = __umul64hi(m1, x2), l1 = m1 * x2;
    const uint64_t y0 = h1 ^ x1 ^ k0;
    const uint64_t y2 = h0 ^ x3 ^ k1;
    x0 = y0;
    x1 = l1;
    x2 = y2;
    x3 = l0;
    k0 += w0;
    k1 += w1;
  }
  u64x4 r;
  r.w[0] = x0;
  r.w[1] = x1;
  r.w[2] = x2;
  r.w[3] = x3;
  return r;
}

// ---------------------------------------------------------------------------
// float-float: value = hi + lo with |lo| <= ulp(hi)/2.
// ---------------------------------------------------------------------------
struct ff {
  float hi, lo;
};

__device__ __forceinline__ ff ff_make(float a) { return ff{a, 0.0f}; }

// Knuth's TwoSum: s + e == a + b exactly.
__device__ __forceinline__ ff two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return ff{s, e};
}

__device__ __forceinline__ ff fast_two_sum(float a, float b) {  // needs |a| >= |b|
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return ff{s, e};
}

// Exact product: p + e == a * b (FMA gives the rounding error).
__device__ __forceinline__ ff two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  float e = __fmaf_rn(a, b, -p);
  return ff{p, e};
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
  ff s = two_sum(a.hi, b.hi);
  ff t = two_sum(a.lo, b.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = fast_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  ff p = two_prod(a.hi, b.hi);
  p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
  p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
  return fast_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
  ff p = two_prod(a.hi, b);
  p.lo = __fmaf_rn(a.lo, b, p.lo);
  return fast_two_sum(p.hi, p.lo);
}

// a / b by one Newton correction of the FP32 quotient.
__device__ __forceinline__ ff ff_div(ff a, ff b) {
  float q1 = __fdiv_rn(a.hi, b.hi);
  ff r = ff_sub(a, ff_mul_f(b, q1));
  float q2 = __fdiv_rn(r.hi, b.hi);
  return fast_two_sum(q1, q2);
}

// ordering on float-float values
__device__ __forceinline__ bool ff_gt(ff a, ff b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
__device__ __forceinline__ bool ff_lt(ff a, ff b) { return ff_gt(b, a); }
__device__ __forceinline__ bool ff_le0(ff a) { return a.hi < 0.0f || (a.hi == 0.0f && a.lo <= 0.0f); }
__device__ __forceinline__ bool ff_gt0(ff a) { return !ff_le0(a); }

__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ ff ff_from_double(double v) {
  float h = (float)v;
  float l = (float)(v - (double)h);
  return ff{h, l};
}

// Compensated dot-product accumulator (Ogita-Rump-Oishi Dot2): products
// exact, sums error-free, result about as accurate as with twice the
// working precision.
struct dot2 {
  float s, c;
  __device__ __forceinline__ dot2() : s(0.0f), c(0.0f) {}
  __device__ __forceinline__ void add_prod(float a, float b) {
    ff p = two_prod(a, b);
    ff t = two_sum(s, p.hi);
    s = t.hi;
    c = __fadd_rn(c, __fadd_rn(t.lo, p.lo));
  }
  __device__ __forceinline__ void add(float a) {
    ff t = two_sum(s, a);
    s = t.hi;
    c = __fadd_rn(c, t.lo);
  }
  __device__ __forceinline__ ff value() const { return fast_two_sum(s, c); }
};

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
__host__ __device__ inline int log2_ceil64(int64_t n) {
  int L = 0;
  while (((int64_t)1 << L) < n) ++L;
  return L;
}

__device__ __forceinline__ float flip_if(float v, uint32_t bit) {
  return __int_as_float(__float_as_int(v) ^ (bit << 31));
}

// Shared-memory word of position p (12 bits) of a 4096-float chunk loaded
// by a tensor copy with 128-byte swizzling into a 1024-byte aligned buffer:
// the 16-byte unit (bits 2-4) is XORed with the 128-byte row (bits 5-7).
__host__ __device__ __forceinline__ uint32_t swz128(uint32_t p) { return p ^ (((p >> 5) & 7u) << 2); }

}  // namespace rnnls

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
struct rnnls_ctx {
  int device;
  cudaStream_t stream;
  int num_sms;
  int sketch_sms;     // SMs the large-n sketch may occupy (0: all)
  rnnls_tuning tune;  // launch-shape choices (0 fields: defaults)
  int max_smem_optin;
  void *ws;          // device workspace
  size_t ws_bytes;
  void *pinned;      // pinned host staging buffer (counts, job tables)
  size_t pinned_bytes;
  cudaEvent_t pinned_ready;  // recorded after the last copy out of `pinned`
  void *aux;         // device: sampled rows when the caller passes none, counts
  size_t aux_bytes;
  unsigned int *counters;  // device: zero-initialised completion counters (reset by their users)
  size_t counters_len;
  void *boost;       // device: the sketches, solutions and partial sums of repeated runs
  size_t boost_bytes;
  cudaEvent_t plan_event;  // borrowed, nullable: recorded after each FP32 sketch's plan launch
  // launch profiling (rnnls_profile_begin / rnnls_profile_end)
  int prof_on;
  int prof_cap;
  int prof_n;
  int *prof_kid;
  cudaEvent_t *prof_ev;  // 2 * prof_cap events
};

namespace rnnls {
// Make sure the context workspace holds at least `bytes` (grows by cudaMalloc).
int ensure_workspace(rnnls_ctx *ctx, size_t bytes);
// Make sure the pinned staging buffer holds `bytes` and is free to overwrite.
int ensure_pinned(rnnls_ctx *ctx, size_t bytes);
// Make sure the auxiliary device buffer holds `bytes`.
int ensure_aux(rnnls_ctx *ctx, size_t bytes);
// At least `n` zeroed completion counters (kernels leave them at zero).
int ensure_counters(rnnls_ctx *ctx, size_t n, unsigned int **out);
inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
// a tuning field, or its default when 0
inline int tune_or(int v, int def) { return v > 0 ? v : def; }

// Kernels the profiler tells apart.
enum kernel_id {
  K_SAMPLE = 0,
  K_PLAN,
  K_SKETCH,
  K_SKETCH_SMALL,
  K_REDUCE,
  K_SKETCH_F64,
  K_GRAM,
  K_GRAM_REDUCE,
  K_COLABS,
  K_LH,
  K_RESIDUAL,
  K_BOOST_RES,
  K_BOOST_SEL,
  K_COLSTATS,
  K_GRAM_TC,
  K_PG,
  K_SKETCH_CSC,
  K_COUNT
};
const char *kernel_name(int kid);

// Records a CUDA event pair around the launches in its scope when the
// context's profiler is on (events on the context stream).
struct prof_scope {
  rnnls_ctx *c;
  int slot;
  cudaStream_t st;
  prof_scope(rnnls_ctx *ctx, int kid) : prof_scope(ctx, kid, ctx ? ctx->stream : nullptr) {}
  prof_scope(rnnls_ctx *ctx, int kid, cudaStream_t s) : c(ctx), slot(-1), st(s) {
    if (c && c->prof_on && c->prof_n < c->prof_cap) {
      slot = c->prof_n++;
      c->prof_kid[slot] = kid;
      cudaEventRecord(c->prof_ev[2 * slot], st);
    }
  }
  ~prof_scope() {
    if (slot >= 0) cudaEventRecord(c->prof_ev[2 * slot + 1], st);
  }
};

// Bump allocator over the workspace.
struct ws_carver {
  char *base;
  size_t off;
  explicit ws_carver(void *b) : base((char *)b), off(0) {}
  template <typename T>
  T *take(size_t count) {
    off = align_up(off, 256);
    T *p = (T *)(base + off);
    off += count * sizeof(T);
    return p;
  }
};
}  // namespace rnnls
