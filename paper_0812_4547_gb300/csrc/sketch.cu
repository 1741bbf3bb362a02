// sketch.cu -- the preconditioning step of Alg. 1: SX = H~ D X for the tall
// X = [A | b], where H~ holds the sampled, rescaled rows of the normalised
// Walsh-Hadamard matrix H_n (Sec. 2, Alg. 1 steps 1-4, cost O(nd log r) per
// Sec. 3.4).
//
// Large n (n >= 2^14): H_n = H_C (x) H_m with m = 2^12 and C = n/m, row
// i = h*m + l.  Then (H_n y)[i] = sum_c (-1)^popcount(h & c) (H_m y_c)[l] for
// the chunks y_c of y.  One block owns a column and a range of 4*NI chunks:
//   - it reads each chunk once from HBM (coalesced 16-byte loads),
//   - flips signs with D (Philox bits regenerated in the block),
//   - transforms the chunk with two 64-point register FWHT passes joined by
//     one swizzled shared-memory transpose (four chunks at a time, one per
//     64-thread worker),
//   - and accumulates, for the sampled rows only, the signed chunk values
//     into per-row registers (the "combine"; the signs for the chunks of one
//     step factor into a per-thread part and a per-row part that is tracked
//     by visiting the steps in Gray-code order).
// Only r values per column leave the block, so HBM sees one read of X plus
// r*(d+1) partial sums per chunk range.
//
// Small n (n <= 2^13): one block per column transforms the whole column in
// shared memory and gathers the sampled rows.
#include <algorithm>
#include <cmath>

#include "kernels.h"

namespace rnnls {

namespace {

__device__ __forceinline__ uint32_t zword(uint32_t p) { return p ^ (((p >> 8) & 7u) << 2); }

__device__ __forceinline__ void bar_worker(int w) {
  asm volatile("bar.sync %0, 64;" ::"r"(w + 1) : "memory");
}

// In-register unnormalised Walsh-Hadamard transform of 64 values,
// v[i] <- sum_j (-1)^popcount(i & j) v[j].
__device__ __forceinline__ void fwht64(float (&v)[64]) {
#pragma unroll
  for (int h = 1; h < 64; h <<= 1) {
#pragma unroll
    for (int i = 0; i < 64; ++i) {
      if ((i & h) == 0) {
        const float a = v[i], b = v[i + h];
        v[i] = a + b;
        v[i + h] = a - b;
      }
    }
  }
}

__device__ __forceinline__ uint32_t gray(uint32_t i) { return i ^ (i >> 1); }

template <int SLOTS, bool VEC>
__global__ void __launch_bounds__(kThreads, 1)
    sketch_chunked_f32(const float *__restrict__ A, int64_t lda, const float *__restrict__ b, int64_t n_raw, int d,
                       int iters, uint64_t seed, uint64_t inst, const uint32_t *__restrict__ plan_pk,
                       const int32_t *__restrict__ plan_k, const uint32_t *__restrict__ plan_cls,
                       float *__restrict__ part, int64_t r_part, float scale, float *__restrict__ SA, int64_t ldsa,
                       float *__restrict__ Sb, int direct) {
  extern __shared__ __align__(16) float zbuf[];  // kWorkers x kM floats
  __shared__ uint64_t sgn[kWorkers][kM / 64];

  const int tid = threadIdx.x;
  const int w = tid >> 6;   // worker
  const int wt = tid & 63;  // thread within worker
  const int col = blockIdx.x;
  const int grp = blockIdx.y;
  const int kg = blockIdx.z;
  const float *__restrict__ x = (col < d) ? A + (int64_t)col * lda : b;
  const uint32_t c0 = (uint32_t)grp * 4u * (uint32_t)iters;

  // combine state: this thread's rows (plan) and their partial sums
  const size_t pbase = (size_t)kg * SLOTS * kThreads;
  uint32_t pk[SLOTS];
  float acc[SLOTS];
#pragma unroll
  for (int s = 0; s < SLOTS; ++s) {
    pk[s] = plan_pk[pbase + (size_t)s * kThreads + tid];
    acc[s] = 0.0f;
  }
  const uint32_t cls = plan_cls[(size_t)kg * kThreads + tid];
  const float s1 = (cls & 1u) ? -1.0f : 1.0f;
  const float s2 = (cls & 2u) ? -1.0f : 1.0f;
  const float s3 = s1 * s2;
  float *__restrict__ zw = zbuf + w * kM;

  for (int it = 0; it < iters; ++it) {
    const uint32_t cbase = c0 + 4u * gray((uint32_t)it);
    const uint32_t c = cbase + (uint32_t)w;
    const int64_t row0 = (int64_t)c * kM;

    // 1. load this worker's chunk: v[4q + e] <- x[row0 + 4*wt + 256*q + e]
    float v[64];
    if (row0 + kM <= n_raw) {
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int64_t row = row0 + 4 * wt + 256 * q;
        if (VEC) {
          const float4 t = __ldcs(reinterpret_cast<const float4 *>(x + row));
          v[4 * q + 0] = t.x;
          v[4 * q + 1] = t.y;
          v[4 * q + 2] = t.z;
          v[4 * q + 3] = t.w;
        } else {
#pragma unroll
          for (int e = 0; e < 4; ++e) v[4 * q + e] = __ldcs(x + row + e);
        }
      }
    } else {
#pragma unroll
      for (int q = 0; q < 16; ++q) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int64_t row = row0 + 4 * wt + 256 * q + e;
          v[4 * q + e] = (row < n_raw) ? __ldcs(x + row) : 0.0f;
        }
      }
    }

    // 2. the 64 sign words of this chunk: Philox block j = 16c + wt, stream 0
    if (wt < 16) {
      const u64x4 u = philox4x64_10((uint64_t)c * 16u + (uint64_t)wt, kStreamSigns, seed, inst);
#pragma unroll
      for (int q = 0; q < 4; ++q) sgn[w][4 * wt + q] = u.w[q];
    }
    __syncthreads();  // signs visible; previous combine done with zbuf

    // 3. D: row 4*wt + 256*q + e uses bit (4*wt + e) mod 64 of word wt/16 + 4q
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const uint64_t word = sgn[w][(wt >> 4) + 4 * q];
      const uint32_t nib = (uint32_t)(word >> ((4 * wt) & 63)) & 0xFu;
#pragma unroll
      for (int e = 0; e < 4; ++e) v[4 * q + e] = flip_if(v[4 * q + e], (nib >> e) & 1u);
    }

    // 4. pass 1: position bits {0,1,8,9,10,11} live in the register index
    fwht64(v);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const uint32_t p = 4u * wt + 256u * q;
      *reinterpret_cast<float4 *>(zw + zword(p)) = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    }
    bar_worker(w);
    // 5. pass 2: position bits {2..7}
    const uint32_t pfix = (wt & 3u) | ((uint32_t)(wt >> 2) << 8);
#pragma unroll
    for (int s = 0; s < 64; ++s) v[s] = zw[zword(pfix | ((uint32_t)s << 2))];
    fwht64(v);
    bar_worker(w);
#pragma unroll
    for (int s = 0; s < 64; ++s) zw[zword(pfix | ((uint32_t)s << 2))] = v[s];
    __syncthreads();  // the four transformed chunks are ready

    // 6. combine at the sampled rows
    const uint32_t beta = (it == 0) ? 0u : (uint32_t)(__ffs(it) - 1);
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) {
      const uint32_t p = pk[s];
      float a = acc[s];
      if (it > 0) a = flip_if(a, (p >> (kLogM + beta)) & 1u);
      const uint32_t wd = p & (kM - 1);
      float t = zbuf[wd];
      t = fmaf(s1, zbuf[kM + wd], t);
      t = fmaf(s2, zbuf[2 * kM + wd], t);
      t = fmaf(s3, zbuf[3 * kM + wd], t);
      acc[s] = a + t;
    }
  }

  // 7. undo the running sign: row factor (-1)^popcount(h & (c0 | 4 gray(iters-1)))
  const uint32_t cmask = c0 | (4u * gray((uint32_t)(iters - 1)));
#pragma unroll
  for (int s = 0; s < SLOTS; ++s) {
    const int32_t k = plan_k[pbase + (size_t)s * kThreads + tid];
    if (k < 0) continue;
    const uint32_t h = ((pk[s] >> kLogM) << 2) | cls;
    const float val = flip_if(acc[s], (uint32_t)__popc(h & cmask) & 1u);
    if (direct) {
      if (col < d)
        SA[(int64_t)col * ldsa + k] = scale * val;
      else
        Sb[k] = scale * val;
    } else {
      part[((int64_t)grp * (d + 1) + col) * r_part + k] = val;
    }
  }
}

// Sum the per-chunk-range partial sums and apply the row scale.
template <typename T>
__global__ void reduce_partials(const float *__restrict__ part, int groups, int d, int64_t r_part,
                                const int64_t *__restrict__ d_count, float scale, T *__restrict__ SA, int64_t ldsa,
                                T *__restrict__ Sb) {
  int64_t rr = r_part;
  if (d_count) rr = min(r_part, *d_count);
  const int col = blockIdx.y;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < rr; k += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int g = 0; g < groups; ++g) s += part[((int64_t)g * (d + 1) + col) * r_part + k];
    if (col < d)
      SA[(int64_t)col * ldsa + k] = scale * s;
    else
      Sb[k] = scale * s;
  }
}

// ---------------------------------------------------------------------------
// whole column in shared memory (n <= 2^13), FP32 or FP64
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) sketch_small(const T *__restrict__ A, int64_t lda, const T *__restrict__ b,
                                                    int64_t n_raw, int d, int L, uint64_t seed, uint64_t inst,
                                                    const int32_t *__restrict__ idx, int64_t r,
                                                    const int64_t *__restrict__ d_count, T scale, T *__restrict__ SA,
                                                    int64_t ldsa, T *__restrict__ Sb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = 1 << L;
  uint64_t *words = reinterpret_cast<uint64_t *>(smem_raw);  // max(n/64, 4) sign words
  T *buf = reinterpret_cast<T *>(words + (n / 64 > 4 ? n / 64 : 4));
  const int col = blockIdx.x;
  const T *__restrict__ x = (col < d) ? A + (int64_t)col * lda : b;
  const int calls = (n + 255) / 256;
  for (int j = threadIdx.x; j < calls; j += blockDim.x) {
    const u64x4 u = philox4x64_10((uint64_t)j, kStreamSigns, seed, inst);
#pragma unroll
    for (int q = 0; q < 4; ++q) words[4 * j + q] = u.w[q];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const T v = (i < n_raw) ? x[i] : T(0);
    const bool neg = (words[i >> 6] >> (i & 63)) & 1ull;
    buf[i] = neg ? -v : v;
  }
  __syncthreads();
  for (int h = 1; h < n; h <<= 1) {
    for (int t = threadIdx.x; t < n / 2; t += blockDim.x) {
      const int i = ((t & ~(h - 1)) << 1) | (t & (h - 1));
      const T a = buf[i], c = buf[i + h];
      buf[i] = a + c;
      buf[i + h] = a - c;
    }
    __syncthreads();
  }
  int64_t rr = r;
  if (d_count) rr = min(r, *d_count);
  T *out = (col < d) ? SA + (int64_t)col * ldsa : Sb;
  for (int64_t k = threadIdx.x; k < rr; k += blockDim.x) out[k] = scale * buf[idx[k]];
}

// ---------------------------------------------------------------------------
// FP64, n > 2^13: transform every chunk of 2^12 rows into a workspace, then
// combine at the sampled rows.  (Correctness path; FP64 is slow on GB300.)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) chunk_transform_f64(const double *__restrict__ A, int64_t lda,
                                                           const double *__restrict__ b, int64_t n_raw, int d,
                                                           int64_t n, uint64_t seed, uint64_t inst,
                                                           double *__restrict__ Z) {
  __shared__ double buf[kM];
  __shared__ uint64_t words[kM / 64];
  const int col = blockIdx.x;
  const int64_t c = blockIdx.y;
  const double *__restrict__ x = (col < d) ? A + (int64_t)col * lda : b;
  if (threadIdx.x < kM / 256) {
    const u64x4 u = philox4x64_10((uint64_t)c * (kM / 256) + threadIdx.x, kStreamSigns, seed, inst);
#pragma unroll
    for (int q = 0; q < 4; ++q) words[4 * threadIdx.x + q] = u.w[q];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kM; i += blockDim.x) {
    const int64_t row = c * kM + i;
    const double v = (row < n_raw) ? x[row] : 0.0;
    buf[i] = ((words[i >> 6] >> (i & 63)) & 1ull) ? -v : v;
  }
  __syncthreads();
  for (int h = 1; h < kM; h <<= 1) {
    for (int t = threadIdx.x; t < kM / 2; t += blockDim.x) {
      const int i = ((t & ~(h - 1)) << 1) | (t & (h - 1));
      const double a = buf[i], e = buf[i + h];
      buf[i] = a + e;
      buf[i + h] = a - e;
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < kM; i += blockDim.x) Z[(int64_t)col * n + c * kM + i] = buf[i];
}

__global__ void combine_f64(const double *__restrict__ Z, int d, int64_t n, const int32_t *__restrict__ idx,
                            int64_t r, const int64_t *__restrict__ d_count, double scale, double *__restrict__ SA,
                            int64_t ldsa, double *__restrict__ Sb) {
  int64_t rr = r;
  if (d_count) rr = min(r, *d_count);
  const int col = blockIdx.y;
  const int64_t C = n / kM;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < rr; k += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t i = (uint32_t)idx[k];
    const uint32_t h = i >> kLogM, l = i & (kM - 1);
    double s = 0.0;
    for (int64_t c = 0; c < C; ++c) {
      const double v = Z[(int64_t)col * n + c * kM + l];
      s += (__popc(h & (uint32_t)c) & 1) ? -v : v;
    }
    if (col < d)
      SA[(int64_t)col * ldsa + k] = scale * s;
    else
      Sb[k] = scale * s;
  }
}

template <int SLOTS, bool VEC>
int launch_chunked(rnnls_ctx *ctx, const sketch_args_f32 &a, const plan_t &plan, int groups, int iters,
                   float *part, int64_t r_part, int direct) {
  auto kern = sketch_chunked_f32<SLOTS, VEC>;
  const size_t smem = (size_t)kWorkers * kM * sizeof(float);
  static bool attr = false;
  if (!attr) {
    RNNLS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  dim3 grid((unsigned)(a.d + 1), (unsigned)groups, (unsigned)plan.kgroups);
  kern<<<grid, kThreads, smem, ctx->stream>>>(a.A, a.lda, a.b, a.n_raw, a.d, iters, a.seed, a.inst, plan.pk, plan.k,
                                               plan.cls, part, r_part, a.scale, a.SA, a.ldsa, a.Sb, direct);
  return cudaGetLastError() == cudaSuccess ? RNNLS_OK : RNNLS_ECUDA;
}

template <int SLOTS>
int launch_chunked_v(rnnls_ctx *ctx, const sketch_args_f32 &a, const plan_t &plan, int groups, int iters,
                     float *part, int64_t r_part, int direct, bool vec) {
  return vec ? launch_chunked<SLOTS, true>(ctx, a, plan, groups, iters, part, r_part, direct)
             : launch_chunked<SLOTS, false>(ctx, a, plan, groups, iters, part, r_part, direct);
}

int pick_slots(int64_t rows) {
  const int64_t need = (rows + kPlanCapacityDen - 1) / kPlanCapacityDen;
  static const int opts[] = {1, 2, 4, 8, 16, 24, 32, 40};
  for (int s : opts)
    if (need <= s) return s;
  return 40;
}

template <int SLOTS>
int occupancy_of(bool vec) {
  int nb = 0;
  const size_t smem = (size_t)kWorkers * kM * sizeof(float);
  if (vec)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sketch_chunked_f32<SLOTS, true>, kThreads, smem);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sketch_chunked_f32<SLOTS, false>, kThreads, smem);
  return std::max(nb, 1);
}

int occupancy_for(int slots, bool vec) {
  switch (slots) {
    case 1: return occupancy_of<1>(vec);
    case 2: return occupancy_of<2>(vec);
    case 4: return occupancy_of<4>(vec);
    case 8: return occupancy_of<8>(vec);
    case 16: return occupancy_of<16>(vec);
    case 24: return occupancy_of<24>(vec);
    case 32: return occupancy_of<32>(vec);
    default: return occupancy_of<40>(vec);
  }
}

}  // namespace

int sketch_f32(rnnls_ctx *ctx, const sketch_args_f32 &a, int num_sms) {
  const int64_t n = (int64_t)1 << a.L;
  cudaStream_t s = ctx->stream;
  if (n <= 8192) {
    const size_t smem = (size_t)n * sizeof(float) + (size_t)std::max<int64_t>(n / 64, 4) * sizeof(uint64_t);
    prof_scope ps(ctx, K_SKETCH_SMALL);
    sketch_small<float><<<(unsigned)(a.d + 1), 256, smem, s>>>(a.A, a.lda, a.b, a.n_raw, a.d, a.L, a.seed, a.inst,
                                                               a.idx, a.r, a.d_count, a.scale, a.SA, a.ldsa, a.Sb);
    return cudaGetLastError() == cudaSuccess ? RNNLS_OK : RNNLS_ECUDA;
  }
  const int64_t C = n / kM;  // >= 4
  const int slots = pick_slots(a.r);
  const int64_t rows_per_group = (int64_t)kPlanCapacityDen * slots;
  const int kgroups = (int)((a.r + rows_per_group - 1) / rows_per_group);
  const bool vec = ((uintptr_t)a.A % 16 == 0) && (a.lda % 4 == 0) && ((uintptr_t)a.b % 16 == 0);

  // chunk groups: powers of two dividing C/4; pick the one that fills the
  // resident block slots best (fewest partial waves), preferring fewer groups
  const int per_sm = occupancy_for(slots, vec);
  const int64_t slots_total = (int64_t)num_sms * per_sm;
  int groups = 1;
  double best = -1.0;
  for (int64_t g = 1; g <= C / 4; g <<= 1) {
    const int64_t units = (int64_t)(a.d + 1) * g * kgroups;
    const int64_t waves = (units + slots_total - 1) / slots_total;
    const double eff = (double)units / (double)(waves * slots_total);
    const double score = eff - 0.02 * std::log2((double)g);
    if (score > best + 1e-9) {
      best = score;
      groups = (int)g;
    }
    if (units >= 8 * slots_total) break;
  }
  const int iters = (int)(C / 4 / groups);
  const int direct = (groups == 1) ? 1 : 0;

  // workspace: plan + partial sums
  const size_t plan_bytes = plan_ws_bytes(slots, kgroups);
  const size_t part_bytes = direct ? 0 : align_up((size_t)groups * (a.d + 1) * a.r * sizeof(float), 256);
  int st = ensure_workspace(ctx, plan_bytes + part_bytes + 256);
  if (st) return st;
  ws_carver wc(ctx->ws);
  plan_t plan;
  plan.pk = wc.take<uint32_t>((size_t)kgroups * slots * kThreads);
  plan.k = wc.take<int32_t>((size_t)kgroups * slots * kThreads);
  plan.cls = wc.take<uint32_t>((size_t)kgroups * kThreads);
  plan.slots = slots;
  plan.kgroups = kgroups;
  plan.rows_per_group = rows_per_group;
  float *part = direct ? nullptr : wc.take<float>((size_t)groups * (a.d + 1) * a.r);

  {
    prof_scope ps(ctx, K_PLAN);
    st = launch_build_plan(s, a.idx, a.r, a.d_count, plan, nullptr);
  }
  if (st) return st;
  {
    prof_scope ps_main(ctx, K_SKETCH);
    switch (slots) {
    case 1: st = launch_chunked_v<1>(ctx, a, plan, groups, iters, part, a.r, direct, vec); break;
    case 2: st = launch_chunked_v<2>(ctx, a, plan, groups, iters, part, a.r, direct, vec); break;
    case 4: st = launch_chunked_v<4>(ctx, a, plan, groups, iters, part, a.r, direct, vec); break;
    case 8: st = launch_chunked_v<8>(ctx, a, plan, groups, iters, part, a.r, direct, vec); break;
    case 16: st = launch_chunked_v<16>(ctx, a, plan, groups, iters, part, a.r, direct, vec); break;
    case 24: st = launch_chunked_v<24>(ctx, a, plan, groups, iters, part, a.r, direct, vec); break;
    case 32: st = launch_chunked_v<32>(ctx, a, plan, groups, iters, part, a.r, direct, vec); break;
    default: st = launch_chunked_v<40>(ctx, a, plan, groups, iters, part, a.r, direct, vec); break;
    }
  }
  if (st) return st;
  if (!direct) {
    prof_scope ps(ctx, K_REDUCE);
    dim3 grid((unsigned)std::min<int64_t>((a.r + 255) / 256, 64), (unsigned)(a.d + 1));
    reduce_partials<float><<<grid, 256, 0, s>>>(part, groups, a.d, a.r, a.d_count, a.scale, a.SA, a.ldsa, a.Sb);
    if (cudaGetLastError() != cudaSuccess) return RNNLS_ECUDA;
  }
  return RNNLS_OK;
}

// Same launches as sketch_f32, but every scratch buffer comes from the
// caller-provided region `scratch` (bytes long) and nothing is allocated.
// Chunk groups are capped so that the partial sums fit in that region.
template <int SLOTS, bool VEC>
int launch_chunked_stream(cudaStream_t s, const sketch_args_f32 &a, const plan_t &plan, int groups, int iters,
                          float *part, int64_t r_part, int direct) {
  auto kern = sketch_chunked_f32<SLOTS, VEC>;
  const size_t smem = (size_t)kWorkers * kM * sizeof(float);
  RNNLS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid((unsigned)(a.d + 1), (unsigned)groups, (unsigned)plan.kgroups);
  kern<<<grid, kThreads, smem, s>>>(a.A, a.lda, a.b, a.n_raw, a.d, iters, a.seed, a.inst, plan.pk, plan.k, plan.cls,
                                     part, r_part, a.scale, a.SA, a.ldsa, a.Sb, direct);
  return cudaGetLastError() == cudaSuccess ? RNNLS_OK : RNNLS_ECUDA;
}

template <int SLOTS>
int launch_chunked_stream_v(cudaStream_t s, const sketch_args_f32 &a, const plan_t &plan, int groups, int iters,
                            float *part, int64_t r_part, int direct, bool vec) {
  return vec ? launch_chunked_stream<SLOTS, true>(s, a, plan, groups, iters, part, r_part, direct)
             : launch_chunked_stream<SLOTS, false>(s, a, plan, groups, iters, part, r_part, direct);
}

int sketch_f32_scratch(cudaStream_t s, const sketch_args_f32 &a, int num_sms, void *scratch, size_t bytes) {
  const int64_t n = (int64_t)1 << a.L;
  if (n <= 8192) {
    const size_t smem = (size_t)n * sizeof(float) + (size_t)std::max<int64_t>(n / 64, 4) * sizeof(uint64_t);
    sketch_small<float><<<(unsigned)(a.d + 1), 256, smem, s>>>(a.A, a.lda, a.b, a.n_raw, a.d, a.L, a.seed, a.inst,
                                                               a.idx, a.r, a.d_count, a.scale, a.SA, a.ldsa, a.Sb);
    return cudaGetLastError() == cudaSuccess ? RNNLS_OK : RNNLS_ECUDA;
  }
  const int64_t C = n / kM;
  const int slots = pick_slots(a.r);
  const int64_t rows_per_group = (int64_t)kPlanCapacityDen * slots;
  const int kgroups = (int)((a.r + rows_per_group - 1) / rows_per_group);
  const bool vec = ((uintptr_t)a.A % 16 == 0) && (a.lda % 4 == 0) && ((uintptr_t)a.b % 16 == 0);
  const size_t plan_bytes = plan_ws_bytes(slots, kgroups);
  if (plan_bytes + 256 > bytes) return RNNLS_EUNSUPPORTED;
  const size_t part_one = align_up((size_t)(a.d + 1) * a.r * sizeof(float), 256);
  const int64_t fit = (int64_t)((bytes - plan_bytes - 256) / part_one);
  const int per_sm = occupancy_for(slots, vec);
  const int64_t slots_total = (int64_t)num_sms * per_sm;
  int groups = 1;
  double best = -1.0;
  for (int64_t g = 1; g <= C / 4; g <<= 1) {
    if (g > 1 && g > fit) break;
    const int64_t units = (int64_t)(a.d + 1) * g * kgroups;
    const int64_t waves = (units + slots_total - 1) / slots_total;
    const double eff = (double)units / (double)(waves * slots_total);
    const double score = eff - 0.02 * std::log2((double)g);
    if (score > best + 1e-9) {
      best = score;
      groups = (int)g;
    }
    if (units >= 8 * slots_total) break;
  }
  const int iters = (int)(C / 4 / groups);
  const int direct = (groups == 1) ? 1 : 0;
  ws_carver wc(scratch);
  plan_t plan;
  plan.pk = wc.take<uint32_t>((size_t)kgroups * slots * kThreads);
  plan.k = wc.take<int32_t>((size_t)kgroups * slots * kThreads);
  plan.cls = wc.take<uint32_t>((size_t)kgroups * kThreads);
  plan.slots = slots;
  plan.kgroups = kgroups;
  plan.rows_per_group = rows_per_group;
  float *part = direct ? nullptr : wc.take<float>((size_t)groups * (a.d + 1) * a.r);
  int st = launch_build_plan(s, a.idx, a.r, a.d_count, plan, nullptr);
  if (st) return st;
  switch (slots) {
    case 1: st = launch_chunked_stream_v<1>(s, a, plan, groups, iters, part, a.r, direct, vec); break;
    case 2: st = launch_chunked_stream_v<2>(s, a, plan, groups, iters, part, a.r, direct, vec); break;
    case 4: st = launch_chunked_stream_v<4>(s, a, plan, groups, iters, part, a.r, direct, vec); break;
    case 8: st = launch_chunked_stream_v<8>(s, a, plan, groups, iters, part, a.r, direct, vec); break;
    case 16: st = launch_chunked_stream_v<16>(s, a, plan, groups, iters, part, a.r, direct, vec); break;
    case 24: st = launch_chunked_stream_v<24>(s, a, plan, groups, iters, part, a.r, direct, vec); break;
    case 32: st = launch_chunked_stream_v<32>(s, a, plan, groups, iters, part, a.r, direct, vec); break;
    default: st = launch_chunked_stream_v<40>(s, a, plan, groups, iters, part, a.r, direct, vec); break;
  }
  if (st) return st;
  if (!direct) {
    dim3 grid((unsigned)std::min<int64_t>((a.r + 255) / 256, 64), (unsigned)(a.d + 1));
    reduce_partials<float><<<grid, 256, 0, s>>>(part, groups, a.d, a.r, a.d_count, a.scale, a.SA, a.ldsa, a.Sb);
    if (cudaGetLastError() != cudaSuccess) return RNNLS_ECUDA;
  }
  return RNNLS_OK;
}

int sketch_f64(rnnls_ctx *ctx, const sketch_args_f64 &a) {
  const int64_t n = (int64_t)1 << a.L;
  cudaStream_t s = ctx->stream;
  prof_scope ps(ctx, K_SKETCH_F64);
  if (n <= 8192) {
    const size_t smem = (size_t)n * sizeof(double) + (size_t)std::max<int64_t>(n / 64, 4) * sizeof(uint64_t);
    static bool attr = false;
    if (!attr) {
      RNNLS_CUDA_TRY(cudaFuncSetAttribute(sketch_small<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)(8192 * sizeof(double) + 128 * sizeof(uint64_t))));
      attr = true;
    }
    sketch_small<double><<<(unsigned)(a.d + 1), 256, smem, s>>>(a.A, a.lda, a.b, a.n_raw, a.d, a.L, a.seed, a.inst,
                                                                a.idx, a.r, a.d_count, a.scale, a.SA, a.ldsa, a.Sb);
    return cudaGetLastError() == cudaSuccess ? RNNLS_OK : RNNLS_ECUDA;
  }
  const size_t zbytes = align_up((size_t)(a.d + 1) * n * sizeof(double), 256);
  int st = ensure_workspace(ctx, zbytes);
  if (st) return st;
  double *Z = (double *)ctx->ws;
  chunk_transform_f64<<<dim3((unsigned)(a.d + 1), (unsigned)(n / kM)), 256, 0, s>>>(a.A, a.lda, a.b, a.n_raw, a.d, n,
                                                                                   a.seed, a.inst, Z);
  dim3 grid((unsigned)std::min<int64_t>((a.r + 255) / 256, 64), (unsigned)(a.d + 1));
  combine_f64<<<grid, 256, 0, s>>>(Z, a.d, n, a.idx, a.r, a.d_count, a.scale, a.SA, a.ldsa, a.Sb);
  return cudaGetLastError() == cudaSuccess ? RNNLS_OK : RNNLS_ECUDA;
}

}  // namespace rnnls
