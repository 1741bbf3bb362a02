// sample.cu -- the random row selection S of Alg. 1 steps 2-3 and the
// combine plan used by the large-n sketch kernel.
//
// Row selection (Philox4x64-10, key = (seed, instance)):
//   iid       : draw k -> row (word k of stream 2) >> (64 - L)
//   Bernoulli : row i kept iff word i of stream 1 < r * 2^(64 - L), i.e. with
//               probability r/n (Alg. 1 step 2); all rows when r >= n.
#include <cub/block/block_reduce.cuh>
#include <cub/block/block_scan.cuh>

#include "kernels.h"

namespace rnnls {

// ---------------------------------------------------------------------------
// iid: one Philox block gives four draws.
// ---------------------------------------------------------------------------
__global__ void sample_iid_kernel(uint64_t seed, uint64_t inst, int L, int64_t r, int32_t *__restrict__ idx) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (4 * j >= r) return;
  const u64x4 u = philox4x64_10((uint64_t)j, kStreamIid, seed, inst);
#pragma unroll
  for (int w = 0; w < 4; ++w) {
    const int64_t k = 4 * j + w;
    if (k < r) idx[k] = (L == 0) ? 0 : (int32_t)(u.w[w] >> (64 - L));
  }
}

int launch_sample_iid(cudaStream_t s, uint64_t seed, uint64_t inst, int L, int64_t r, int32_t *idx) {
  const int64_t blocks_needed = (r + 3) / 4;
  const int threads = 256;
  const int64_t grid = (blocks_needed + threads - 1) / threads;
  sample_iid_kernel<<<(unsigned)grid, threads, 0, s>>>(seed, inst, L, r, idx);
  return cudaGetLastError() == cudaSuccess ? RNNLS_OK : RNNLS_ECUDA;
}

// ---------------------------------------------------------------------------
// Bernoulli: count per tile, scan tile counts, write kept rows in order.
// A tile is 4096 rows: 1024 threads x one Philox block (4 rows) each.
// ---------------------------------------------------------------------------
constexpr int kBernThreads = 1024;
constexpr int kBernTile = 4 * kBernThreads;

__device__ __forceinline__ uint32_t bernoulli_keep4(uint64_t seed, uint64_t inst, int L, int64_t r, int64_t j) {
  // bit w set iff row 4j + w is kept
  const int64_t n = (int64_t)1 << L;
  uint32_t bits = 0;
  if (r >= n) return 0xFu;
  const uint64_t thresh = (uint64_t)r << (64 - L);
  const u64x4 u = philox4x64_10((uint64_t)j, kStreamBernoulli, seed, inst);
#pragma unroll
  for (int w = 0; w < 4; ++w) bits |= (u.w[w] < thresh ? 1u : 0u) << w;
  return bits;
}

__global__ void __launch_bounds__(kBernThreads) bernoulli_count_kernel(uint64_t seed, uint64_t inst, int L,
                                                                       int64_t r, uint32_t *__restrict__ tile_count) {
  const int64_t n = (int64_t)1 << L;
  const int64_t j = (int64_t)blockIdx.x * kBernThreads + threadIdx.x;
  uint32_t c = 0;
  if (4 * j < n) {
    uint32_t bits = bernoulli_keep4(seed, inst, L, r, j);
    if (n < 4) bits &= (1u << n) - 1u;
    c = __popc(bits);
  }
  typedef cub::BlockReduce<uint32_t, kBernThreads> reduce_t;
  __shared__ typename reduce_t::TempStorage tmp;
  const uint32_t tot = reduce_t(tmp).Sum(c);
  if (threadIdx.x == 0) tile_count[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kBernThreads) bernoulli_scan_kernel(const uint32_t *__restrict__ tile_count,
                                                                      int64_t tiles, int64_t *__restrict__ tile_off,
                                                                      int64_t *__restrict__ d_count) {
  typedef cub::BlockScan<int64_t, kBernThreads> scan_t;
  __shared__ typename scan_t::TempStorage tmp;
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < tiles; base += kBernThreads) {
    const int64_t t = base + threadIdx.x;
    int64_t v = (t < tiles) ? (int64_t)tile_count[t] : 0;
    int64_t ex, agg;
    scan_t(tmp).ExclusiveSum(v, ex, agg);
    if (t < tiles) tile_off[t] = carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry += agg;
    __syncthreads();
  }
  if (threadIdx.x == 0) *d_count = carry;
}

__global__ void __launch_bounds__(kBernThreads) bernoulli_write_kernel(uint64_t seed, uint64_t inst, int L, int64_t r,
                                                                       const int64_t *__restrict__ tile_off,
                                                                       int32_t *__restrict__ idx, int64_t cap) {
  const int64_t n = (int64_t)1 << L;
  const int64_t j = (int64_t)blockIdx.x * kBernThreads + threadIdx.x;
  uint32_t bits = 0;
  if (4 * j < n) {
    bits = bernoulli_keep4(seed, inst, L, r, j);
    if (n < 4) bits &= (1u << n) - 1u;
  }
  typedef cub::BlockScan<uint32_t, kBernThreads> scan_t;
  __shared__ typename scan_t::TempStorage tmp;
  uint32_t ex;
  scan_t(tmp).ExclusiveSum((uint32_t)__popc(bits), ex);
  int64_t pos = tile_off[blockIdx.x] + ex;
#pragma unroll
  for (int w = 0; w < 4; ++w) {
    if (bits & (1u << w)) {
      if (pos < cap) idx[pos] = (int32_t)(4 * j + w);
      ++pos;
    }
  }
}

size_t bernoulli_ws_bytes(int64_t n) {
  const int64_t tiles = (n + kBernTile - 1) / kBernTile;
  return align_up((size_t)tiles * sizeof(uint32_t), 256) + align_up((size_t)tiles * sizeof(int64_t), 256);
}

int launch_sample_bernoulli(cudaStream_t s, uint64_t seed, uint64_t inst, int L, int64_t r, int32_t *idx,
                            int64_t cap, int64_t *d_count, void *ws) {
  const int64_t n = (int64_t)1 << L;
  const int64_t tiles = (n + kBernTile - 1) / kBernTile;
  ws_carver c(ws);
  uint32_t *tile_count = c.take<uint32_t>((size_t)tiles);
  int64_t *tile_off = c.take<int64_t>((size_t)tiles);
  bernoulli_count_kernel<<<(unsigned)tiles, kBernThreads, 0, s>>>(seed, inst, L, r, tile_count);
  bernoulli_scan_kernel<<<1, kBernThreads, 0, s>>>(tile_count, tiles, tile_off, d_count);
  bernoulli_write_kernel<<<(unsigned)tiles, kBernThreads, 0, s>>>(seed, inst, L, r, tile_off, idx, cap);
  return cudaGetLastError() == cudaSuccess ? RNNLS_OK : RNNLS_ECUDA;
}

// ---------------------------------------------------------------------------
// Combine plan of the large-n sketch.
//
// Row i = h * 2^kLogM + l is read from the transformed chunks at position l;
// chunk c contributes with sign (-1)^popcount(h & c).  A sketch block
// combines four chunks c0+0..c0+3 at a time, so the factor for those four is
// (-1)^popcount(h & c0) * (-1)^popcount((h & 3) & w): the second factor is
// the same for all rows with the same class h & 3.  Rows are therefore
// grouped by class; class k gets ceil(size_k / slots) threads, which always
// fits in kThreads when slots >= ceil(rows / (kThreads - 4)).  Within a class
// rows are sorted by l so that the 32 lanes of a warp read 32 nearby words
// of shared memory (few bank conflicts).
//
// Entry encoding: pk = (smem word of l) | ((h >> 2) << 12); k = row index in
// the sketch (-1 for an unused slot).
// ---------------------------------------------------------------------------
constexpr int kPlanThreads = 1024;
constexpr int kBins = 4 * kM;

__device__ __forceinline__ uint32_t smem_word(uint32_t p) {
  // swizzle used by the sketch kernel's shared-memory chunk buffers
  return p ^ (((p >> 8) & 7u) << 2);
}

__global__ void __launch_bounds__(kPlanThreads) build_plan_kernel(const int32_t *__restrict__ idx, int64_t r,
                                                                  const int64_t *__restrict__ d_count,
                                                                  uint32_t *__restrict__ plan_pk,
                                                                  int32_t *__restrict__ plan_k,
                                                                  uint32_t *__restrict__ plan_cls, int slots,
                                                                  int64_t rows_per_group) {
  extern __shared__ uint32_t hist[];  // kBins
  __shared__ uint32_t cls_size[4], cls_start[4], t_count[4], t_start[4];
  const int g = blockIdx.x;
  int64_t rr = r;
  if (d_count) rr = min(r, *d_count);
  const int64_t k0 = (int64_t)g * rows_per_group;
  const int64_t k1 = min(rr, k0 + rows_per_group);
  uint32_t *pk_out = plan_pk + (size_t)g * slots * kThreads;
  int32_t *k_out = plan_k + (size_t)g * slots * kThreads;

  for (int i = threadIdx.x; i < kBins; i += kPlanThreads) hist[i] = 0;
  for (int e = threadIdx.x; e < slots * kThreads; e += kPlanThreads) {
    pk_out[e] = 0;
    k_out[e] = -1;
  }
  if (threadIdx.x < 4) cls_size[threadIdx.x] = 0;
  __syncthreads();
  for (int64_t k = k0 + threadIdx.x; k < k1; k += kPlanThreads) {
    const uint32_t i = (uint32_t)idx[k];
    const uint32_t l = i & (kM - 1), h = i >> kLogM;
    atomicAdd(&hist[(h & 3u) * kM + l], 1u);
    atomicAdd(&cls_size[h & 3u], 1u);
  }
  __syncthreads();
  // exclusive scan of the histogram: each thread owns kBins/kPlanThreads bins
  {
    constexpr int per = kBins / kPlanThreads;
    uint32_t local[per];
    uint32_t sum = 0;
#pragma unroll
    for (int q = 0; q < per; ++q) {
      local[q] = hist[threadIdx.x * per + q];
      sum += local[q];
    }
    typedef cub::BlockScan<uint32_t, kPlanThreads> scan_t;
    __shared__ typename scan_t::TempStorage tmp;
    uint32_t ex;
    scan_t(tmp).ExclusiveSum(sum, ex);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < per; ++q) {
      hist[threadIdx.x * per + q] = ex;
      ex += local[q];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t ts = 0;
    for (int c = 0; c < 4; ++c) {
      cls_start[c] = hist[c * kM];
      const uint32_t tc = (cls_size[c] + (uint32_t)slots - 1u) / (uint32_t)slots;
      t_count[c] = tc;
      t_start[c] = ts;
      ts += tc;
    }
  }
  __syncthreads();
  if (threadIdx.x < kThreads) {
    uint32_t c = 0;
    for (uint32_t q = 0; q < 4; ++q)
      if (threadIdx.x >= t_start[q] && threadIdx.x < t_start[q] + t_count[q]) c = q;
    plan_cls[(size_t)g * kThreads + threadIdx.x] = c;
  }
  for (int64_t k = k0 + threadIdx.x; k < k1; k += kPlanThreads) {
    const uint32_t i = (uint32_t)idx[k];
    const uint32_t l = i & (kM - 1), h = i >> kLogM, c = h & 3u;
    const uint32_t pos = atomicAdd(&hist[c * kM + l], 1u);
    const uint32_t u = pos - cls_start[c];
    const uint32_t thread = t_start[c] + u % t_count[c];
    const uint32_t slot = u / t_count[c];
    pk_out[(size_t)slot * kThreads + thread] = smem_word(l) | ((h >> 2) << kLogM);
    k_out[(size_t)slot * kThreads + thread] = (int32_t)k;
  }
}

size_t plan_ws_bytes(int slots, int kgroups) {
  const size_t e = (size_t)kgroups * slots * kThreads;
  return align_up(e * sizeof(uint32_t), 256) + align_up(e * sizeof(int32_t), 256) +
         align_up((size_t)kgroups * kThreads * sizeof(uint32_t), 256);
}

int launch_build_plan(cudaStream_t s, const int32_t *idx, int64_t r, const int64_t *d_count, plan_t plan,
                      void *ws_sort) {
  (void)ws_sort;
  const size_t smem = kBins * sizeof(uint32_t);
  static bool attr_set = false;
  if (!attr_set) {
    if (cudaFuncSetAttribute(build_plan_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return RNNLS_ECUDA;
    attr_set = true;
  }
  build_plan_kernel<<<plan.kgroups, kPlanThreads, smem, s>>>(idx, r, d_count, plan.pk, plan.k, plan.cls,
                                                              plan.slots, plan.rows_per_group);
  return cudaGetLastError() == cudaSuccess ? RNNLS_OK : RNNLS_ECUDA;
}

}  // namespace rnnls
