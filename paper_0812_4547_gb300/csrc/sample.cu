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
// Row i = h * 2^kLogM + l of H_n D X is sum_c (-1)^popcount(h & c) z_c[l],
// z_c the transformed chunk c.  A sketch block holds four transformed chunks
// c = 4j + w (w = 0..3) at a time; thread t adds, for each of its rows,
//   (-1)^popcount((h >> 2) & j) * sum_w (-1)^popcount((h & 3) & w) z_w[l].
// The loads z_w[l] are shared-memory gathers, so rows are placed to keep
// the 32 lanes of a warp on 32 different banks: the bank of row i is
// (word of l) mod 32, and the rows of bank q go to lane q of successive
// (warp, slot) pairs.  A bank with more than 8 * slots rows spills the rest
// into free positions of other lanes (one extra shared-memory wavefront
// each); empty positions read a word of their own bank and write nothing.
//
// Entry encoding: pk = 4 * (smem word of l) | ((h >> 2) << 14) | ((h & 1) << 31)
// | (((h >> 1) & 1) << 30), so bits 2-13 are the byte offset of l in a
// chunk, bit 31 the sign of chunk 4j + 1 and bit 30 that of chunk 4j + 2;
// k = row index in the sketch (-1: empty).  n <= 2^28 keeps h >> 2 below
// 2^14.
// ---------------------------------------------------------------------------
constexpr int kPlanThreads = 512;  // half an SM's registers: plans run beside other work

__global__ void __launch_bounds__(kPlanThreads, 2) build_plan_kernel(int32_t *__restrict__ idx, int64_t r,
                                                                  const int64_t *__restrict__ d_count,
                                                                  uint32_t *__restrict__ plan_pk,
                                                                  int32_t *__restrict__ plan_k, int slots,
                                                                  int64_t rows_per_group, int gen_iid, uint64_t seed,
                                                                  uint64_t inst, int L, uint64_t *__restrict__ sign_table,
                                                                  int64_t sign_words, int64_t sign_block0) {
  extern __shared__ uint16_t rank_of[];  // rows_per_group entries
  __shared__ uint32_t wcnt[kPlanThreads / 32][33];
  __shared__ uint32_t cnt[32], ov_start[32], free_start[32];
  const int g = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (g >= (int)gridDim.x - (int)((sign_words / 4 + kPlanThreads - 1) / kPlanThreads)) {
    // sign words of D: word W (counted from the table's first chunk) is word
    // W % 4 of Philox block sign_block0 + W / 4 of stream 0
    const int64_t first = (int64_t)(g - ((int)gridDim.x - (int)((sign_words / 4 + kPlanThreads - 1) / kPlanThreads)));
    const int64_t blk = first * kPlanThreads + tid;
    if (4 * blk < sign_words) {
      const u64x4 u = philox4x64_10((uint64_t)(sign_block0 + blk), kStreamSigns, seed, inst);
#pragma unroll
      for (int q = 0; q < 4; ++q) sign_table[4 * blk + q] = u.w[q];
    }
    return;
  }
  int64_t rr = r;
  if (d_count) rr = min(r, *d_count);
  const int64_t k0 = (int64_t)g * rows_per_group;
  const int64_t k1 = min(rr, k0 + rows_per_group);
  uint32_t *pk_out = plan_pk + (size_t)g * slots * kThreads;
  int32_t *k_out = plan_k + (size_t)g * slots * kThreads;
  const uint32_t cap = 8u * (uint32_t)slots;  // rows per bank without spilling

  for (int e = tid; e < slots * kThreads; e += kPlanThreads) {
    pk_out[e] = (uint32_t)(e & 31) << 2;
    k_out[e] = -1;
  }
  if (gen_iid) {
    // the iid rows of this group: draw k is word k of stream 2 (k0 is a multiple of 4)
    for (int64_t j = k0 / 4 + tid; 4 * j < k1; j += kPlanThreads) {
      const u64x4 u = philox4x64_10((uint64_t)j, kStreamIid, seed, inst);
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        const int64_t k = 4 * j + w;
        if (k < k1) idx[k] = (L == 0) ? 0 : (int32_t)(u.w[w] >> (64 - L));
      }
    }
  }
  __syncthreads();
  // 1. rank of each row within its bank, in row order (stable)
  uint32_t seen = 0;  // thread q < 32: rows of bank q in earlier tiles
  for (int64_t t0 = k0; t0 < k1; t0 += kPlanThreads) {
    const int64_t k = t0 + tid;
    const bool valid = k < k1;
    const uint32_t bank = valid ? (swz128((uint32_t)idx[k] & (kM - 1)) & 31u) : 32u;
    const uint32_t same = __match_any_sync(0xffffffffu, bank);
    const uint32_t below = __popc(same & ((1u << lane) - 1u));
    wcnt[warp][lane] = 0;
    __syncwarp();
    if (valid && below == 0) wcnt[warp][bank] = __popc(same);
    __syncthreads();
    if (tid < 32) {
      uint32_t run = seen;
      for (int q = 0; q < kPlanThreads / 32; ++q) {
        const uint32_t c = wcnt[q][tid];
        wcnt[q][tid] = run;
        run += c;
      }
      seen = run;
    }
    __syncthreads();
    if (valid) rank_of[k - k0] = (uint16_t)(wcnt[warp][bank] + below);
    __syncthreads();
  }
  if (tid < 32) cnt[tid] = seen;
  __syncthreads();
  if (tid == 0) {
    uint32_t ov = 0, fr = 0;
    for (int q = 0; q < 32; ++q) {
      ov_start[q] = ov;
      free_start[q] = fr;
      ov += cnt[q] > cap ? cnt[q] - cap : 0u;
      fr += cnt[q] < cap ? cap - cnt[q] : 0u;
    }
  }
  __syncthreads();
  // 2. place: rank t of bank q -> lane q of (warp t % 8, slot t / 8); spilled
  //    rows fill the free positions of the banks in bank order
  for (int64_t k = k0 + tid; k < k1; k += kPlanThreads) {
    const uint32_t i = (uint32_t)idx[k];
    const uint32_t l = i & (kM - 1), h = i >> kLogM;
    const uint32_t wd = swz128(l);
    const uint32_t bank = wd & 31u;
    const uint32_t rank = rank_of[k - k0];
    uint32_t q = bank, pos = rank;
    if (rank >= cap) {
      const uint32_t e = ov_start[bank] + (rank - cap);
      for (uint32_t b2 = 0; b2 < 32; ++b2) {
        const uint32_t f = cnt[b2] < cap ? cap - cnt[b2] : 0u;
        if (e >= free_start[b2] && e < free_start[b2] + f) {
          q = b2;
          pos = cnt[b2] + (e - free_start[b2]);
        }
      }
    }
    if (pos >= cap) continue;  // unreachable: the free positions outnumber the spilled rows
    const uint32_t thread = (pos & 7u) * 32u + q;
    const uint32_t slot = pos >> 3;
    pk_out[(size_t)slot * kThreads + thread] = (wd << 2) | ((h >> 2) << 14) | ((h & 1u) << 31) | (((h >> 1) & 1u) << 30);
    k_out[(size_t)slot * kThreads + thread] = (int32_t)k;
  }
}

size_t plan_ws_bytes(int slots, int kgroups) {
  const size_t e = (size_t)kgroups * slots * kThreads;
  return align_up(e * sizeof(uint32_t), 256) + align_up(e * sizeof(int32_t), 256);
}

int launch_build_plan(cudaStream_t s, int32_t *idx, int64_t r, const int64_t *d_count, plan_t plan,
                      const iid_gen *gen, uint64_t *sign_table, int64_t sign_words, int64_t sign_block0, uint64_t seed,
                      uint64_t inst) {
  if (plan.rows_per_group > kPlanMaxRows || plan.rows_per_group > (int64_t)plan.slots * kThreads)
    return RNNLS_EUNSUPPORTED;
  if (!sign_table) sign_words = 0;
  const int64_t sign_blocks = (sign_words / 4 + kPlanThreads - 1) / kPlanThreads;
  static bool attr_set = false;
  if (!attr_set) {
    if (cudaFuncSetAttribute(build_plan_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(kPlanMaxRows * sizeof(uint16_t))) != cudaSuccess)
      return RNNLS_ECUDA;
    attr_set = true;
  }
  const size_t smem = (size_t)plan.rows_per_group * sizeof(uint16_t);
  build_plan_kernel<<<(unsigned)(plan.kgroups + sign_blocks), kPlanThreads, smem, s>>>(
      idx, r, d_count, plan.pk, plan.k, plan.slots, plan.rows_per_group, gen ? 1 : 0, seed, inst, gen ? gen->L : 0,
      sign_table, sign_words, sign_block0);
  return cudaGetLastError() == cudaSuccess ? RNNLS_OK : RNNLS_ECUDA;
}

}  // namespace rnnls
