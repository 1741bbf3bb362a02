// sample.cu -- the random row selection S of Alg. 1 steps 2-3 and the
// combine plan used by the large-n sketch kernel.
//
// Row selection (Philox4x64-10, key = (seed, instance)):
//   iid       : draw k -> row (word k of stream 2) >> (64 - L)
//   Bernoulli : row i kept iff word i of stream 1 < r * 2^(64 - L), i.e. with
//               probability r/n (Alg. 1 step 2); all rows when r >= n.

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

// Block-wide sum and exclusive prefix sum over kBernThreads threads: warp
// shuffles, then one pass over the per-warp totals in shared memory.
constexpr int kBernWarps = kBernThreads / 32;
template <typename T>
__device__ __forceinline__ T warp_inclusive_sum(T v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}
// Exclusive prefix of v over the block (thread order); *total gets the sum.
template <typename T>
__device__ __forceinline__ T block_exclusive_sum(T v, T *total) {
  __shared__ T warp_tot[kBernWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const T inc = warp_inclusive_sum(v);
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const T t = (lane < kBernWarps) ? warp_tot[lane] : (T)0;
    const T ti = warp_inclusive_sum(t);
    if (lane < kBernWarps) warp_tot[lane] = ti - t;  // exclusive prefix of the warp totals
    if (lane == kBernWarps - 1) *total = ti;
  }
  __syncthreads();
  const T out = warp_tot[warp] + inc - v;
  __syncthreads();  // warp_tot reusable by the caller's next call
  return out;
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
  __shared__ uint32_t tot;
  block_exclusive_sum<uint32_t>(c, &tot);
  if (threadIdx.x == 0) tile_count[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kBernThreads) bernoulli_scan_kernel(const uint32_t *__restrict__ tile_count,
                                                                      int64_t tiles, int64_t *__restrict__ tile_off,
                                                                      int64_t *__restrict__ d_count) {
  __shared__ int64_t carry, agg;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < tiles; base += kBernThreads) {
    const int64_t t = base + threadIdx.x;
    const int64_t v = (t < tiles) ? (int64_t)tile_count[t] : 0;
    const int64_t ex = block_exclusive_sum<int64_t>(v, &agg);
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
  __shared__ uint32_t tot;
  const uint32_t ex = block_exclusive_sum<uint32_t>((uint32_t)__popc(bits), &tot);
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
// Entry encoding: pk = 4 * (smem word of l) | ((h & 3) << 14) | ((h >> 2) << 16)
// | ((h & 1) << 31) | (((h >> 1) & 1) << 30), so bits 2-13 are the byte
// offset of l in a chunk, bits 2-15 its byte offset in the step's chunk
// (h & 3) (used once the step's four chunks have been transformed into one
// another), bit 31 the sign of chunk 4j + 1 and bit 30 that of chunk 4j + 2;
// k = row index in the sketch (-1: empty).  n <= 2^28 keeps h >> 2 below
// 2^14.
// ---------------------------------------------------------------------------
constexpr int kPlanThreads = 1024;

__device__ __forceinline__ uint32_t warp_inclusive_sum(uint32_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// One block per plan group g, plus the sign-table blocks.  The block ranks
// the group's rows within their banks in one pass: 1024 rows at a time (one
// per thread), a row's rank is the count of its bank's rows in earlier
// sub-passes, in earlier warps of this one (a per-warp bank histogram,
// scanned over the warps) and in earlier lanes of its warp (__match_any_sync).  Rows
// with rank below 8 * slots go to lane q of successive (warp, slot) pairs;
// the others (a bank's overflow) are kept per bank in shared memory and,
// once every bank's count is known, take the free positions of the other
// lanes in bank order; free positions left over become empty entries.  If
// a bank overflows by more than the kept number, a second pass places the
// rest.  Which position a row takes does not change any sum (each row adds
// its steps in step order wherever it sits); only the shared-memory banks
// its gathers hit.
// gen_L > 0: the block draws the iid rows itself (draw k = word k % 4 of
// Philox block k / 4 of stream 2, shifted right by 64 - gen_L, as
// sample_iid_kernel does) and writes them to idx; gen_L = 0: rows read from idx.
constexpr int kPlanWarps = kPlanThreads / 32;
constexpr uint32_t kSpillPerBank = 96;  // overflow rows kept per bank

__device__ __forceinline__ void plan_block(int blk, int32_t *__restrict__ idx, int64_t r,
                                           const int64_t *__restrict__ d_count, uint32_t *__restrict__ plan_pk,
                                           int32_t *__restrict__ plan_k, int slots, int64_t rows_per_group,
                                           int kgroups, uint64_t seed, uint64_t inst,
                                           uint64_t *__restrict__ sign_table, int64_t sign_words,
                                           int64_t sign_block0, int gen_L) {
  __shared__ uint32_t wcnt[2][kPlanWarps][33];  // per sub-pass (alternating): rows of bank b in warp w
  __shared__ uint32_t base[32];              // rows of bank b in earlier passes
  __shared__ uint32_t cnt[32], ov_start[32], free_start[32];
  __shared__ uint32_t total_ov, redo;
  __shared__ uint32_t spill_row[32][kSpillPerBank];
  __shared__ int32_t spill_k[32][kSpillPerBank];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (blk >= kgroups) {
    // sign words of D: word W (counted from the table's first chunk) is word
    // W % 4 of Philox block sign_block0 + W / 4 of stream 0
    const int64_t pb = (int64_t)(blk - kgroups) * kPlanThreads + tid;
    if (4 * pb < sign_words) {
      const u64x4 u = philox4x64_10((uint64_t)(sign_block0 + pb), kStreamSigns, seed, inst);
#pragma unroll
      for (int e = 0; e < 4; ++e) sign_table[4 * pb + e] = u.w[e];
    }
    return;
  }
  const int g = blk;
  int64_t rr = r;
  if (d_count) rr = min(r, *d_count);
  const int64_t k0 = (int64_t)g * rows_per_group;
  const int64_t k1 = min(rr, k0 + rows_per_group);
  uint32_t *pk_out = plan_pk + (size_t)g * slots * kThreads;
  int32_t *k_out = plan_k + (size_t)g * slots * kThreads;
  const uint32_t cap = 8u * (uint32_t)slots;  // rows per bank without spilling
  const uint32_t lt = (1u << lane) - 1u;
  if (tid < 32) base[tid] = 0;
  uint32_t sub = 0;  // sub-passes done (selects the count table)

  auto entry = [&](uint32_t pos, uint32_t ln) { return (size_t)(pos >> 3) * kThreads + (pos & 7u) * 32u + ln; };
  auto encode = [&](uint32_t row) {
    const uint32_t l = row & (kM - 1), h = row >> kLogM;
    return (swz128(l) << 2) | ((h & 3u) << 14) | ((h >> 2) << 16) | ((h & 1u) << 31) | (((h >> 1) & 1u) << 30);
  };
  // One pass over the group's rows, 4096 at a time (draws t0 + 4 tid + e, one
  // Philox block per thread), ranked in sub-passes e = 0..3 of 1024 rows each:
  // a row's rank within its bank counts the bank's rows of earlier sub-passes,
  // of earlier warps of its sub-pass and of earlier lanes of its warp.
  // place = 0: place ranks below cap and keep the overflow; place = 1 (the
  // rare second pass): place only overflow rows the first pass could not keep.
  auto pass = [&](int place) {
    for (int64_t t0 = k0; t0 < k1; t0 += 4 * kPlanThreads) {
      const int64_t kb = t0 + 4 * tid;
      uint32_t rows[4];
      if (gen_L > 0) {
        // kb is a multiple of 4: one Philox block gives draws kb .. kb + 3
        const u64x4 u = philox4x64_10((uint64_t)(kb >> 2), kStreamIid, seed, inst);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          rows[e] = (uint32_t)(u.w[e] >> (64 - gen_L));
          if (place == 0 && kb + e < k1) idx[kb + e] = (int32_t)rows[e];
        }
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) rows[e] = (kb + e < k1) ? (uint32_t)idx[kb + e] : 0u;
      }
#pragma unroll 1
      for (int e = 0; e < 4; ++e) {
        const int64_t k = kb + e;
        const bool valid = k < k1;
        const uint32_t row = rows[e];
        const uint32_t bank = valid ? (swz128(row & (kM - 1)) & 31u) : 32u;
        const uint32_t peers = __match_any_sync(0xffffffffu, bank);
        // lane b counts the warp's rows of bank b from five bit-slice ballots
        uint32_t same = __ballot_sync(0xffffffffu, valid);
#pragma unroll
        for (int j = 0; j < 5; ++j) {
          const uint32_t bj = __ballot_sync(0xffffffffu, (bank >> j) & 1u);
          same &= ((lane >> j) & 1) ? bj : ~bj;
        }
        // two tables in turn: the one written here was last read two sub-passes ago
        uint32_t(&wc)[kPlanWarps][33] = wcnt[sub & 1];
        ++sub;
        wc[warp][lane] = __popc(same);
        __syncthreads();
        // warp b scans bank b's counts over the warps
        {
          const uint32_t v = (lane < kPlanWarps) ? wc[lane][warp] : 0u;
          const uint32_t vi = warp_inclusive_sum(v);
          if (lane < kPlanWarps) wc[lane][warp] = base[warp] + vi - v;  // exclusive, earlier sub-passes included
          __syncwarp();
          if (lane == 31) base[warp] += vi;
        }
        __syncthreads();
        if (valid) {
          const uint32_t rank = wc[warp][bank] + __popc(peers & lt);
          if (rank < cap) {
            if (place == 0) {
              const size_t en = entry(rank, bank);
              pk_out[en] = encode(row);
              k_out[en] = (int32_t)k;
            }
          } else {
            const uint32_t o = rank - cap;
            if (place == 0) {
              if (o < kSpillPerBank) {
                spill_row[bank][o] = row;
                spill_k[bank][o] = (int32_t)k;
              }
            } else if (o >= kSpillPerBank) {
              // the e-th overflow row overall takes the e-th free position (bank order)
              const uint32_t ev = ov_start[bank] + o;
              for (uint32_t b2 = 0; b2 < 32; ++b2) {
                const uint32_t f = cnt[b2] < cap ? cap - cnt[b2] : 0u;
                if (ev >= free_start[b2] && ev < free_start[b2] + f) {
                  const size_t en = entry(cnt[b2] + (ev - free_start[b2]), b2);
                  pk_out[en] = encode(row);
                  k_out[en] = (int32_t)k;
                }
              }
            }
          }
        }
      }
    }
    __syncthreads();  // the last sub-pass's ranks are read
  };
  pass(0);
  if (tid < 32) cnt[tid] = base[tid];
  __syncthreads();
  if (tid == 0) {
    uint32_t ov = 0, fr = 0, big = 0;
    for (int b2 = 0; b2 < 32; ++b2) {
      ov_start[b2] = ov;
      free_start[b2] = fr;
      ov += cnt[b2] > cap ? cnt[b2] - cap : 0u;
      fr += cnt[b2] < cap ? cap - cnt[b2] : 0u;
      big |= (cnt[b2] > cap + kSpillPerBank) ? 1u : 0u;
    }
    total_ov = ov;
    redo = big;
  }
  __syncthreads();
  // kept overflow rows into free positions, in bank order
  for (uint32_t i = tid; i < 32 * kSpillPerBank; i += kPlanThreads) {
    const uint32_t bank = i / kSpillPerBank, o = i % kSpillPerBank;
    if (cnt[bank] <= cap || o >= cnt[bank] - cap) continue;
    const uint32_t ev = ov_start[bank] + o;
    for (uint32_t b2 = 0; b2 < 32; ++b2) {
      const uint32_t f = cnt[b2] < cap ? cap - cnt[b2] : 0u;
      if (ev >= free_start[b2] && ev < free_start[b2] + f) {
        const size_t e = entry(cnt[b2] + (ev - free_start[b2]), b2);
        pk_out[e] = encode(spill_row[bank][o]);
        k_out[e] = spill_k[bank][o];
      }
    }
  }
  // free positions no overflow row takes: empty entries (read a word of the
  // lane's own bank, write nothing)
  for (uint32_t i = tid; i < 32 * cap; i += kPlanThreads) {
    const uint32_t q = i / cap, pos = i % cap;
    if (pos < cnt[q]) continue;
    if (free_start[q] + (pos - cnt[q]) < total_ov) continue;
    const size_t e = entry(pos, q);
    pk_out[e] = q << 2;
    k_out[e] = -1;
  }
  if (redo) {
    __syncthreads();
    if (tid < 32) base[tid] = 0;
    __syncthreads();
    pass(1);
  }
}

__global__ void __launch_bounds__(kPlanThreads) build_plan_kernel(int32_t *__restrict__ idx, int64_t r,
                                                                  const int64_t *__restrict__ d_count,
                                                                  uint32_t *__restrict__ plan_pk,
                                                                  int32_t *__restrict__ plan_k, int slots,
                                                                  int64_t rows_per_group, int kgroups, uint64_t seed,
                                                                  uint64_t inst, uint64_t *__restrict__ sign_table,
                                                                  int64_t sign_words, int64_t sign_block0,
                                                                  int gen_L) {
  // the sketch launch that follows may be scheduled now (it waits for this
  // launch's completion before it reads the plan)
  asm volatile("griddepcontrol.launch_dependents;");
  plan_block((int)blockIdx.x, idx, r, d_count, plan_pk, plan_k, slots, rows_per_group, kgroups, seed, inst,
             sign_table, sign_words, sign_block0, gen_L);
}

// ---- many instances in one launch -----------------------------------------------
// Block b belongs to the instance p with first[p] <= b < first[p + 1].
__device__ __forceinline__ int batch_owner(const int64_t *__restrict__ first, int count, int64_t b) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (first[mid] <= b)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

__global__ void sample_iid_batched_kernel(const plan_job *__restrict__ jobs, const int64_t *__restrict__ first,
                                          int count) {
  const int p = batch_owner(first, count, blockIdx.x);
  const plan_job jb = jobs[p];
  const int64_t j = (int64_t)(blockIdx.x - first[p]) * blockDim.x + threadIdx.x;
  if (4 * j >= jb.r) return;
  const u64x4 u = philox4x64_10((uint64_t)j, kStreamIid, jb.seed, jb.inst);
#pragma unroll
  for (int w = 0; w < 4; ++w) {
    const int64_t k = 4 * j + w;
    if (k < jb.r) jb.idx[k] = (jb.L == 0) ? 0 : (int32_t)(u.w[w] >> (64 - jb.L));
  }
}

__global__ void __launch_bounds__(kPlanThreads) build_plan_batched_kernel(const plan_job *__restrict__ jobs,
                                                                          const int64_t *__restrict__ first,
                                                                          int count) {
  const int p = batch_owner(first, count, blockIdx.x);
  const plan_job jb = jobs[p];
  plan_block((int)(blockIdx.x - first[p]), jb.idx, jb.r, nullptr, jb.pk, jb.k, jb.slots, jb.rows_per_group,
             jb.kgroups, jb.seed, jb.inst, jb.signs, jb.sign_words, 0, 0);
}

int64_t sample_blocks(int64_t r) { return ((r + 3) / 4 + 255) / 256; }
int64_t plan_blocks(const plan_job &j) {
  return (int64_t)j.kgroups + (j.sign_words / 4 + kPlanThreads - 1) / kPlanThreads;
}

int launch_plan_batched(cudaStream_t s, const plan_job *d_jobs, const int64_t *d_first_sample,
                        const int64_t *d_first_plan, int count, int64_t sample_total, int64_t plan_total) {
  sample_iid_batched_kernel<<<(unsigned)sample_total, 256, 0, s>>>(d_jobs, d_first_sample, count);
  build_plan_batched_kernel<<<(unsigned)plan_total, kPlanThreads, 0, s>>>(d_jobs, d_first_plan, count);
  return cudaGetLastError() == cudaSuccess ? RNNLS_OK : RNNLS_ECUDA;
}

size_t plan_ws_bytes(int slots, int kgroups) {
  const size_t e = (size_t)kgroups * slots * kThreads;
  return align_up(e * sizeof(uint32_t), 256) + align_up(e * sizeof(int32_t), 256);
}

int launch_build_plan(cudaStream_t s, int32_t *idx, int64_t r, const int64_t *d_count, plan_t plan,
                      uint64_t *sign_table, int64_t sign_words, int64_t sign_block0, uint64_t seed, uint64_t inst,
                      int gen_L) {
  if (plan.rows_per_group > kPlanMaxRows || plan.rows_per_group > (int64_t)plan.slots * kThreads)
    return RNNLS_EUNSUPPORTED;
  if (!sign_table) sign_words = 0;
  const int64_t sign_blocks = (sign_words / 4 + kPlanThreads - 1) / kPlanThreads;
  build_plan_kernel<<<(unsigned)(plan.kgroups + sign_blocks), kPlanThreads, 0, s>>>(
      idx, r, d_count, plan.pk, plan.k, plan.slots, plan.rows_per_group, plan.kgroups, seed, inst, sign_table,
      sign_words, sign_block0, gen_L);
  return cudaGetLastError() == cudaSuccess ? RNNLS_OK : RNNLS_ECUDA;
}

}  // namespace rnnls
