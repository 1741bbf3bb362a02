// gram_tc.cu -- the sketch moments of Sec. 3.4 (Q = X'X for X = [SA | Sb],
// i.e. Q~ = (H~DA)'(H~DA), q~ = (H~DA)'H~Db and ||H~Db||^2) on the tcgen05
// tensor cores, with every product exact.
//
// The tensor cores multiply BF16 operands and accumulate in FP32, which
// rounds; the Lawson-Hanson decisions need the Gram to about 1e-13 of
// sqrt(Q_ii Q_jj).  So the products are made exact by an integer split (the
// error-free splitting of Ozaki et al., Numer. Algorithms 59, 2012):
//   * column j of X is scaled by 2^(7 - E_j), E_j the exponent of its
//     largest magnitude (2^(E_j - 1) <= max_k |x_kj| < 2^E_j), so that
//     every scaled value v has |v| < 128;
//   * v is cut into six integer slices s_0..s_5 by repeated rounding,
//     v = s_0 + 2^-8 s_1 + ... + 2^-40 s_5 + (a rest below 2^-41), each
//     |s_p| <= 128 and therefore exact in BF16;
//   * Q_ij = 2^(E_i + E_j - 14) sum_w 2^(-8w) G_w, G_w = sum over p + q = w
//     (w <= 5) of sum_k s_p[k, i] s_q[k, j].  A slice product is an integer
//     of at most 2^14 in magnitude, and an FP32 accumulator holds sums of
//     such integers exactly while they stay below 2^24: group w has its own
//     accumulator in tensor memory and is drained (read, scaled by the
//     power of two, added to float-float sums in registers) before
//     (w + 1) * rows * 2^14 can reach 2^24, i.e. after 512, 256, 256, 128,
//     128 and 128 rows for w = 0..5.
// What is dropped (the rests and the products with p + q > 5) is below about
// 2^-40 of max_k |x_ki| max_k |x_kj| per row.  The column magnitudes limit
// the data to the FP32 exponent range, as FP32 products would.
//
// Work split: a CTA of 128 threads owns one tile of Q (128 rows i x 64
// columns j; tiles wholly below the diagonal are skipped) and a range of
// 32-row chunks of X.  Per chunk every thread loads and slices its share of
// the tile's columns into shared memory (K-major core matrices, two buffers),
// then one thread issues 21 x 2 tcgen05.mma (M = 128, N = 64, K = 16) into
// six accumulators of 64 TMEM columns and commits them to an mbarrier; the
// slicing of chunk t + 1 runs while the tensor cores work on chunk t.
// K-splits of one tile add their FP64 partials in a fixed order in the last
// CTA to finish (a counter per tile, reset by that CTA).
#include <cuda_bf16.h>

#include <algorithm>

#include "kernels.h"
#include "launch_attr.h"
#include "tcgen05.cuh"

namespace rnnls {
namespace {

constexpr int kTM = 128;                     // tile rows (MMA M)
constexpr int kTN = 64;                      // tile columns (MMA N)
constexpr int kKC = 32;                      // rows of X per chunk
constexpr int kSl = 6;                       // slices per value
constexpr int kGroups = 6;                   // weight groups w = p + q
constexpr int kTcThreads = 128;
constexpr uint32_t kTmemCols = 512;          // 6 x 64 accumulator columns + 2 x 64 for the float-float sums
constexpr uint32_t kColHi = kGroups * kTN;   // TMEM columns of the running sums (hi, then lo)
constexpr uint32_t kColLo = kColHi + kTN;
constexpr uint32_t kLead = 128;              // bytes between core matrices adjacent along K
constexpr uint32_t kStride = (kKC / 8) * 128;  // bytes between core matrices adjacent along M / N
constexpr uint32_t kASlice = kTM * kKC * 2;  // bytes of one slice of the 128-row operand
constexpr uint32_t kBSlice = kTN * kKC * 2;  // bytes of one slice of the 64-row operand
constexpr uint32_t kBufBytes = kSl * (kASlice + kBSlice);
constexpr size_t kTcSmem = 2 * (size_t)kBufBytes;
constexpr uint32_t kWaitLimit = 1u << 22;    // mbarrier polls before a wait gives up
constexpr uint32_t kIdesc = tc::idesc_bf16_f32(kTM, kTN);

static_assert(kTcSmem <= 200 * 1024, "tile buffers exceed shared memory");
static_assert(kColLo + kTN <= kTmemCols, "accumulators exceed the TMEM allocation");

// Chunks between drains of group w: (w + 1) * 32 * period * 2^14 < 2^24.
__device__ __forceinline__ int drain_period(int w) { return w == 0 ? 16 : (w <= 2 ? 8 : 4); }

__device__ __forceinline__ const float *tc_col(const gram_tc_job &j, int g) {
  if (g < j.d) return j.S + (int64_t)g * j.lds;
  if (g < j.c) return j.s + (int64_t)(g - j.d) * j.ldt;
  return nullptr;
}

// x[0..7] = rows k..k+7 of column `col` (zero past m or for a missing column)
__device__ __forceinline__ void load8(const float *col, int64_t k, int64_t m, int vec4, float *x) {
  if (col && vec4 && k + 8 <= m) {
    const float4 a = __ldg(reinterpret_cast<const float4 *>(col + k));
    const float4 b = __ldg(reinterpret_cast<const float4 *>(col + k + 4));
    x[0] = a.x, x[1] = a.y, x[2] = a.z, x[3] = a.w, x[4] = b.x, x[5] = b.y, x[6] = b.z, x[7] = b.w;
  } else {
#pragma unroll
    for (int e = 0; e < 8; ++e) x[e] = (col && k + e < m) ? __ldg(col + k + e) : 0.0f;
  }
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // lo in the lower half (lower address)
  return *reinterpret_cast<const uint32_t *>(&v);
}

// The six slices of eight values (one 16-byte row of a core matrix each),
// written to dst + p * slice_bytes.  f1 * f2 = 2^(7 - E) (two factors so
// that each stays a normal FP32 number); every step is exact.
__device__ __forceinline__ void store_slices(uint32_t dst, uint32_t slice_bytes, const float *x, float f1, float f2) {
  float v[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) v[e] = __fmul_rn(__fmul_rn(x[e], f1), f2);
#pragma unroll
  for (int p = 0; p < kSl; ++p) {
    float s[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      s[e] = rintf(v[e]);
      v[e] = __fmul_rn(__fsub_rn(v[e], s[e]), 256.0f);
    }
    const uint32_t w0 = pack_bf16x2(s[0], s[1]), w1 = pack_bf16x2(s[2], s[3]);
    const uint32_t w2 = pack_bf16x2(s[4], s[5]), w3 = pack_bf16x2(s[6], s[7]);
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(dst + (uint32_t)p * slice_bytes), "r"(w0), "r"(w1),
                 "r"(w2), "r"(w3)
                 : "memory");
  }
}

__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float y) {
  const float s = __fadd_rn(hi, y);
  const float bp = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(y, bp));
  hi = s;
  lo = __fadd_rn(lo, e);
}

__device__ __forceinline__ void gram_tc_block(const gram_tc_job &jb, int64_t local) {
  extern __shared__ __align__(128) unsigned char tc_smem[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_base_s;
  __shared__ float colun_s[kTN];
  __shared__ int last_s;  // this CTA finished the tile's last K-split
  const int tid = threadIdx.x;
  const int tile = (int)(local % jb.tiles);
  const int split = (int)(local / jb.tiles);
  int mt = 0, nt = 0;
  gram_tc_tile_at(tile, jb.c, jb.d, jb.multi, mt, nt);
  const int i0 = mt * kTM, j0 = nt * kTN;
  // the 64 columns lie inside the 128 rows: their slices are rows of the A tile
  const bool alias = (j0 >= i0) && (j0 + kTN <= i0 + kTM);
  const int64_t nchunks = (jb.m + kKC - 1) / kKC;
  const int64_t ch0 = (int64_t)split * jb.chunks_per_split;
  const int64_t nch = max((int64_t)0, min(nchunks, ch0 + jb.chunks_per_split) - ch0);

  const uint32_t sbase = tc::smem_addr(tc_smem);
  const uint32_t bar0 = tc::smem_addr(&mbar[0]), bar1 = tc::smem_addr(&mbar[1]);
  if (tid == 0) {
    tc::mbar_init(bar0, 1);
    tc::mbar_init(bar1, 1);
    tc::fence_mbar_init();
    last_s = 0;
  }
  if (tid < 32) tc::tmem_alloc(tc::smem_addr(&tmem_base_s), kTmemCols);
  if (tid < kTN) colun_s[tid] = (j0 + tid < jb.c) ? jb.colunscale[j0 + tid] : 0.0f;

  // this thread's A column (tile row tid, TMEM lane tid) and B column
  const int gi = i0 + tid;
  const float *colA = tc_col(jb, gi);
  const float fa1 = colA ? jb.colscale[2 * gi] : 0.0f, fa2 = colA ? jb.colscale[2 * gi + 1] : 0.0f;
  const float row_un = colA ? jb.colunscale[gi] : 0.0f;
  const int gb = j0 + (tid & (kTN - 1));
  const float *colB = alias ? nullptr : tc_col(jb, gb);
  const float fb1 = colB ? jb.colscale[2 * gb] : 0.0f, fb2 = colB ? jb.colscale[2 * gb + 1] : 0.0f;

  auto slice_chunk = [&](int64_t ch, int buf) {
    const int64_t k0 = ch * kKC;
    const uint32_t bA = sbase + (uint32_t)buf * kBufBytes;
    const uint32_t rowA = bA + (uint32_t)(tid >> 3) * kStride + (uint32_t)(tid & 7) * 16;
#pragma unroll
    for (int ki = 0; ki < kKC / 8; ++ki) {
      float x[8];
      load8(colA, k0 + 8 * ki, jb.m, jb.vec4, x);
      store_slices(rowA + (uint32_t)ki * kLead, kASlice, x, fa1, fa2);
    }
    if (!alias) {
      const uint32_t bB = bA + kSl * kASlice;
      const int f = tid & (kTN - 1);
      const uint32_t rowB = bB + (uint32_t)(f >> 3) * kStride + (uint32_t)(f & 7) * 16;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int ki = (tid >> 6) + 2 * q;
        float x[8];
        load8(colB, k0 + 8 * ki, jb.m, jb.vec4, x);
        store_slices(rowB + (uint32_t)ki * kLead, kBSlice, x, fb1, fb2);
      }
    }
  };

  if (nch > 0) slice_chunk(ch0, 0);
  tc::fence_proxy_async();
  tc::tmem_fence_before();
  __syncthreads();
  tc::tmem_fence_after();
  const uint32_t tbase = tmem_base_s;
  const uint32_t tlane = tbase + ((uint32_t)(32 * (tid >> 5)) << 16);
  {
    // the running float-float sums of this thread's row start at zero
    uint32_t z[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) z[q] = 0u;
#pragma unroll
    for (int h = 0; h < 2 * kTN / 16; ++h) tc::tmem_st16(tlane + kColHi + 16 * h, z);
    tc::tmem_wait_st();
  }
  uint32_t fresh = (1u << kGroups) - 1;  // groups whose next MMA overwrites (thread 0's view)
  int64_t last_commit = -1;
  bool stalled = false;  // a bounded wait gave up (the same in every thread after each barrier)

  for (int64_t t = 0; t < nch; ++t) {
    const int buf = (int)(t & 1);
    if (tid == 0) {
      tc::tmem_fence_after();
      const uint32_t bA = sbase + (uint32_t)buf * kBufBytes;
      const uint32_t bB = alias ? bA + (uint32_t)((j0 - i0) >> 3) * kStride : bA + kSl * kASlice;
      const uint32_t bSl = alias ? kASlice : kBSlice;
#pragma unroll
      for (int w = 0; w < kGroups; ++w) {
        const uint32_t dcol = tbase + (uint32_t)(w * kTN);
        for (int p = 0; p <= w; ++p) {
#pragma unroll
          for (int kk = 0; kk < kKC / 16; ++kk) {
            const uint64_t ad = tc::smem_desc(bA + (uint32_t)p * kASlice + (uint32_t)kk * 2 * kLead, kLead, kStride);
            const uint64_t bd = tc::smem_desc(bB + (uint32_t)(w - p) * bSl + (uint32_t)kk * 2 * kLead, kLead, kStride);
            const uint32_t acc = ((fresh >> w) & 1u) && p == 0 && kk == 0 ? 0u : 1u;
            tc::mma_bf16(dcol, ad, bd, kIdesc, acc);
          }
        }
      }
      tc::mma_commit(buf ? bar1 : bar0);
      fresh = 0;
    }
    last_commit = t;
    if (t + 1 < nch) {
      // the other buffer was read by the MMAs of chunk t - 1
      if (t >= 1 && !tc::mbar_wait_bounded(buf ? bar0 : bar1, (uint32_t)(((t - 1) >> 1) & 1), kWaitLimit))
        stalled = true;
      slice_chunk(ch0 + t + 1, buf ^ 1);
      tc::fence_proxy_async();
    }
    uint32_t due = 0;
#pragma unroll
    for (int w = 0; w < kGroups; ++w)
      if (t + 1 == nch || ((t + 1) % drain_period(w)) == 0) due |= 1u << w;
    if (due) {
      if (!tc::mbar_wait_bounded(buf ? bar1 : bar0, (uint32_t)((t >> 1) & 1), kWaitLimit)) stalled = true;
      tc::tmem_fence_after();
#pragma unroll 1
      for (int half = 0; half < 2; ++half) {
        // columns 32 half .. + 31 of the row: running sums in, every due group added, sums out
        uint32_t h[32], l[32];
        tc::tmem_ld16(tlane + kColHi + 32 * half, h);
        tc::tmem_ld16(tlane + kColHi + 32 * half + 16, h + 16);
        tc::tmem_ld16(tlane + kColLo + 32 * half, l);
        tc::tmem_ld16(tlane + kColLo + 32 * half + 16, l + 16);
#pragma unroll 1
        for (int w = 0; w < kGroups; ++w) {
          if (!((due >> w) & 1u)) continue;
          uint32_t r[32];
          tc::tmem_ld16(tlane + (uint32_t)(w * kTN + 32 * half), r);
          tc::tmem_ld16(tlane + (uint32_t)(w * kTN + 32 * half + 16), r + 16);
          tc::tmem_wait_ld();
          const float fw = __fmul_rn(row_un, __int_as_float((127 - 8 * w) << 23));  // row scale x 2^-8w
#pragma unroll
          for (int q = 0; q < 32; ++q) {
            float hv = __uint_as_float(h[q]), lv = __uint_as_float(l[q]);
            two_sum_acc(hv, lv, __fmul_rn(__fmul_rn(__uint_as_float(r[q]), fw), colun_s[32 * half + q]));
            h[q] = __float_as_uint(hv);
            l[q] = __float_as_uint(lv);
          }
        }
        tc::tmem_st16(tlane + kColHi + 32 * half, h);
        tc::tmem_st16(tlane + kColHi + 32 * half + 16, h + 16);
        tc::tmem_st16(tlane + kColLo + 32 * half, l);
        tc::tmem_st16(tlane + kColLo + 32 * half + 16, l + 16);
        tc::tmem_wait_st();
      }
      tc::tmem_fence_before();
      if (tid == 0) fresh |= due;
    }
    stalled = __syncthreads_or(stalled) != 0;
    if (stalled) break;
  }

  if (stalled && last_commit >= 0) {
    // let the MMAs in flight finish (bounded) before the memory they use is released
    const int64_t t = last_commit;
    tc::mbar_wait_bounded((t & 1) ? bar1 : bar0, (uint32_t)((t >> 1) & 1), kWaitLimit);
  }
  const double nanv = __longlong_as_double(0x7ff8000000000000ll);
  const int c = jb.c;
  auto write_q = [&](int i, int j, double v) {
    const float h = (float)v;
    const float l = (float)(v - (double)h);
    jb.Qd[(int64_t)i * c + j] = v;
    jb.Qd[(int64_t)j * c + i] = v;
    jb.Qhi[(int64_t)i * c + j] = h;
    jb.Qhi[(int64_t)j * c + i] = h;
    jb.Qlo[(int64_t)i * c + j] = l;
    jb.Qlo[(int64_t)j * c + i] = l;
  };
  // the row's sums as FP64, 32 columns at a time (the final drain ended with wait::st)
  auto row_sums = [&](int half, double *v) {
    uint32_t h[32], l[32];
    tc::tmem_ld16(tlane + kColHi + 32 * half, h);
    tc::tmem_ld16(tlane + kColHi + 32 * half + 16, h + 16);
    tc::tmem_ld16(tlane + kColLo + 32 * half, l);
    tc::tmem_ld16(tlane + kColLo + 32 * half + 16, l + 16);
    tc::tmem_wait_ld();
#pragma unroll
    for (int q = 0; q < 32; ++q)
      v[q] = stalled ? nanv : (double)__uint_as_float(h[q]) + (double)__uint_as_float(l[q]);
  };
  if (jb.splits == 1) {
#pragma unroll 1
    for (int half = 0; half < 2; ++half) {
      double v[32];
      row_sums(half, v);
      if (gi < c) {
#pragma unroll
        for (int q = 0; q < 32; ++q) {
          const int j = j0 + 32 * half + q;
          if (j < c && gi <= j) write_q(gi, j, v[q]);
        }
      }
    }
  } else {
    double *mine = jb.part + ((int64_t)split * jb.tiles + tile) * (kTM * kTN) + (int64_t)tid * kTN;
#pragma unroll 1
    for (int half = 0; half < 2; ++half) {
      double v[32];
      row_sums(half, v);
#pragma unroll
      for (int q = 0; q < 32; ++q) mine[32 * half + q] = v[q];
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) {
      const unsigned int done = atomicAdd(&jb.counters[tile], 1u);
      if (done == (unsigned int)(jb.splits - 1)) last_s = 1;
    }
    __syncthreads();
    if (last_s) {
      __threadfence();
#pragma unroll 1
      for (int half = 0; half < 2; ++half) {
        double acc[32];
#pragma unroll
        for (int q = 0; q < 32; ++q) acc[q] = 0.0;
        for (int sp = 0; sp < jb.splits; ++sp) {
          const double *src =
              jb.part + ((int64_t)sp * jb.tiles + tile) * (kTM * kTN) + (int64_t)tid * kTN + 32 * half;
#pragma unroll
          for (int q = 0; q < 32; ++q) acc[q] += __ldcg(src + q);
        }
        if (gi < c) {
#pragma unroll
          for (int q = 0; q < 32; ++q) {
            const int j = j0 + 32 * half + q;
            if (j < c && gi <= j) write_q(gi, j, acc[q]);
          }
        }
      }
      if (tid == 0) jb.counters[tile] = 0u;
    }
  }
  tc::tmem_fence_before();
  __syncthreads();
  tc::tmem_fence_after();
  if (tid < 32) tc::tmem_dealloc(tbase, kTmemCols);
}

__global__ void __launch_bounds__(kTcThreads, 1) gram_tc_kernel_one(const gram_tc_job jb) {
  gram_tc_block(jb, blockIdx.x);
}

// Many problems in one launch: CTA b belongs to the problem p with
// first[p] <= b < first[p + 1] (tiles x splits CTAs each).
__global__ void __launch_bounds__(kTcThreads, 1) gram_tc_kernel_batched(const gram_tc_job *__restrict__ jobs,
                                                                        const int64_t *__restrict__ first, int count) {
  int lo = 0, hi = count - 1;
  const int64_t bid = blockIdx.x;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (first[mid] <= bid)
      lo = mid;
    else
      hi = mid - 1;
  }
  const gram_tc_job jb = jobs[lo];
  gram_tc_block(jb, bid - first[lo]);
}

// Per column g of X: the scale 2^(7 - E_g) as two factors, its inverse
// 2^(E_g - 7), and for columns of S the compensated sum of magnitudes
// (||S||_1 = max_g of these sums).  One block per column.
constexpr int kStatThreads = 256;
__device__ __forceinline__ void colstats_block(const gram_tc_job &jb, int g) {
  __shared__ float smax[kStatThreads / 32];
  __shared__ double ssum[kStatThreads / 32];
  const float *col = tc_col(jb, g);
  float mx = 0.0f;
  dot2 acc;
  for (int64_t k = threadIdx.x; k < jb.m; k += kStatThreads) {
    const float a = fabsf(__ldg(col + k));
    mx = fmaxf(mx, a);
    acc.add(a);
  }
  const ff v = acc.value();
  double sum = (double)v.hi + (double)v.lo;
  for (int o = 16; o > 0; o >>= 1) {
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    sum += __shfl_xor_sync(0xffffffffu, sum, o);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    smax[w] = mx;
    ssum[w] = sum;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float m = 0.0f;
    double s = 0.0;
    for (int q = 0; q < kStatThreads / 32; ++q) {
      m = fmaxf(m, smax[q]);
      s += ssum[q];
    }
    float f1 = 0.0f, f2 = 0.0f, un = 0.0f;
    if (m > 0.0f && isfinite(m)) {
      int E = 0;
      frexpf(m, &E);  // m = f 2^E, f in [0.5, 1)
      const int k = 7 - E;
      const int k1 = k / 2;
      f1 = ldexpf(1.0f, k1);
      f2 = ldexpf(1.0f, k - k1);
      un = ldexpf(1.0f, E - 7);
    } else if (!(m == 0.0f)) {
      // an infinity or NaN in the column: make the Gram non-finite so that
      // the solve reports it
      f1 = f2 = un = __int_as_float(0x7fc00000);
    }
    jb.colscale[2 * g] = f1;
    jb.colscale[2 * g + 1] = f2;
    jb.colunscale[g] = un;
    if (g < jb.d && jb.colabs) jb.colabs[g] = s;
  }
}

__global__ void __launch_bounds__(kStatThreads) colstats_kernel_one(const gram_tc_job jb) {
  colstats_block(jb, blockIdx.x);
}

__global__ void __launch_bounds__(kStatThreads) colstats_kernel_batched(const gram_tc_job *__restrict__ jobs,
                                                                        const int64_t *__restrict__ first, int count) {
  int lo = 0, hi = count - 1;
  const int64_t bid = blockIdx.x;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (first[mid] <= bid)
      lo = mid;
    else
      hi = mid - 1;
  }
  const gram_tc_job jb = jobs[lo];
  colstats_block(jb, (int)(bid - first[lo]));
}

smem_attr g_tc_one_attr, g_tc_batched_attr;

}  // namespace

int gram_tc_tile_count(int c, int d, int multi) {
  int n = 0;
  for (int mt = 0; mt * kTM < c; ++mt)
    for (int nt = 0; nt * kTN < c; ++nt) n += gram_tc_tile_needed(mt, nt, c, d, multi) ? 1 : 0;
  return n;
}

gram_tc_job gram_tc_plan(const float *S, int64_t lds, const float *s, int64_t ldt, int nb, int64_t m, int d,
                         int multi, int want_ctas, int64_t max_chunks_per_cta) {
  gram_tc_job j{};
  j.S = S;
  j.s = s;
  j.lds = lds;
  j.ldt = ldt;
  j.nb = nb;
  j.m = m;
  j.d = d;
  j.c = d + nb;
  j.multi = multi;
  j.tiles = gram_tc_tile_count(j.c, d, multi);
  const int64_t chunks = std::max<int64_t>(1, (m + kKC - 1) / kKC);
  int64_t splits = std::max<int64_t>(1, ((int64_t)want_ctas + j.tiles - 1) / j.tiles);
  splits = std::min<int64_t>(splits, std::max<int64_t>(1, chunks / 8));  // at least 8 chunks per CTA
  splits = std::max<int64_t>(splits, (chunks + max_chunks_per_cta - 1) / max_chunks_per_cta);
  j.chunks_per_split = (chunks + splits - 1) / splits;
  j.splits = (int)((chunks + j.chunks_per_split - 1) / j.chunks_per_split);
  const auto al = [](const void *p) { return ((uintptr_t)p & 15u) == 0; };
  j.vec4 = (al(S) && (lds % 4) == 0 && (nb == 0 || (al(s) && (nb == 1 || (ldt % 4) == 0)))) ? 1 : 0;
  return j;
}

size_t gram_tc_ws_bytes(const gram_tc_job &j) {
  size_t b = align_up((size_t)2 * j.c * sizeof(float), 256) + align_up((size_t)j.c * sizeof(float), 256);
  if (j.splits > 1) b += align_up((size_t)j.splits * j.tiles * kTM * kTN * sizeof(double), 256);
  return b;
}

void gram_tc_carve(gram_tc_job &j, ws_carver &wc, unsigned int *counters, double *Qd, float *Qhi, float *Qlo,
                   double *colabs) {
  j.colscale = wc.take<float>((size_t)2 * j.c);
  j.colunscale = wc.take<float>((size_t)j.c);
  j.part = j.splits > 1 ? wc.take<double>((size_t)j.splits * j.tiles * kTM * kTN) : nullptr;
  j.counters = counters;
  j.Qd = Qd;
  j.Qhi = Qhi;
  j.Qlo = Qlo;
  j.colabs = colabs;
}

int gram_tc_launch_one(rnnls_ctx *ctx, const gram_tc_job &j) {
  cudaStream_t s = ctx->stream;
  {
    prof_scope ps(ctx, K_COLSTATS);
    colstats_kernel_one<<<(unsigned)j.c, kStatThreads, 0, s>>>(j);
  }
  prof_scope ps(ctx, K_GRAM_TC);
  RNNLS_CUDA_TRY(g_tc_one_attr.ensure((const void *)gram_tc_kernel_one, kTcSmem));
  gram_tc_kernel_one<<<(unsigned)((int64_t)j.tiles * j.splits), kTcThreads, kTcSmem, s>>>(j);
  return cudaGetLastError() == cudaSuccess ? RNNLS_OK : RNNLS_ECUDA;
}

int gram_tc_launch_batched(rnnls_ctx *ctx, const gram_tc_job *d_jobs, const int64_t *d_first_col,
                           const int64_t *d_first_cta, int count, int64_t cols, int64_t ctas) {
  cudaStream_t s = ctx->stream;
  {
    prof_scope ps(ctx, K_COLSTATS);
    colstats_kernel_batched<<<(unsigned)cols, kStatThreads, 0, s>>>(d_jobs, d_first_col, count);
  }
  prof_scope ps(ctx, K_GRAM_TC);
  RNNLS_CUDA_TRY(g_tc_batched_attr.ensure((const void *)gram_tc_kernel_batched, kTcSmem));
  gram_tc_kernel_batched<<<(unsigned)ctas, kTcThreads, kTcSmem, s>>>(d_jobs, d_first_cta, count);
  return cudaGetLastError() == cudaSuccess ? RNNLS_OK : RNNLS_ECUDA;
}

int gram_f32(rnnls_ctx *ctx, const float *SA, int64_t ldsa, const float *Sb, int64_t r, int64_t d, double *Q,
             double *colabs) {
  gram_tc_job gj = gram_tc_plan(SA, ldsa, Sb, r, 1, r, (int)d, 0, ctx->num_sms, (int64_t)1 << 40);
  const size_t D1 = (size_t)d + 1;
  const size_t bytes = 2 * align_up(D1 * D1 * 4, 256) + gram_tc_ws_bytes(gj) + 1024;
  int st = ensure_workspace(ctx, bytes);
  if (st) return st;
  unsigned int *counters = nullptr;
  st = ensure_counters(ctx, (size_t)gj.tiles, &counters);
  if (st) return st;
  ws_carver wc(ctx->ws);
  float *Qhi = wc.take<float>(D1 * D1);
  float *Qlo = wc.take<float>(D1 * D1);
  gram_tc_carve(gj, wc, counters, Q, Qhi, Qlo, colabs);
  return gram_tc_launch_one(ctx, gj);
}

}  // namespace rnnls
