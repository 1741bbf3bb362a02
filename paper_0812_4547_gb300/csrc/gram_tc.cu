// gram_tc.cu -- the sketch moments of Sec. 3.4 (Q = X'X for X = [SA | Sb],
// i.e. Q~ = (H~DA)'(H~DA), q~ = (H~DA)'H~Db and ||H~Db||^2) on the tcgen05
// tensor cores, with the leading products exact.
//
// The tensor cores multiply BF16 operands and accumulate in FP32, which
// rounds; the Lawson-Hanson decisions need the Gram to about 1e-13 of
// sqrt(Q_ii Q_jj).  So the products are made exact by an integer split (the
// error-free splitting of Ozaki et al., Numer. Algorithms 59, 2012):
//   * column j of X is scaled by 2^(7 - E_j), E_j the exponent of its
//     largest magnitude (2^(E_j - 1) <= max_k |x_kj| < 2^E_j), so that
//     every scaled value v has |v| < 128;
//   * v is cut into six slices by rounding to multiples of 2^-8p,
//     v = t_0 + t_1 + ... + t_5 + (a rest below 2^-41), t_p = 2^-8p s_p with
//     an integer |s_p| <= 128, so every t_p is exact in BF16;
//   * Q_ij = 2^(E_i + E_j - 14) sum_w G_w, G_w = sum over p + q = w of
//     sum_k t_p[k, i] t_q[k, j].  Every product in G_w is an integer
//     multiple of 2^-8w of magnitude at most 2^(14 - 8w), and an FP32
//     accumulator holds sums of such multiples exactly while they stay below
//     2^(24 - 8w): G_0, G_1 and G_2 have their own tensor-memory
//     accumulators, drained (read, scaled by the power of two, added to
//     float-float sums) after 512, 256 and 256 rows, well before that bound;
//     G_3 + G_4 + G_5 (weights 2^-24 and below) share one accumulator that
//     rounds, drained every 256 rows.
// What is dropped or rounded (the rests, the products with p + q > 5, the
// shared accumulator's roundings) is below about 2^-39 of
// max_k |x_ki| max_k |x_kj| per row.  The column magnitudes limit the data to
// the FP32 exponent range, as FP32 products would.
//
// Work split: a CTA owns one tile of Q (128 rows i x 64 columns j; tiles
// wholly below the diagonal are skipped) and a range of 32-row chunks of X.
// Eight warps slice their share of the tile's columns into shared memory
// (K-major core matrices, two buffers; the values of the next three chunks
// are copied ahead into a ring in shared memory with cp.async) and drain the
// accumulators; a ninth warp issues, per
// chunk, 21 x 2 tcgen05.mma (M = 128, N = 64, K = 16) into the four
// accumulators and commits them to an mbarrier.  The warps meet only at
// mbarriers: "full" (a buffer is sliced), "mma_done" (the tensor cores are
// through a buffer) and "drained" (the due accumulators were read back), so
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

constexpr int kTM = 128;                       // tile rows (MMA M)
constexpr int kTN = 64;                        // tile columns (MMA N)
constexpr int kKC = 32;                        // rows of X per chunk
constexpr int kSl = 6;                         // slices per value
constexpr int kSliceThreads = 256;            // eight slicing / draining warps
constexpr int kTcThreads = kSliceThreads + 32; // plus the MMA warp
constexpr uint32_t kTmemCols = 512;            // 4 accumulators + 2 running sums of 64 columns, rounded up
constexpr uint32_t kColHi = 4 * kTN;           // TMEM columns of the running sums (hi, then lo)
constexpr uint32_t kColLo = kColHi + kTN;
constexpr uint32_t kLead = 128;                // bytes between core matrices adjacent along K
constexpr uint32_t kStride = (kKC / 8) * 128;  // bytes between core matrices adjacent along M / N
constexpr uint32_t kASlice = kTM * kKC * 2;    // bytes of one slice of the 128-row operand
constexpr uint32_t kBSlice = kTN * kKC * 2;    // bytes of one slice of the 64-row operand
constexpr uint32_t kBufBytes = kSl * (kASlice + kBSlice);
// raw FP32 values of a chunk, copied ahead: per slicing thread 16 rows of its
// A feature and 8 of its B feature, stored as 16-byte units [unit][thread]
constexpr int kRawDepth = 3;                       // chunks copied ahead of the one being sliced
constexpr uint32_t kRawA = kSliceThreads * 64;     // bytes of a chunk's A values
constexpr uint32_t kRawBytes = kRawA + kSliceThreads * 32;
constexpr size_t kTcSmem = 2 * (size_t)kBufBytes + (size_t)kRawDepth * kRawBytes;
constexpr uint32_t kWaitLimit = 1u << 22;      // mbarrier polls before a wait gives up
constexpr uint32_t kShortWait = 64;            // polls once some wait has given up
constexpr uint32_t kIdesc = tc::idesc_bf16_f32(kTM, kTN);

static_assert(kTcSmem <= 220 * 1024, "tile buffers exceed shared memory");
static_assert(kColLo + kTN <= kTmemCols, "accumulators exceed the TMEM allocation");

// Accumulator a (0, 1, 2: the exact groups G_0, G_1, G_2; 3: G_3 + G_4 + G_5)
// is drained after every drain_period(a) chunks: (w + 1) * 32 * period *
// 2^14 stays within 2^23 for the exact ones.
__host__ __device__ constexpr int drain_period(int a) { return a == 0 ? 16 : 8; }
__device__ __forceinline__ constexpr int acc_of(int w) { return w < 3 ? w : 3; }

__device__ __forceinline__ const float *tc_col(const gram_tc_job &j, int g) {
  if (g < j.d) return j.S + (int64_t)g * j.lds;
  if (g < j.c) return j.s + (int64_t)(g - j.d) * j.ldt;
  return nullptr;
}

// x[0..n-1] = rows k..k+n-1 of column `col` (zero past m or for a missing column)
template <int n>
__device__ __forceinline__ void load_rows(const float *col, int64_t k, int64_t m, int vec4, float *x) {
  if (col && vec4 && k + n <= m) {
#pragma unroll
    for (int e = 0; e < n; e += 4) {
      const float4 a = __ldg(reinterpret_cast<const float4 *>(col + k + e));
      x[e] = a.x, x[e + 1] = a.y, x[e + 2] = a.z, x[e + 3] = a.w;
    }
  } else {
#pragma unroll
    for (int e = 0; e < n; ++e) x[e] = (col && k + e < m) ? __ldg(col + k + e) : 0.0f;
  }
}

// Rows k..k+n-1 of column `col` copied to shared memory at dst, dst + ustride,
// ... (16 bytes each): cp.async when the rows are 16-byte aligned and inside
// the column, else plain loads (zero past m or for a missing column) stored
// by the thread itself.
template <int n>
__device__ __forceinline__ void copy_rows(const float *col, int64_t k, int64_t m, int vec4, uint32_t dst,
                                          uint32_t ustride) {
  if (col && vec4 && k + n <= m) {
#pragma unroll
    for (int e = 0; e < n; e += 4)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst + (uint32_t)(e / 4) * ustride),
                   "l"(col + k + e)
                   : "memory");
  } else {
    float x[n];
    load_rows<n>(col, k, m, 0, x);
#pragma unroll
    for (int e = 0; e < n; e += 4)
      asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(dst + (uint32_t)(e / 4) * ustride), "f"(x[e]),
                   "f"(x[e + 1]), "f"(x[e + 2]), "f"(x[e + 3])
                   : "memory");
  }
}
template <int n>
__device__ __forceinline__ void read_rows(uint32_t src, uint32_t ustride, float *x) {
#pragma unroll
  for (int e = 0; e < n; e += 4)
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(x[e]), "=f"(x[e + 1]), "=f"(x[e + 2]), "=f"(x[e + 3])
                 : "r"(src + (uint32_t)(e / 4) * ustride)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// wait until at most `pending` (0, 1 or 2) of this thread's copy groups are still in flight
__device__ __forceinline__ void cp_async_wait(int pending) {
  if (pending >= 2)
    asm volatile("cp.async.wait_group 2;" ::: "memory");
  else if (pending == 1)
    asm volatile("cp.async.wait_group 1;" ::: "memory");
  else
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ uint64_t f2_pack(float lo, float hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t f2_sub(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
// two FP32 values (lower half first) as a BF16 pair, the first in the lower half
__device__ __forceinline__ uint32_t f2_to_bf16x2(uint64_t v) {
  uint32_t d;
  asm("{\n\t.reg .f32 lo, hi;\n\tmov.b64 {lo, hi}, %1;\n\tcvt.rn.bf16x2.f32 %0, hi, lo;\n\t}" : "=r"(d) : "l"(v));
  return d;
}

// The six slices of eight values (one 16-byte row of a core matrix each),
// written to dst + p * slice_bytes.  sc = (f1, f1), (f2, f2) with
// f1 f2 = 2^(7 - E).  Slice p rounds the rest to a multiple of 2^-8p by
// adding and subtracting 1.5 * 2^(23 - 8p) (round to nearest even); every
// step is exact, on pairs of values (packed f32x2).
__device__ __forceinline__ void store_slices(uint32_t dst, uint32_t slice_bytes, const float *x, uint64_t sc1,
                                             uint64_t sc2) {
  uint64_t v[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) v[e] = f2_mul(f2_mul(f2_pack(x[2 * e], x[2 * e + 1]), sc1), sc2);
#pragma unroll
  for (int p = 0; p < kSl; ++p) {
    const float cf = 1.5f * __int_as_float((127 + 23 - 8 * p) << 23);
    const uint64_t C = f2_pack(cf, cf);
    uint32_t w[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const uint64_t t = f2_sub(f2_add(v[e], C), C);
      v[e] = f2_sub(v[e], t);
      w[e] = f2_to_bf16x2(t);
    }
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(dst + (uint32_t)p * slice_bytes), "r"(w[0]),
                 "r"(w[1]), "r"(w[2]), "r"(w[3])
                 : "memory");
  }
}

__device__ __forceinline__ void store_zero_slices(uint32_t dst, uint32_t slice_bytes) {
#pragma unroll
  for (int p = 0; p < kSl; ++p)
    asm volatile("st.shared.v4.b32 [%0], {%1, %1, %1, %1};" ::"r"(dst + (uint32_t)p * slice_bytes), "r"(0u) : "memory");
}

__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float y) {
  const float s = __fadd_rn(hi, y);
  const float bp = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(y, bp));
  hi = s;
  lo = __fadd_rn(lo, e);
}

// Accumulators drained after chunk t (relative to the CTA's first chunk).
__device__ __forceinline__ uint32_t due_after(int64_t t, int64_t nch) {
  uint32_t due = 0;
#pragma unroll
  for (int a = 0; a < 4; ++a)
    if (t + 1 == nch || ((t + 1) % drain_period(a)) == 0) due |= 1u << a;
  return due;
}

__device__ __forceinline__ void gram_tc_block(const gram_tc_job &jb, int64_t local) {
  extern __shared__ __align__(128) unsigned char tc_smem[];
  __shared__ __align__(8) uint64_t mbar[5];  // full[2], mma_done[2], drained
  __shared__ uint32_t tmem_base_s;
  __shared__ float colun_s[kTN];
  __shared__ int last_s;  // this CTA finished the tile's last K-split
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
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
  const uint32_t full0 = tc::smem_addr(&mbar[0]), done0 = tc::smem_addr(&mbar[2]);
  const uint32_t drained = tc::smem_addr(&mbar[4]);
  auto full_bar = [&](int b) { return full0 + 8u * (uint32_t)b; };
  auto done_bar = [&](int b) { return done0 + 8u * (uint32_t)b; };
  if (tid == 0) {
    tc::mbar_init(full_bar(0), kSliceThreads / 32);
    tc::mbar_init(full_bar(1), kSliceThreads / 32);
    tc::mbar_init(done_bar(0), 1);
    tc::mbar_init(done_bar(1), 1);
    tc::mbar_init(drained, kSliceThreads / 32);
    tc::fence_mbar_init();
    last_s = 0;
  }
  if (warp == 0) tc::tmem_alloc(tc::smem_addr(&tmem_base_s), kTmemCols);
  if (tid < kTN) colun_s[tid] = (j0 + tid < jb.c) ? jb.colunscale[j0 + tid] : 0.0f;
  tc::tmem_fence_before();
  __syncthreads();
  tc::tmem_fence_after();
  const uint32_t tbase = tmem_base_s;
  bool stalled = false;  // some bounded wait of this thread gave up
  auto wait = [&](uint32_t bar, uint32_t parity) {
    if (!tc::mbar_wait_bounded(bar, parity, stalled ? kShortWait : kWaitLimit)) stalled = true;
  };

  // drain roles: TMEM lane (tile row) 32 (warp % 4) + lane, columns 32 (warp / 4) ..
  const int drow = 32 * (warp & 3) + lane, dcol = 32 * ((warp >> 2) & 1);
  const uint32_t tlane = tbase + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)dcol;

  if (warp < kSliceThreads / 32) {
    // ---- slicing and draining warps ----------------------------------------
    // A feature fa (tile row), its rows 16 ha .. 16 ha + 15 of a chunk (core
    // matrices ki = 2 ha, 2 ha + 1); B feature fb, rows 8 kb .. 8 kb + 7
    const int fa = tid & (kTM - 1), ha = tid >> 7;
    const float *colA = tc_col(jb, i0 + fa);
    const float a1 = colA ? jb.colscale[2 * (i0 + fa)] : 0.0f, a2 = colA ? jb.colscale[2 * (i0 + fa) + 1] : 0.0f;
    const uint64_t scA1 = f2_pack(a1, a1), scA2 = f2_pack(a2, a2);
    const int fb = tid & (kTN - 1), kb = tid >> 6;
    const float *colB = alias ? nullptr : tc_col(jb, j0 + fb);
    const float b1 = colB ? jb.colscale[2 * (j0 + fb)] : 0.0f, b2 = colB ? jb.colscale[2 * (j0 + fb) + 1] : 0.0f;
    const uint64_t scB1 = f2_pack(b1, b1), scB2 = f2_pack(b2, b2);
    const uint32_t offA = (uint32_t)(fa >> 3) * kStride + (uint32_t)(fa & 7) * 16 + (uint32_t)(2 * ha) * kLead;
    const uint32_t offB =
        kSl * kASlice + (uint32_t)(fb >> 3) * kStride + (uint32_t)(fb & 7) * 16 + (uint32_t)kb * kLead;
    const float row_un = (i0 + drow < jb.c) ? jb.colunscale[i0 + drow] : 0.0f;

    // the values of chunk t are copied into ring slot t % kRawDepth, kRawDepth
    // chunks ahead (one copy group per chunk); this thread reads back only
    // what it copied itself
    const uint32_t rawbase = sbase + 2 * kBufBytes + (uint32_t)tid * 16;
    constexpr uint32_t kUnit = kSliceThreads * 16;  // between a thread's 16-byte units
    auto issue_chunk = [&](int64_t t) {
      if (t < nch) {
        const int64_t k0 = (ch0 + t) * kKC;
        const uint32_t slot = rawbase + (uint32_t)(t % kRawDepth) * kRawBytes;
        if (colA) copy_rows<16>(colA, k0 + 16 * ha, jb.m, jb.vec4, slot, kUnit);
        if (colB) copy_rows<8>(colB, k0 + 8 * kb, jb.m, jb.vec4, slot + kRawA, kUnit);
      }
      cp_async_commit();  // an empty group past the last chunk keeps the counting uniform
    };
    // columns past c slice to zero: written once into both buffers
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const uint32_t base = sbase + (uint32_t)b * kBufBytes;
      if (!colA) {
        store_zero_slices(base + offA, kASlice);
        store_zero_slices(base + offA + kLead, kASlice);
      }
      if (!alias && !colB) store_zero_slices(base + offB, kBSlice);
    }
    {
      // the running float-float sums of this thread's 32 entries start at zero
      uint32_t z[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) z[q] = 0u;
      tc::tmem_st16(tlane + kColHi, z);
      tc::tmem_st16(tlane + kColHi + 16, z);
      tc::tmem_st16(tlane + kColLo, z);
      tc::tmem_st16(tlane + kColLo + 16, z);
      tc::tmem_wait_st();
    }
    // due accumulators into the running sums, 16 of the thread's 32 columns at a time
    auto drain = [&](uint32_t due) {
#pragma unroll 1
      for (int hh = 0; hh < 32; hh += 16) {
        uint32_t h[16], l[16];
        tc::tmem_ld16(tlane + kColHi + hh, h);
        tc::tmem_ld16(tlane + kColLo + hh, l);
#pragma unroll 1
        for (int a = 0; a < 4; ++a) {
          if (!((due >> a) & 1u)) continue;
          uint32_t r[16];
          tc::tmem_ld16(tlane + (uint32_t)(a * kTN + hh), r);
          tc::tmem_wait_ld();
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            float hv = __uint_as_float(h[q]), lv = __uint_as_float(l[q]);
            two_sum_acc(hv, lv, __fmul_rn(__fmul_rn(__uint_as_float(r[q]), row_un), colun_s[dcol + hh + q]));
            h[q] = __float_as_uint(hv);
            l[q] = __float_as_uint(lv);
          }
        }
        tc::tmem_st16(tlane + kColHi + hh, h);
        tc::tmem_st16(tlane + kColLo + hh, l);
      }
      tc::tmem_wait_st();
    };

    // one chunk: slice it from its ring slot, copy chunk t + kRawDepth into
    // that slot, then drain what is due after chunk t - 1
    auto step = [&](int64_t t) {
      const int b = (int)(t & 1);
      cp_async_wait(kRawDepth - 1);  // chunk t's group has landed (later groups may be in flight)
      float xa[16], xb[8];
      const uint32_t slot = rawbase + (uint32_t)(t % kRawDepth) * kRawBytes;
      if (colA) read_rows<16>(slot, kUnit, xa);
      if (colB) read_rows<8>(slot + kRawA, kUnit, xb);
      if (t >= 2) wait(done_bar(b), (uint32_t)(((t - 2) >> 1) & 1));  // the MMAs of chunk t - 2 read this buffer
      const uint32_t base = sbase + (uint32_t)b * kBufBytes;
      if (colA) {
        store_slices(base + offA, kASlice, xa, scA1, scA2);
        store_slices(base + offA + kLead, kASlice, xa + 8, scA1, scA2);
      }
      if (colB) store_slices(base + offB, kBSlice, xb, scB1, scB2);
      tc::fence_proxy_async();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(full_bar(b));
      issue_chunk(t + kRawDepth);
      if (t >= 1) {
        const uint32_t due = due_after(t - 1, nch);
        if (due) {
          wait(done_bar((int)((t - 1) & 1)), (uint32_t)(((t - 1) >> 1) & 1));
          tc::tmem_fence_after();
          drain(due);
          tc::tmem_fence_before();
          __syncwarp();
          if (lane == 0) tc::mbar_arrive(drained);
        }
      }
    };
    for (int q = 0; q < kRawDepth; ++q) issue_chunk(q);
    for (int64_t t = 0; t < nch; ++t) step(t);
    cp_async_wait(0);
    if (nch > 0) {
      const int64_t t = nch - 1;
      wait(done_bar((int)(t & 1)), (uint32_t)((t >> 1) & 1));
      tc::tmem_fence_after();
      drain(due_after(t, nch));
    }
  } else if (lane == 0) {
    // ---- the MMA warp (one issuing thread) ---------------------------------
    uint32_t fresh = 0xFu;  // accumulators whose next MMA overwrites
    uint32_t events = 0;    // drain events waited for
    for (int64_t t = 0; t < nch; ++t) {
      const int b = (int)(t & 1);
      wait(full_bar(b), (uint32_t)((t >> 1) & 1));
      if (t >= 1) {
        const uint32_t due = due_after(t - 1, nch);
        if (due) {
          wait(drained, events & 1u);
          ++events;
          fresh |= due;
        }
      }
      tc::tmem_fence_after();
      const uint32_t bA = sbase + (uint32_t)b * kBufBytes;
      const uint32_t bB = alias ? bA + (uint32_t)((j0 - i0) >> 3) * kStride : bA + kSl * kASlice;
      const uint32_t bSl = alias ? kASlice : kBSlice;
      const uint64_t dA = tc::smem_desc(bA, kLead, kStride);
      const uint64_t dB = tc::smem_desc(bB, kLead, kStride);
#pragma unroll
      for (int w = 0; w < kSl; ++w) {
        const int a = acc_of(w);
#pragma unroll
        for (int p = 0; p <= w; ++p) {
#pragma unroll
          for (int kk = 0; kk < kKC / 16; ++kk) {
            const uint64_t ad = dA + (uint64_t)((p * kASlice + kk * 2 * kLead) >> 4);
            const uint64_t bd = dB + (uint64_t)(((uint32_t)(w - p) * bSl + (uint32_t)kk * 2 * kLead) >> 4);
            const bool first = (p == 0 && kk == 0 && (a < 3 || w == 3));
            tc::mma_bf16(tbase + (uint32_t)(a * kTN), ad, bd, kIdesc, (first && ((fresh >> a) & 1u)) ? 0u : 1u);
          }
        }
      }
      tc::mma_commit(done_bar(b));
      fresh = 0;
    }
  }
  stalled = __syncthreads_or(stalled) != 0;

  const double nanv = __longlong_as_double(0x7ff8000000000000ll);
  const int c = jb.c;
  const int gi = i0 + drow;
  const bool worker = tid < kSliceThreads;
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
  double v[32];
  if (worker) {
    // this thread's 32 sums as FP64 (the final drain ended with wait::st)
    uint32_t h[32], l[32];
    tc::tmem_ld16(tlane + kColHi, h);
    tc::tmem_ld16(tlane + kColHi + 16, h + 16);
    tc::tmem_ld16(tlane + kColLo, l);
    tc::tmem_ld16(tlane + kColLo + 16, l + 16);
    tc::tmem_wait_ld();
#pragma unroll
    for (int q = 0; q < 32; ++q)
      v[q] = stalled ? nanv : (double)__uint_as_float(h[q]) + (double)__uint_as_float(l[q]);
  }
  if (jb.splits == 1) {
    if (worker && gi < c) {
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const int j = j0 + dcol + q;
        if (j < c && gi <= j) write_q(gi, j, v[q]);
      }
    }
  } else {
    // partial tiles as [entry q][thread]: each warp instruction moves 256
    // contiguous bytes (thread tid holds row drow, columns dcol .. dcol + 31)
    double *mine = jb.part + ((int64_t)split * jb.tiles + tile) * (kTM * kTN) + tid;
    if (worker) {
#pragma unroll
      for (int q = 0; q < 32; ++q) __stcg(mine + q * kSliceThreads, v[q]);
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) {
      const unsigned int done = atomicAdd(&jb.counters[tile], 1u);
      if (done == (unsigned int)(jb.splits - 1)) last_s = 1;
    }
    __syncthreads();
    if (last_s && worker) {
      __threadfence();
#pragma unroll
      for (int q = 0; q < 32; ++q) v[q] = 0.0;
      // splits added in order 0, 1, ...; loads of two splits in flight at a time
      const double *src = jb.part + (int64_t)tile * (kTM * kTN) + tid;
      const int64_t sstride = (int64_t)jb.tiles * (kTM * kTN);
      int sp = 0;
      for (; sp + 2 <= jb.splits; sp += 2) {
        double t0[32], t1[32];
#pragma unroll
        for (int q = 0; q < 32; ++q) t0[q] = __ldcg(src + sp * sstride + q * kSliceThreads);
#pragma unroll
        for (int q = 0; q < 32; ++q) t1[q] = __ldcg(src + (sp + 1) * sstride + q * kSliceThreads);
#pragma unroll
        for (int q = 0; q < 32; ++q) v[q] = (v[q] + t0[q]) + t1[q];
      }
      if (sp < jb.splits) {
#pragma unroll
        for (int q = 0; q < 32; ++q) v[q] += __ldcg(src + sp * sstride + q * kSliceThreads);
      }
      if (gi < c) {
#pragma unroll
        for (int q = 0; q < 32; ++q) {
          const int j = j0 + dcol + q;
          if (j < c && gi <= j) write_q(gi, j, v[q]);
        }
      }
      if (tid == 0) jb.counters[tile] = 0u;
    }
  }
  tc::tmem_fence_before();
  __syncthreads();
  tc::tmem_fence_after();
  if (warp == 0) tc::tmem_dealloc(tbase, kTmemCols);
}

__global__ void __launch_bounds__(kTcThreads, 1) gram_tc_kernel_one(const gram_tc_job jb) {
  gram_tc_block(jb, blockIdx.x);
}

// Many problems in one launch: CTA b belongs to the problem p with
// first[p] <= b < first[p + 1] (tiles x splits CTAs each).
__global__ void __launch_bounds__(kTcThreads, 1) gram_tc_kernel_batched(const gram_tc_job *__restrict__ jobs,
                                                                        const int64_t *__restrict__ first, int count) {
  const int64_t bid = blockIdx.x;
  if (bid >= first[count]) return;  // a grid sized by an upper bound
  int lo = 0, hi = count - 1;
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
constexpr int kStatThreads = 512;
__device__ __forceinline__ void colstats_block(const gram_tc_job &jb, int g) {
  __shared__ float smax[kStatThreads / 32];
  __shared__ double ssum[kStatThreads / 32];
  const float *col = tc_col(jb, g);
  float mx = 0.0f;
  dot2 acc;
  // four rows per load where the column is 16-byte aligned (rows before the
  // first aligned one and after the last full group one by one)
  const int64_t head = jb.vec4 ? min(jb.m, (int64_t)((16 - ((uintptr_t)col & 15)) & 15) / 4) : jb.m;
  for (int64_t k = threadIdx.x; k < head; k += kStatThreads) {
    const float a = fabsf(__ldg(col + k));
    mx = fmaxf(mx, a);
    acc.add(a);
  }
  if (jb.vec4) {
    const int64_t nq = (jb.m - head) / 4;
    const float4 *c4 = reinterpret_cast<const float4 *>(col + head);
    for (int64_t k = threadIdx.x; k < nq; k += kStatThreads) {
      const float4 a = __ldg(c4 + k);
      const float v0 = fabsf(a.x), v1 = fabsf(a.y), v2 = fabsf(a.z), v3 = fabsf(a.w);
      mx = fmaxf(fmaxf(mx, fmaxf(v0, v1)), fmaxf(v2, v3));
      acc.add(v0);
      acc.add(v1);
      acc.add(v2);
      acc.add(v3);
    }
    for (int64_t k = head + 4 * nq + threadIdx.x; k < jb.m; k += kStatThreads) {
      const float a = fabsf(__ldg(col + k));
      mx = fmaxf(mx, a);
      acc.add(a);
    }
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
  const int64_t bid = blockIdx.x;
  if (bid >= first[count]) return;  // a grid sized by an upper bound
  int lo = 0, hi = count - 1;
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

gram_tc_job gram_tc_plan(const float *S, int64_t lds, const float *s, int64_t ldt, int nb, int64_t m, int d,
                         int multi, int want_ctas, int64_t max_chunks_per_cta, int min_chunks, int max_splits) {
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
  // the last CTA of a tile adds every split's partial tile: splits are capped
  gram_tc_splits(m, j.tiles, want_ctas, max_chunks_per_cta, min_chunks, max_splits, j.splits, j.chunks_per_split);
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
  gram_tc_job gj = gram_tc_plan(SA, ldsa, Sb, r, 1, r, (int)d, 0, ctx->num_sms, (int64_t)1 << 40,
                                gram_min_chunks(ctx), gram_max_splits(ctx));
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
