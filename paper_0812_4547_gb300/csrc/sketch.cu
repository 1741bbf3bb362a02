// sketch.cu -- the preconditioning step of Alg. 1: SX = H~ D X for the tall
// X = [A | b], where H~ holds the sampled, rescaled rows of the normalised
// Walsh-Hadamard matrix H_n (Sec. 2, Alg. 1 steps 1-4, cost O(nd log r) per
// Sec. 3.4).
//
// Large n (n >= 2^14): H_n = H_C (x) H_m with m = 2^12 and C = n/m, row
// i = h*m + l.  Then (H_n y)[i] = sum_c (-1)^popcount(h & c) (H_m y_c)[l] for
// the chunks y_c of y.  The work is a list of steps, one per column and
// group j of four chunks c = 4j..4j+3 that hold data; a persistent grid of
// one 256-thread block per SM walks equal contiguous stretches of that list:
//   - thread 0 issues tensor copies (cp.async.bulk.tensor, 128-byte swizzle,
//     completion on an mbarrier) of the four chunks of a step and a bulk copy
//     of their sign words, two steps ahead (three stage buffers),
//   - each 64-thread worker flips its chunk's signs with D (words of the sign
//     table the plan launch writes), transforms it with two 64-point register
//     FWHT passes joined by one swizzled transpose, in place in its stage buffer,
//   - and every thread adds, for the sampled rows it owns (the plan, kept in
//     registers or TMEM), the four signed chunk values into per-row sums.
// A column handled by several blocks leaves one partial-sum vector per
// block; the last of them to finish adds them in block order.  HBM sees one
// read of X plus, per split column, a few r-vectors.
//
// Small n (n <= 2^13): one block per column transforms the whole column in
// shared memory and gathers the sampled rows.
#include <cuda.h>  // CUtensorMap and its enums (the encoder is fetched at run time)

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "kernels.h"
#include "launch_attr.h"
#include "tcgen05.cuh"

namespace rnnls {

namespace {

constexpr int kStages = 3;                                   // stage buffers (steps in flight + 1)
constexpr int kStageFloats = kWorkers * kM;                  // one step: four chunks
// stage buffers plus slack to place them at a 1 KiB boundary (the 128-byte
// swizzle repeats every 1 KiB); kept small so that a Gram block (17 KiB) of a
// concurrent solve fits on the same SM
constexpr size_t kSketchSmem = (size_t)kStages * kStageFloats * sizeof(float) + 1024;  // 193 KiB
constexpr uint32_t kSpinLimit = 1u << 22;                    // bounded wait on a bulk copy
// From this many plan rows per thread on, a step's four chunks are first
// transformed into one another (a 16384-point transform per step), so that
// each row reads one word instead of four.
#ifndef RNNLS_FULL_MIN_SLOTS
#define RNNLS_FULL_MIN_SLOTS 48
#endif
constexpr int kFullMinSlots = RNNLS_FULL_MIN_SLOTS;
// From this many plan rows per thread on (in the full-step mode), the
// batched kernel combines steps in pairs (each row reads one word per two
// steps).
#ifndef RNNLS_PAIR_MIN_SLOTS
#define RNNLS_PAIR_MIN_SLOTS 48
#endif
constexpr int kPairMinSlots = RNNLS_PAIR_MIN_SLOTS;

__device__ __forceinline__ void bar_worker(int w) {
  asm volatile("bar.sync %0, 64;" ::"r"(w + 1) : "memory");
}

__device__ __forceinline__ unsigned long long pack2(float a, float b) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void unpack2(unsigned long long r, float &a, float &b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}

// In-register unnormalised Walsh-Hadamard transform of 64 values,
// v[i] <- sum_j (-1)^popcount(i & j) v[j]; strides >= 2 use packed f32x2
// butterflies (same roundings as scalar ones).
__device__ __forceinline__ void fwht64(float (&v)[64]) {
#pragma unroll
  for (int i = 0; i < 64; i += 2) {
    const float a = v[i], b = v[i + 1];
    v[i] = a + b;
    v[i + 1] = a - b;
  }
#pragma unroll
  for (int h = 2; h < 64; h <<= 1) {
#pragma unroll
    for (int i = 0; i < 64; i += 2) {
      if ((i & h) == 0) {
        const unsigned long long x = pack2(v[i], v[i + 1]);
        const unsigned long long y = pack2(v[i + h], v[i + h + 1]);
        unsigned long long su, df;
        asm("add.rn.f32x2 %0, %1, %2;" : "=l"(su) : "l"(x), "l"(y));
        asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(df) : "l"(x), "l"(y));
        unpack2(su, v[i], v[i + 1]);
        unpack2(df, v[i + h], v[i + h + 1]);
      }
    }
  }
}

__device__ __forceinline__ float xor_sign(float v, uint32_t m) { return __int_as_float(__float_as_int(v) ^ (int)m); }

// ---- mbarrier and tensor-copy primitives (PTX) -------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ uint64_t mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  uint64_t state;
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 %0, [%1], %2;" : "=l"(state) : "r"(bar), "r"(bytes) : "memory");
  return state;
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// tiled tensor copy global -> shared of box (32, 128, 1) at (0, y, z); the
// innermost coordinate is 0, so the 16-byte alignment rule always holds
__device__ __forceinline__ void tma_load_chunk(uint32_t dst, const CUtensorMap *map, int y, int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(y), "r"(z), "r"(bar)
      : "memory");
}
// global -> shared bulk copy; dst, src 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
// order this thread's earlier generic-proxy shared accesses before later async-proxy ones
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// the four chunks' words at byte offset `a` of a step's buffer
__device__ __forceinline__ void lds_x4(uint32_t a, float &z0, float &z1, float &z2, float &z3) {
  asm volatile(
      "ld.shared.f32 %0, [%4];\n\tld.shared.f32 %1, [%4+16384];\n\tld.shared.f32 %2, [%4+32768];\n\tld.shared.f32 %3, "
      "[%4+49152];"
      : "=f"(z0), "=f"(z1), "=f"(z2), "=f"(z3)
      : "r"(a));
}

// one word at byte address `a` of shared memory
__device__ __forceinline__ float lds_1(uint32_t a) {
  float z;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(z) : "r"(a));
  return z;
}

// (a, b) <- (a + b, a - b) on four lanes, as two packed f32x2 pairs
__device__ __forceinline__ void bfly4(float4 &a, float4 &b) {
  const unsigned long long a0 = pack2(a.x, a.y), a1 = pack2(a.z, a.w);
  const unsigned long long b0 = pack2(b.x, b.y), b1 = pack2(b.z, b.w);
  unsigned long long s0, s1, d0, d1;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(s0) : "l"(a0), "l"(b0));
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(s1) : "l"(a1), "l"(b1));
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d0) : "l"(a0), "l"(b0));
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d1) : "l"(a1), "l"(b1));
  unpack2(s0, a.x, a.y);
  unpack2(s1, a.z, a.w);
  unpack2(d0, b.x, b.y);
  unpack2(d1, b.z, b.w);
}

// The 4-point transform across a step's four transformed chunks, word by
// word: chunk slot c <- sum_c' (-1)^popcount(c & c') z_c' (the H_4 factor of
// H_16384 = H_4 (x) H_4096; the same word of every chunk holds the same
// position l).  Thread t takes the 16-byte units t, t + 256, ...
__device__ __forceinline__ void cross_chunk_h4(float *__restrict__ st, int tid) {
#pragma unroll
  for (int k = 0; k < kM / (4 * kThreads); ++k) {
    const int o = 4 * (tid + kThreads * k);
    float4 z0 = *reinterpret_cast<const float4 *>(st + o);
    float4 z1 = *reinterpret_cast<const float4 *>(st + kM + o);
    float4 z2 = *reinterpret_cast<const float4 *>(st + 2 * kM + o);
    float4 z3 = *reinterpret_cast<const float4 *>(st + 3 * kM + o);
    bfly4(z0, z1);
    bfly4(z2, z3);
    bfly4(z0, z2);
    bfly4(z1, z3);
    *reinterpret_cast<float4 *>(st + o) = z0;
    *reinterpret_cast<float4 *>(st + kM + o) = z1;
    *reinterpret_cast<float4 *>(st + 2 * kM + o) = z2;
    *reinterpret_cast<float4 *>(st + 3 * kM + o) = z3;
  }
}

// cross_chunk_h4 on a pair's second step (buffer `sb`), then the butterfly
// with the first step's already transformed buffer `fb`, word by word:
// fb <- fb + sb, sb <- fb - sb.
__device__ __forceinline__ void cross_chunk_h4_pair(float *__restrict__ fb, float *__restrict__ sb, int tid) {
#pragma unroll 2
  for (int k = 0; k < kM / (4 * kThreads); ++k) {
    const int o = 4 * (tid + kThreads * k);
    float4 z0 = *reinterpret_cast<const float4 *>(sb + o);
    float4 z1 = *reinterpret_cast<const float4 *>(sb + kM + o);
    float4 z2 = *reinterpret_cast<const float4 *>(sb + 2 * kM + o);
    float4 z3 = *reinterpret_cast<const float4 *>(sb + 3 * kM + o);
    float4 f0 = *reinterpret_cast<const float4 *>(fb + o);
    float4 f1 = *reinterpret_cast<const float4 *>(fb + kM + o);
    float4 f2 = *reinterpret_cast<const float4 *>(fb + 2 * kM + o);
    float4 f3 = *reinterpret_cast<const float4 *>(fb + 3 * kM + o);
    bfly4(z0, z1);
    bfly4(z2, z3);
    bfly4(z0, z2);
    bfly4(z1, z3);
    bfly4(f0, z0);
    bfly4(f1, z1);
    bfly4(f2, z2);
    bfly4(f3, z3);
    *reinterpret_cast<float4 *>(fb + o) = f0;
    *reinterpret_cast<float4 *>(fb + kM + o) = f1;
    *reinterpret_cast<float4 *>(fb + 2 * kM + o) = f2;
    *reinterpret_cast<float4 *>(fb + 3 * kM + o) = f3;
    *reinterpret_cast<float4 *>(sb + o) = z0;
    *reinterpret_cast<float4 *>(sb + kM + o) = z1;
    *reinterpret_cast<float4 *>(sb + 2 * kM + o) = z2;
    *reinterpret_cast<float4 *>(sb + 3 * kM + o) = z3;
  }
}

// ---- tensor memory (TMEM) ----------------------------------------------------
// The block allocates all 512 columns.  Thread (warp w, lane l) owns TMEM lane
// 32 (w % 4) + l, columns (w / 4) * 2 kMaxSlots ...: its plan words first,
// then its row sums (kMaxSlots each), moved eight columns at a time.
__device__ __forceinline__ void tmem_ld8(uint32_t ta, uint32_t *r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(ta)
               : "memory");
}
__device__ __forceinline__ void tmem_st8(uint32_t ta, const uint32_t *r) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(ta), "r"(r[0]),
               "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
               : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
constexpr uint32_t kTmemCols = 512;

// ---- split-precision pass 1 on the tensor cores (RNNLS_PREC_BF16X2) ---------
// H_4096 factors over position bits into H_64 (bits 0-4 and 11) (x) H_64
// (bits 5-10).  In this mode the first factor is a matrix product on the
// tensor cores: each value x (D applied) is carried as hi + lo with
// hi = bf16(x), lo = bf16(x - hi), so |x - hi - lo| <= 2^-18 |x|, and
// (hi + lo) H_64 is formed by tcgen05.mma (H_64's entries +-1 are exact in
// BF16) with FP32 accumulation in TMEM.  The second factor stays a register
// pass in FP32.  A pair of chunks (workers 2p, 2p + 1: 128 threads) is one
// M = 128 tile: row m = 64 (w & 1) + wt holds the thread's 64 pass-1 values
// in K order k = 32 h + e (position (h << 11) | (wt << 5) | e), and column
// n of the product is the transform's output at the position with the same
// bits.  The operands overwrite the pair's 32 KiB of the stage buffer (hi in
// the first chunk's slot, lo in the second's), K-major core matrices of
// 8 rows x 16 bytes, the eight core matrices of an 8-row group adjacent
// (128 bytes apart along K, groups 1 KiB apart); H_64 has its own 8 KiB in
// the same layout.
constexpr int kTcRowSlots = 96;       // rows per thread kept in TMEM beside the accumulators
constexpr uint32_t kTcAccCols = 128;  // two pairs x 64 FP32 columns
constexpr uint32_t kTcIdesc = tc::idesc_bf16_f32(128, 64);

__device__ __forceinline__ void bar_pair(int p) { asm volatile("bar.sync %0, 128;" ::"r"(p + 5) : "memory"); }

// H_64 as the B operand (row n, column k: (-1)^popcount(n & k), BF16 +-1)
__device__ __forceinline__ void init_h64(uint32_t *hm, int tid) {
  for (int i = tid; i < 2048; i += kThreads) {
    const int byte = 4 * i;
    const int n = 8 * (byte >> 10) + ((byte >> 4) & 7);
    const int k = 8 * ((byte >> 7) & 7) + ((byte & 15) >> 1);
    const uint32_t e0 = (__popc(n & k) & 1) ? 0xBF80u : 0x3F80u;
    const uint32_t e1 = (__popc(n & (k + 1)) & 1) ? 0xBF80u : 0x3F80u;
    hm[i] = e0 | (e1 << 16);
  }
  fence_proxy_async();
}

// Pass 1 of the thread's chunk on the tensor cores.  v: its 64 values (D
// applied) in K order; zw: its chunk's slot; pair_u32: the pair's operand
// region (shared address); h_u32: H_64; d_tmem: the pair's accumulator
// (lane 0); t_row: the same columns at this warp's lanes; bar / parity: the
// pair's MMA mbarrier and the phase to wait for.  Writes the 64 outputs back
// to the thread's pass-1 positions.  A wait that runs out sets `stalled`.
__device__ __forceinline__ void tc_pass1(const float (&v)[64], float *zw, uint32_t pair_u32, uint32_t h_u32,
                                         uint32_t d_tmem, uint32_t t_row, uint32_t bar, uint32_t parity, int tid,
                                         int *stalled) {
  const int p = tid >> 7, m = tid & 127, wt = tid & 63;
  uint32_t hi2[32], lo2[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    const float a = v[2 * i], b = v[2 * i + 1];
    uint32_t h, l;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(h) : "f"(b), "f"(a));
    const float ra = a - __uint_as_float(h << 16), rb = b - __uint_as_float(h & 0xffff0000u);
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(l) : "f"(rb), "f"(ra));
    hi2[i] = h;
    lo2[i] = l;
  }
  bar_pair(p);  // every thread of the pair holds its values: the region may be overwritten
  const uint32_t row = pair_u32 + (uint32_t)((m >> 3) * 1024 + (m & 7) * 16);
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(row + 128u * c), "r"(hi2[4 * c]),
                 "r"(hi2[4 * c + 1]), "r"(hi2[4 * c + 2]), "r"(hi2[4 * c + 3])
                 : "memory");
    asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(row + 16384u + 128u * c), "r"(lo2[4 * c]),
                 "r"(lo2[4 * c + 1]), "r"(lo2[4 * c + 2]), "r"(lo2[4 * c + 3])
                 : "memory");
  }
  fence_proxy_async();
  bar_pair(p);
  if (m == 0) {
    tmem_fence_after();
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      const uint64_t bd = tc::smem_desc(h_u32 + 256u * kk, 128, 1024);
      tc::mma_bf16(d_tmem, tc::smem_desc(pair_u32 + 256u * kk, 128, 1024), bd, kTcIdesc, kk > 0 ? 1u : 0u);
      tc::mma_bf16(d_tmem, tc::smem_desc(pair_u32 + 16384u + 256u * kk, 128, 1024), bd, kTcIdesc, 1u);
    }
    tc::mma_commit(bar);
  }
  {
    const uint32_t limit = *(volatile int *)stalled ? 64u : kSpinLimit;
    bool ok = false;
    for (uint32_t it = 0; it < limit && !ok; ++it) ok = mbar_try_wait(bar, parity);
    if (!ok) *(volatile int *)stalled = 1;
  }
  tmem_fence_after();
  uint32_t o[64];
#pragma unroll
  for (int c = 0; c < 4; ++c) tc::tmem_ld16(t_row + 16u * c, o + 16 * c);
  tc::tmem_wait_ld();
  tmem_fence_before();
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int g = 0; g < 8; ++g)
      *reinterpret_cast<float4 *>(zw + ((h << 11) | (wt << 5) | ((g ^ (wt & 7)) << 2))) =
          make_float4(__uint_as_float(o[32 * h + 4 * g]), __uint_as_float(o[32 * h + 4 * g + 1]),
                      __uint_as_float(o[32 * h + 4 * g + 2]), __uint_as_float(o[32 * h + 4 * g + 3]));
}

// Partition of the step list over the blocks.  Unit u = kg * (d + 1) + col
// (plan group kg, column col) owns steps u*J .. u*J + J - 1.  Balanced:
// block b takes steps [T b / B, T (b+1) / B).  Aligned: block b takes the
// whole units [U b / B, U (b+1) / B) (no column is split).
struct srht_part {
  int64_t J;    // chunk groups with data per column: ceil(n_raw / 4m)
  int64_t U;    // units
  int64_t T;    // steps = U * J
  int aligned;
  int full_min;  // rows per thread from which a step's chunks are combined by H_4 first
};

__host__ __device__ __forceinline__ int64_t part_start(int64_t b, int64_t B, const srht_part &P) {
  return P.aligned ? P.J * ((P.U * b) / B) : (P.T * b) / B;
}
// block holding step s (balanced partition)
__host__ __device__ __forceinline__ int64_t part_block_of(int64_t s, int64_t B, const srht_part &P) {
  return ((s + 1) * B - 1) / P.T;
}

// position of a step in the unit list, advanced without divisions
struct step_cursor {
  int64_t u, j, kg;
  int col;
  __device__ void init(int64_t s, const srht_part &P, int64_t D1) {
    u = s / P.J;
    j = s - u * P.J;
    kg = u / D1;
    col = (int)(u - kg * D1);
  }
  __device__ void next(const srht_part &P, int64_t D1) {
    if (++j == P.J) {
      j = 0;
      ++u;
      if (++col == D1) {
        col = 0;
        ++kg;
      }
    }
  }
};

// ---------------------------------------------------------------------------
// The large-n sketch kernel (FP32).  Plan group kg's rows are entries
// [kg][slot][thread] of plan_pk / plan_k (see the plan kernel).
// Columns: d of A, then nb of B (outputs SA, SB).  jg0: full-problem index of
// the first chunk group (row shards; 0 otherwise), which sets the Hadamard
// signs and D's words.  tmA / tmB: column views (32, n_raw / 32, cols) of A
// and B for the tensor copies (vec = 1); with vec = 0 the threads load X with
// plain loads.
// part: [segment][unit][rows_per_group] partial sums of split units;
// counters: one per unit, zero before and after the launch.
//
// Chunk layout in shared memory: position p at word swz128(p) of its 16 KiB
// slot (the tensor copy's 128-byte swizzle).  Pass 1: thread t of a worker
// holds rows t and t + 64 of 32 positions (bits 0-4 and 11 of p in its
// registers); pass 2: lane l, warp h of the worker holds the 64 positions
// with bits 0-4 = l and bit 11 = h.  Both passes read and write back the
// same words, so only pass 2 has to wait for the other threads of the worker.
// ---------------------------------------------------------------------------
template <int SLOTS, bool TC>
__global__ void __launch_bounds__(kThreads, 1)
    sketch_srht_f32(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                    const float *__restrict__ A, int64_t lda, const float *__restrict__ Bm, int64_t ldb,
                    int64_t n_raw, int d, int nb, int64_t jg0, srht_part P, int vec, uint64_t seed, uint64_t inst,
                    const uint64_t *__restrict__ sign_table, const uint32_t *__restrict__ plan_pk,
                    const int32_t *__restrict__ plan_k, int slots, int64_t rpg, float *__restrict__ part,
                    float scale, float *__restrict__ SA, int64_t ldsa, float *__restrict__ SB, int64_t ldsb,
                    unsigned int *__restrict__ counters) {
  extern __shared__ __align__(1024) float dyn_smem[];  // kStages x kWorkers x kM (+ alignment slack)
  __shared__ __align__(16) uint32_t sgn[kStages][kWorkers][kM / 32];  // D's bits, 32-bit halves of the words
  __shared__ __align__(8) uint64_t mbar[kStages];
  __shared__ unsigned int last_flag;
  __shared__ int stalled;  // a tensor copy did not land within the wait limit
  __shared__ uint32_t tmem_base_s;
  __shared__ __align__(1024) uint32_t h64_s[TC ? 2048 : 4];  // H_64 operand (split-precision mode)
  __shared__ __align__(8) uint64_t mma_bar[2];                // one per chunk pair (split-precision mode)

  const int tid = threadIdx.x;
  const int w = tid >> 6;   // worker: chunk 4j + w of a step
  const int wt = tid & 63;  // thread within worker
  const int64_t B = gridDim.x;
  const int64_t bid = blockIdx.x;
  const int64_t s0 = part_start(bid, B, P);
  const int64_t nsteps = part_start(bid + 1, B, P) - s0;
  if (nsteps <= 0) return;
  const int64_t D1 = (int64_t)d + nb;
  // stage buffers at a 1 KiB boundary (the tensor copies' swizzle pattern)
  const uint32_t raw_u32 = smem_u32(dyn_smem);
  const uint32_t stage_u32 = (raw_u32 + 1023u) & ~1023u;
  float *stage = dyn_smem + (stage_u32 - raw_u32) / 4;
  const int64_t nrow32 = n_raw >> 5;  // whole 32-row lines of a column
  const bool full = SLOTS > 0 ? (SLOTS >= kFullMinSlots) : (slots >= P.full_min);

  if (tid == 0) {
    for (int q = 0; q < kStages; ++q) mbar_init(smem_u32(&mbar[q]), 1);
    if constexpr (TC) {
      mbar_init(smem_u32(&mma_bar[0]), 1);
      mbar_init(smem_u32(&mma_bar[1]), 1);
    }
    fence_mbar_init();
    stalled = 0;
  }
  if constexpr (TC) init_h64(h64_s, tid);
  // SLOTS > 0: that many plan rows per thread, words and sums in registers;
  // SLOTS == 0: `slots` rows (a multiple of 8, up to kMaxSlots, kTcRowSlots
  // with TC) kept in TMEM.  TC: the pass-1 accumulators take the last
  // kTcAccCols columns.
  constexpr uint32_t kCols = (SLOTS == 0) ? kTmemCols : kTcAccCols;
  constexpr int kRowCols = TC ? kTcRowSlots : kMaxSlots;
  constexpr uint32_t kAcc0 = (SLOTS == 0) ? kTmemCols - kTcAccCols : 0u;
  if constexpr (SLOTS == 0 || TC) {
    if (tid < 32) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_s)),
                   "r"(kCols)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
  }
  tmem_fence_before();
  __syncthreads();
  tmem_fence_after();
  const uint32_t t_pk = tmem_base_s + ((uint32_t)(32 * ((tid >> 5) & 3)) << 16) + (uint32_t)((tid >> 7) * 2 * kRowCols);
  const uint32_t t_acc = t_pk + kRowCols;
  // TC: this pair's accumulator (lane 0) and its columns at this warp's lanes
  const uint32_t tc_d = tmem_base_s + kAcc0 + 64u * (uint32_t)(tid >> 7);
  const uint32_t tc_row = tc_d + ((uint32_t)(32 * ((tid >> 5) & 3)) << 16);
  const uint32_t tc_pair_off = (uint32_t)(2 * (tid >> 7) * kM) * 4u;  // the pair's bytes in a stage buffer
  uint32_t tc_phase = 0;
  const uint32_t zero8[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
  constexpr int RS = SLOTS > 0 ? SLOTS : 1;
  uint32_t pk_r[RS];
  float acc_r[RS];
#pragma unroll
  for (int e = 0; e < RS; ++e) acc_r[e] = 0.0f;

  // thread 0: tensor copies of one step (4 chunks = 4 boxes of 32 x 128)
  step_cursor ic;
  ic.init(s0, P, D1);
  int iq = 0;
  auto issue = [&](bool with_signs) {
    const uint32_t bar = smem_u32(&mbar[iq]);
    mbar_arrive_expect_tx(bar, (uint32_t)(kWorkers * kM * sizeof(float)) + (sign_table ? 2048u : 0u));
    if (sign_table && with_signs) bulk_g2s(smem_u32(&sgn[iq][0][0]), sign_table + 4 * ic.j * (kM / 64), 2048u, bar);
    const CUtensorMap *map = (ic.col < d) ? &tmA : &tmB;
    const int z = (ic.col < d) ? ic.col : ic.col - d;
#pragma unroll
    for (int c = 0; c < kWorkers; ++c)
      tma_load_chunk(stage_u32 + (uint32_t)(iq * kStageFloats + c * kM) * 4u, map, (int)((4 * ic.j + c) * (kM / 32)),
                     z, bar);
    ic.next(P, D1);
    iq = (iq + 1 == kStages) ? 0 : iq + 1;
  };
  // sign words of this worker's chunk of a step: 64-bit word i of the chunk
  // is Philox block 16c + i/4 (stream 0), word i % 4; stored as 32-bit halves
  // (without tensor copies: from the table with plain loads, or from Philox)
  auto make_signs = [&](int64_t j, int buf) {
    if (sign_table) {
      const uint32_t *src = reinterpret_cast<const uint32_t *>(sign_table + 4 * j * (kM / 64));
      for (int i = tid; i < kWorkers * (kM / 32); i += kThreads) (&sgn[buf][0][0])[i] = src[i];
    } else if (wt < 16) {
      const uint64_t c = (uint64_t)(4 * (j + jg0) + w);
      const u64x4 r4 = philox4x64_10(c * 16u + (uint64_t)wt, kStreamSigns, seed, inst);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        sgn[buf][w][8 * wt + 2 * q] = (uint32_t)r4.w[q];
        sgn[buf][w][8 * wt + 2 * q + 1] = (uint32_t)(r4.w[q] >> 32);
      }
    }
  };

  // The first two steps' data copies need nothing from the plan launch that
  // precedes this one in the stream: launched as its programmatic dependent,
  // this block issues them while that launch finishes, then waits for it
  // (griddepcontrol.wait: the plan, sign table and rows are complete and
  // visible) before the sign words and plan entries are read.
  int64_t j_first[2] = {-1, -1};
  if (vec && tid == 0) {
    j_first[0] = ic.j;
    issue(false);
    if (nsteps > 1) {
      j_first[1] = ic.j;
      issue(false);
    }
  }
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (vec && tid == 0 && sign_table) {
#pragma unroll
    for (int f = 0; f < 2; ++f)
      if (j_first[f] >= 0)
        bulk_g2s(smem_u32(&sgn[f][0][0]), sign_table + 4 * j_first[f] * (kM / 64), 2048u, smem_u32(&mbar[f]));
  }
  step_cursor cur;
  cur.init(s0, P, D1);
  const bool signs_by_copy = vec && sign_table;
  if (!signs_by_copy) make_signs(cur.j, 0);

  int64_t kg_loaded = -1;
  int q = 0;
  uint32_t phase = 0;

  if constexpr (SLOTS >= 24 && !TC) {
    // Pipelined order (24 or more plan rows per thread in registers): the
    // combine of step ls runs beside pass 1 of step ls + 1 (different stage
    // buffers), so each step has one block barrier and the gather's loads
    // overlap the transform's.  With fewer rows the extra registers this
    // order needs cost more than it saves (a concurrent Gram block no longer
    // fits beside the sketch block).
    auto wait_copy = [&](int64_t sidx) {
      if (!vec) return;
      const uint32_t bar = smem_u32(&mbar[sidx % kStages]);
      const uint32_t par = (uint32_t)((sidx / kStages) & 1);
      const uint32_t limit = *(volatile int *)&stalled ? 64u : kSpinLimit;
      bool ok = false;
      for (uint32_t it = 0; it < limit && !ok; ++it) ok = mbar_try_wait(bar, par);
      if (!ok) *(volatile int *)&stalled = 1;
    };
    auto fill = [&](int64_t jj, int cc, float *zw) {
      const float *x = (cc < d) ? A + (int64_t)cc * lda : Bm + (int64_t)(cc - d) * ldb;
      if (!vec) {
        const int64_t row0 = (4 * jj + w) * (int64_t)kM;
#pragma unroll 16
        for (int i = wt; i < kM; i += 64) {
          const int64_t row = row0 + i;
          zw[swz128((uint32_t)i)] = (row < n_raw) ? x[row] : 0.0f;
        }
        bar_worker(w);
      } else {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int64_t line = (4 * jj + w) * (int64_t)(kM / 32) + 64 * h + wt;
          if (line == nrow32) {
#pragma unroll
            for (int e = 0; e < 32; ++e) {
              const int64_t row = 32 * line + e;
              zw[swz128((uint32_t)((h << 11) | (wt << 5) | e))] = (row < n_raw) ? x[row] : 0.0f;
            }
          }
        }
      }
    };
    auto pass1 = [&](float (&v)[64], float *zw, int bq) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint32_t sw = sgn[bq][w][2 * ((h << 5) | (wt >> 1)) + (wt & 1)];
#pragma unroll
        for (int g = 0; g < 8; ++g) {
          const float4 t =
              *reinterpret_cast<const float4 *>(zw + ((h << 11) | (wt << 5) | ((g ^ (wt & 7)) << 2)));
          v[32 * h + 4 * g + 0] = xor_sign(t.x, (sw << (31 - (4 * g + 0))) & 0x80000000u);
          v[32 * h + 4 * g + 1] = xor_sign(t.y, (sw << (31 - (4 * g + 1))) & 0x80000000u);
          v[32 * h + 4 * g + 2] = xor_sign(t.z, (sw << (31 - (4 * g + 2))) & 0x80000000u);
          v[32 * h + 4 * g + 3] = xor_sign(t.w, (sw << (31 - (4 * g + 3))) & 0x80000000u);
        }
      }
      fwht64(v);
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int g = 0; g < 8; ++g)
          *reinterpret_cast<float4 *>(zw + ((h << 11) | (wt << 5) | ((g ^ (wt & 7)) << 2))) =
              make_float4(v[32 * h + 4 * g], v[32 * h + 4 * g + 1], v[32 * h + 4 * g + 2], v[32 * h + 4 * g + 3]);
    };
    auto pass2 = [&](float (&v)[64], float *zw) {
      const uint32_t lane = (uint32_t)(wt & 31), hi = (uint32_t)(wt >> 5) << 11;
#pragma unroll
      for (int s2 = 0; s2 < 64; ++s2) v[s2] = zw[hi | ((uint32_t)s2 << 5) | (lane ^ (((uint32_t)s2 & 7u) << 2))];
      fwht64(v);
#pragma unroll
      for (int s2 = 0; s2 < 64; ++s2) zw[hi | ((uint32_t)s2 << 5) | (lane ^ (((uint32_t)s2 & 7u) << 2))] = v[s2];
    };
    step_cursor tc = cur;  // the step being transformed (one ahead of `cur`)
    {
      wait_copy(0);
      float *zw = stage + w * kM;
      fill(tc.j, tc.col, zw);
      float v[64];
      pass1(v, zw, 0);
      bar_worker(w);
      pass2(v, zw);
      tc.next(P, D1);
    }
    if (!signs_by_copy && nsteps > 1) make_signs(tc.j, 1);
    for (int64_t ls = 0; ls < nsteps; ++ls) {
      const int64_t j = cur.j;
      const int col = cur.col;
      const int bq = (int)(ls % kStages);
      __syncthreads();  // step ls transformed; step ls-1 combined (its buffer is free); next signs visible
      if (vec && tid == 0 && ls + 2 < nsteps) {
        fence_proxy_async();
        issue(true);
      }
      if (cur.kg != kg_loaded) {  // this plan group's words (row sums are zero here)
#pragma unroll
        for (int e = 0; e < SLOTS; ++e) pk_r[e] = plan_pk[((size_t)cur.kg * SLOTS + e) * kThreads + tid];
        kg_loaded = cur.kg;
      }
      const bool more = ls + 1 < nsteps;
      const int bn = (int)((ls + 1) % kStages);
      float *zn = stage + bn * kStageFloats + w * kM;
      float v[64];
      if (more) {
        wait_copy(ls + 1);
        fill(tc.j, tc.col, zn);
        pass1(v, zn, bn);
      }
      {
        const uint32_t step_u32 = stage_u32 + (uint32_t)(bq * kStageFloats) * 4u;
        const uint32_t jm = (uint32_t)(j + jg0) << 16;
#pragma unroll
        for (int e = 0; e < SLOTS; ++e) {
          const uint32_t p = pk_r[e];
          float z0, z1, z2, z3;
          lds_x4(step_u32 + (p & 0x3ffcu), z0, z1, z2, z3);
          const float s1 = __int_as_float((int)((p & 0x80000000u) | 0x3f800000u));
          const float s2 = __int_as_float((int)(((p << 1) & 0x80000000u) | 0x3f800000u));
          const float t = fmaf(s2, fmaf(s1, z3, z2), fmaf(s1, z1, z0));
          acc_r[e] += xor_sign(t, (uint32_t)__popc(p & jm) << 31);
        }
      }
      cur.next(P, D1);
    // end of this block's part of unit u: write or hand over the sums
      if (j == P.J - 1 || ls == nsteps - 1) {
        const int64_t u = cur.u - ((j == P.J - 1) ? 1 : 0);  // cursor already moved on
        const int64_t kg = kg_loaded;
        const bool poisoned = *(volatile int *)&stalled != 0;
        int64_t first = bid, last = bid;
        if (!P.aligned) {
          first = part_block_of(u * P.J, B, P);
          last = part_block_of(u * P.J + P.J - 1, B, P);
        }
        const int64_t nseg = last - first + 1;
        const int64_t seg = bid - first;
        const int nsl = SLOTS > 0 ? SLOTS : slots;
        if constexpr (SLOTS > 0) {
          if (nseg == 1) {
#pragma unroll
            for (int e = 0; e < RS; ++e) {
              const int32_t k = plan_k[((size_t)kg * SLOTS + e) * kThreads + tid];
              if (k < 0) continue;
              const float val = poisoned ? __int_as_float(0x7fc00000) : scale * acc_r[e];
              if (col < d)
                SA[(int64_t)col * ldsa + k] = val;
              else
                SB[(int64_t)(col - d) * ldsb + k] = val;
            }
          } else {
#pragma unroll
            for (int e = 0; e < RS; ++e) {
              const int32_t k = plan_k[((size_t)kg * SLOTS + e) * kThreads + tid];
              if (k < 0) continue;
              part[((size_t)seg * P.U + u) * rpg + (size_t)e * kThreads + tid] =
                  poisoned ? __int_as_float(0x7fc00000) : acc_r[e];
            }
          }
#pragma unroll
          for (int e = 0; e < RS; ++e) acc_r[e] = 0.0f;
        } else {
          tmem_wait_st();
          // 32 rows at a time: their indices and sums are fetched together
          for (int s32 = 0; s32 < slots; s32 += 32) {
            const int n8 = min(4, (slots - s32) >> 3);
            int32_t kk[32];
            uint32_t acc[32];
#pragma unroll
            for (int e = 0; e < 32; ++e)
              kk[e] = (e < 8 * n8) ? plan_k[((size_t)kg * slots + s32 + e) * kThreads + tid] : -1;
#pragma unroll
            for (int b8 = 0; b8 < 4; ++b8)
              if (b8 < n8) tmem_ld8(t_acc + s32 + 8 * b8, acc + 8 * b8);
            tmem_wait_ld();
#pragma unroll
            for (int e = 0; e < 32; ++e) {
              if (kk[e] < 0) continue;
              const float a = poisoned ? __int_as_float(0x7fc00000) : __uint_as_float(acc[e]);
              if (nseg == 1) {
                if (col < d)
                  SA[(int64_t)col * ldsa + kk[e]] = scale * a;
                else
                  SB[(int64_t)(col - d) * ldsb + kk[e]] = scale * a;
              } else {
                part[((size_t)seg * P.U + u) * rpg + (size_t)(s32 + e) * kThreads + tid] = a;
              }
            }
#pragma unroll
            for (int b8 = 0; b8 < 4; ++b8)
              if (b8 < n8) tmem_st8(t_acc + s32 + 8 * b8, zero8);
          }
        }
        if (nseg > 1) {
          __threadfence();
          __syncthreads();
          if (tid == 0) last_flag = (atomicAdd(&counters[u], 1u) == (unsigned int)(nseg - 1)) ? 1u : 0u;
          __syncthreads();
          if (last_flag) {
            __threadfence();
            // every row's segment loads in flight together (register variants),
            // or 32 rows at a time (TMEM variant)
            constexpr int RB = SLOTS > 0 ? SLOTS : 32;
            for (int s0b = 0; s0b < nsl; s0b += RB) {
              int32_t kk[RB];
              float sum[RB];
#pragma unroll
              for (int e = 0; e < RB; ++e) {
                kk[e] = (s0b + e < nsl) ? plan_k[((size_t)kg * slots + s0b + e) * kThreads + tid] : -1;
                sum[e] = 0.0f;
              }
              for (int64_t g = 0; g < nseg; ++g) {
                const float *pg = part + ((size_t)g * P.U + u) * rpg + (size_t)s0b * kThreads + tid;
                float t[RB];
#pragma unroll
                for (int e = 0; e < RB; ++e) t[e] = (kk[e] >= 0) ? __ldcg(pg + (size_t)e * kThreads) : 0.0f;
#pragma unroll
                for (int e = 0; e < RB; ++e) sum[e] += t[e];
              }
#pragma unroll
              for (int e = 0; e < RB; ++e) {
                if (kk[e] < 0) continue;
                if (col < d)
                  SA[(int64_t)col * ldsa + kk[e]] = scale * sum[e];
                else
                  SB[(int64_t)(col - d) * ldsb + kk[e]] = scale * sum[e];
              }
            }
            if (tid == 0) counters[u] = 0u;
          }
        }
      }

      if (more) {
        bar_worker(w);
        pass2(v, zn);
        tc.next(P, D1);
      }
      if (!signs_by_copy && ls + 2 < nsteps) make_signs(tc.j, (int)((ls + 2) % kStages));
    }
    return;
  }

  for (int64_t ls = 0; ls < nsteps; ++ls) {
    const int64_t j = cur.j;
    const int col = cur.col;
    if (cur.kg != kg_loaded) {  // this plan group's words (row sums are zero here)
      if constexpr (SLOTS > 0) {
#pragma unroll
        for (int e = 0; e < SLOTS; ++e) pk_r[e] = plan_pk[((size_t)cur.kg * SLOTS + e) * kThreads + tid];
      } else {
        tmem_wait_st();
        for (int s8 = 0; s8 < slots; s8 += 8) {
          uint32_t r8[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) r8[e] = plan_pk[((size_t)cur.kg * slots + s8 + e) * kThreads + tid];
          tmem_st8(t_pk + s8, r8);
          tmem_st8(t_acc + s8, zero8);
        }
      }
      kg_loaded = cur.kg;
    }
    float *__restrict__ zw = stage + q * kStageFloats + w * kM;
    const uint32_t step_u32 = stage_u32 + (uint32_t)(q * kStageFloats) * 4u;
    __syncthreads();  // step ls-1 is done with its buffer; this step's signs are visible
    if (vec) {
      if (tid == 0 && ls + 2 < nsteps) {
        fence_proxy_async();
        issue(true);
      }
      const uint32_t bar = smem_u32(&mbar[q]);
      const uint32_t limit = *(volatile int *)&stalled ? 64u : kSpinLimit;
      bool ok = false;
      for (uint32_t it = 0; it < limit && !ok; ++it) ok = mbar_try_wait(bar, phase);
      if (!ok) *(volatile int *)&stalled = 1;
    }
    {
      const float *x = (col < d) ? A + (int64_t)col * lda : Bm + (int64_t)(col - d) * ldb;
      if (!vec) {
        // no tensor copies: the worker loads its chunk with coalesced plain loads
        const int64_t row0 = (4 * j + w) * (int64_t)kM;
#pragma unroll 16
        for (int i = wt; i < kM; i += 64) {
          const int64_t row = row0 + i;
          zw[swz128((uint32_t)i)] = (row < n_raw) ? x[row] : 0.0f;
        }
        bar_worker(w);
      } else {
        // the partial last line of a column (the copy filled it with zeros)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int64_t line = (4 * j + w) * (int64_t)(kM / 32) + 64 * h + wt;
          if (line == nrow32) {
#pragma unroll
            for (int e = 0; e < 32; ++e) {
              const int64_t row = 32 * line + e;
              zw[swz128((uint32_t)((h << 11) | (wt << 5) | e))] = (row < n_raw) ? x[row] : 0.0f;
            }
          }
        }
      }
    }

    // pass 1 (bits 0-4, 11): v[32 h + 4 g + e] <- position (h<<11)|(wt<<5)|(4g+e), D applied
    float v[64];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint32_t sw = sgn[q][w][2 * ((h << 5) | (wt >> 1)) + (wt & 1)];
#pragma unroll
      for (int g = 0; g < 8; ++g) {
        const float4 t =
            *reinterpret_cast<const float4 *>(zw + ((h << 11) | (wt << 5) | ((g ^ (wt & 7)) << 2)));
        v[32 * h + 4 * g + 0] = xor_sign(t.x, (sw << (31 - (4 * g + 0))) & 0x80000000u);
        v[32 * h + 4 * g + 1] = xor_sign(t.y, (sw << (31 - (4 * g + 1))) & 0x80000000u);
        v[32 * h + 4 * g + 2] = xor_sign(t.z, (sw << (31 - (4 * g + 2))) & 0x80000000u);
        v[32 * h + 4 * g + 3] = xor_sign(t.w, (sw << (31 - (4 * g + 3))) & 0x80000000u);
      }
    }
    if constexpr (TC) {
      tc_pass1(v, zw, stage_u32 + (uint32_t)(q * kStageFloats) * 4u + tc_pair_off, smem_u32(h64_s), tc_d, tc_row,
               smem_u32(&mma_bar[tid >> 7]), tc_phase, tid, &stalled);
      tc_phase ^= 1u;
    } else {
      fwht64(v);
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int g = 0; g < 8; ++g)
          *reinterpret_cast<float4 *>(zw + ((h << 11) | (wt << 5) | ((g ^ (wt & 7)) << 2))) =
              make_float4(v[32 * h + 4 * g], v[32 * h + 4 * g + 1], v[32 * h + 4 * g + 2], v[32 * h + 4 * g + 3]);
    }
    bar_worker(w);
    // pass 2 (bits 5-10): v[s] <- position ((wt>>5)<<11) | (s<<5) | (wt & 31)
    {
      const uint32_t lane = (uint32_t)(wt & 31), hi = (uint32_t)(wt >> 5) << 11;
#pragma unroll
      for (int s = 0; s < 64; ++s) v[s] = zw[hi | ((uint32_t)s << 5) | (lane ^ (((uint32_t)s & 7u) << 2))];
      fwht64(v);
#pragma unroll
      for (int s = 0; s < 64; ++s) zw[hi | ((uint32_t)s << 5) | (lane ^ (((uint32_t)s & 7u) << 2))] = v[s];
    }
    __syncthreads();  // the four transformed chunks are ready
    if (full) {       // ... and transformed into one another
      cross_chunk_h4(stage + q * kStageFloats, tid);
      __syncthreads();
    }

    // combine: row (hq, c1, c2) adds (-1)^popcount(hq & j) (z0 + s1 z1 + s2 (z2 + s1 z3))[l]
    // (full: the word of l in chunk slot h & 3), eight rows at a time (plan words and sums
    // move between TMEM and registers)
    const uint32_t jm = (uint32_t)(j + jg0) << 16;
    if constexpr (SLOTS > 0) {
      if constexpr (SLOTS >= kFullMinSlots) {
#pragma unroll
        for (int e = 0; e < SLOTS; ++e) {
          const uint32_t p = pk_r[e];
          acc_r[e] += xor_sign(lds_1(step_u32 + (p & 0xfffcu)), (uint32_t)__popc(p & jm) << 31);
        }
      } else {
#pragma unroll
        for (int e = 0; e < SLOTS; ++e) {
          const uint32_t p = pk_r[e];
          float z0, z1, z2, z3;
          lds_x4(step_u32 + (p & 0x3ffcu), z0, z1, z2, z3);
          const float s1 = __int_as_float((int)((p & 0x80000000u) | 0x3f800000u));
          const float s2 = __int_as_float((int)(((p << 1) & 0x80000000u) | 0x3f800000u));
          const float t = fmaf(s2, fmaf(s1, z3, z2), fmaf(s1, z1, z0));
          acc_r[e] += xor_sign(t, (uint32_t)__popc(p & jm) << 31);
        }
      }
    } else {
      // batch k+1 is loaded from TMEM while batch k is combined
      uint32_t pk[8], acc[8], pkn[8], accn[8];
      tmem_wait_st();
      tmem_ld8(t_pk, pk);
      tmem_ld8(t_acc, acc);
      tmem_wait_ld();
      for (int s8 = 0; s8 < slots; s8 += 8) {
        const bool more = s8 + 8 < slots;
        if (more) {
          tmem_ld8(t_pk + s8 + 8, pkn);
          tmem_ld8(t_acc + s8 + 8, accn);
        }
        if (full) {
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const uint32_t p = pk[e];
            const float y = lds_1(step_u32 + (p & 0xfffcu));
            acc[e] = __float_as_uint(__uint_as_float(acc[e]) + xor_sign(y, (uint32_t)__popc(p & jm) << 31));
          }
        } else {
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const uint32_t p = pk[e];
            float z0, z1, z2, z3;
            lds_x4(step_u32 + (p & 0x3ffcu), z0, z1, z2, z3);
            const float s1 = __int_as_float((int)((p & 0x80000000u) | 0x3f800000u));
            const float s2 = __int_as_float((int)(((p << 1) & 0x80000000u) | 0x3f800000u));
            const float t = fmaf(s2, fmaf(s1, z3, z2), fmaf(s1, z1, z0));
            acc[e] = __float_as_uint(__uint_as_float(acc[e]) + xor_sign(t, (uint32_t)__popc(p & jm) << 31));
          }
        }
        tmem_st8(t_acc + s8, acc);
        if (more) {
          tmem_wait_ld();
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            pk[e] = pkn[e];
            acc[e] = accn[e];
          }
        }
      }
    }
    cur.next(P, D1);
    if (++q == kStages) {
      q = 0;
      phase ^= 1u;
    }
    if (!signs_by_copy && ls + 1 < nsteps) make_signs(cur.j, q);

    // end of this block's part of unit u: write or hand over the sums
    if (j == P.J - 1 || ls == nsteps - 1) {
      const int64_t u = cur.u - ((j == P.J - 1) ? 1 : 0);  // cursor already moved on
      const int64_t kg = kg_loaded;
      const bool poisoned = *(volatile int *)&stalled != 0;
      int64_t first = bid, last = bid;
      if (!P.aligned) {
        first = part_block_of(u * P.J, B, P);
        last = part_block_of(u * P.J + P.J - 1, B, P);
      }
      const int64_t nseg = last - first + 1;
      const int64_t seg = bid - first;
      const int nsl = SLOTS > 0 ? SLOTS : slots;
      if constexpr (SLOTS > 0) {
        if (nseg == 1) {
#pragma unroll
          for (int e = 0; e < RS; ++e) {
            const int32_t k = plan_k[((size_t)kg * SLOTS + e) * kThreads + tid];
            if (k < 0) continue;
            const float val = poisoned ? __int_as_float(0x7fc00000) : scale * acc_r[e];
            if (col < d)
              SA[(int64_t)col * ldsa + k] = val;
            else
              SB[(int64_t)(col - d) * ldsb + k] = val;
          }
        } else {
#pragma unroll
          for (int e = 0; e < RS; ++e) {
            const int32_t k = plan_k[((size_t)kg * SLOTS + e) * kThreads + tid];
            if (k < 0) continue;
            part[((size_t)seg * P.U + u) * rpg + (size_t)e * kThreads + tid] =
                poisoned ? __int_as_float(0x7fc00000) : acc_r[e];
          }
        }
#pragma unroll
        for (int e = 0; e < RS; ++e) acc_r[e] = 0.0f;
      } else {
        tmem_wait_st();
        // 32 rows at a time: their indices and sums are fetched together
        for (int s32 = 0; s32 < slots; s32 += 32) {
          const int n8 = min(4, (slots - s32) >> 3);
          int32_t kk[32];
          uint32_t acc[32];
#pragma unroll
          for (int e = 0; e < 32; ++e)
            kk[e] = (e < 8 * n8) ? plan_k[((size_t)kg * slots + s32 + e) * kThreads + tid] : -1;
#pragma unroll
          for (int b8 = 0; b8 < 4; ++b8)
            if (b8 < n8) tmem_ld8(t_acc + s32 + 8 * b8, acc + 8 * b8);
          tmem_wait_ld();
#pragma unroll
          for (int e = 0; e < 32; ++e) {
            if (kk[e] < 0) continue;
            const float a = poisoned ? __int_as_float(0x7fc00000) : __uint_as_float(acc[e]);
            if (nseg == 1) {
              if (col < d)
                SA[(int64_t)col * ldsa + kk[e]] = scale * a;
              else
                SB[(int64_t)(col - d) * ldsb + kk[e]] = scale * a;
            } else {
              part[((size_t)seg * P.U + u) * rpg + (size_t)(s32 + e) * kThreads + tid] = a;
            }
          }
#pragma unroll
          for (int b8 = 0; b8 < 4; ++b8)
            if (b8 < n8) tmem_st8(t_acc + s32 + 8 * b8, zero8);
        }
      }
      if (nseg > 1) {
        __threadfence();
        __syncthreads();
        if (tid == 0) last_flag = (atomicAdd(&counters[u], 1u) == (unsigned int)(nseg - 1)) ? 1u : 0u;
        __syncthreads();
        if (last_flag) {
          __threadfence();
          // every row's segment loads in flight together (register variants),
          // or 32 rows at a time (TMEM variant)
          constexpr int RB = SLOTS > 0 ? SLOTS : 32;
          for (int s0b = 0; s0b < nsl; s0b += RB) {
            int32_t kk[RB];
            float sum[RB];
#pragma unroll
            for (int e = 0; e < RB; ++e) {
              kk[e] = (s0b + e < nsl) ? plan_k[((size_t)kg * slots + s0b + e) * kThreads + tid] : -1;
              sum[e] = 0.0f;
            }
            for (int64_t g = 0; g < nseg; ++g) {
              const float *pg = part + ((size_t)g * P.U + u) * rpg + (size_t)s0b * kThreads + tid;
              float t[RB];
#pragma unroll
              for (int e = 0; e < RB; ++e) t[e] = (kk[e] >= 0) ? __ldcg(pg + (size_t)e * kThreads) : 0.0f;
#pragma unroll
              for (int e = 0; e < RB; ++e) sum[e] += t[e];
            }
#pragma unroll
            for (int e = 0; e < RB; ++e) {
              if (kk[e] < 0) continue;
              if (col < d)
                SA[(int64_t)col * ldsa + kk[e]] = scale * sum[e];
              else
                SB[(int64_t)(col - d) * ldsb + kk[e]] = scale * sum[e];
            }
          }
          if (tid == 0) counters[u] = 0u;
        }
      }
    }
  }
  if constexpr (SLOTS == 0 || TC) {
    tmem_wait_st();
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (tid < 32)
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base_s), "r"(kCols)
                   : "memory");
  }
}

// ---------------------------------------------------------------------------
// Many instances in one launch (iid rows, one target each).  The step list
// is the concatenation of the instances' step lists (instance i owns global
// steps step0 .. step0 + T - 1, its units ordered as in the one-instance
// kernel); blocks take balanced stretches of it.  Plan words and row sums
// live in TMEM (a runtime number of rows per thread, the instance's).  A
// unit split between blocks is finished through the partial-sum slots of
// the block where it starts (at most one such unit per block boundary).
// Tensor maps are read from the job table in global memory, after a
// tensormap acquire fence per instance.
// ---------------------------------------------------------------------------
struct srht_job {  // 64-byte aligned through its tensor maps
  CUtensorMap tmA, tmB;
  const float *A, *B;
  const uint64_t *signs;
  const uint32_t *pk;
  const int32_t *pkk;
  float *SA, *SB;
  int64_t lda, ldb, ldsa, ldsb, n_raw, J, U, step0, rpg;
  float scale;
  int d, slots, vec, r, full_min;
};

__device__ __forceinline__ void fence_tensormap_acquire(const void *map) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(map))
               : "memory");
}

// instance holding global step s
__device__ __forceinline__ int job_of_step(const srht_job *__restrict__ jobs, int njobs, int64_t s) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].step0 <= s)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// block whose step range [starts[b], starts[b+1]) holds step s (empty ranges skipped)
__host__ __device__ __forceinline__ int64_t block_of_step(const int64_t *starts, int64_t B, int64_t s) {
  int64_t lo = 0, hi = B - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (starts[mid] <= s)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// position (instance, unit u, group j, column, plan group) of a global step
struct batch_cursor {
  int ji;
  int64_t u, j, kg;
  int col;
  __device__ void init(const srht_job *__restrict__ jobs, int njobs, int64_t s) {
    ji = job_of_step(jobs, njobs, s);
    const srht_job &J0 = jobs[ji];
    const int64_t ls = s - J0.step0;
    u = ls / J0.J;
    j = ls - u * J0.J;
    kg = u / (J0.d + 1);
    col = (int)(u - kg * (J0.d + 1));
  }
  __device__ void next(const srht_job *__restrict__ jobs, int njobs) {
    const srht_job &J0 = jobs[ji];
    if (++j < J0.J) return;
    j = 0;
    if (++u < J0.U) {
      if (++col == J0.d + 1) {
        col = 0;
        ++kg;
      }
      return;
    }
    if (ji + 1 < njobs) ++ji;
    u = 0;
    kg = 0;
    col = 0;
  }
};

template <bool TC>
__global__ void __launch_bounds__(kThreads, 1)
    sketch_srht_batch_f32(const srht_job *__restrict__ jobs, int njobs, const int64_t *__restrict__ starts,
                          float *__restrict__ part, int maxseg, int64_t rpg_max, unsigned int *__restrict__ counters) {
  extern __shared__ __align__(1024) float dyn_smem[];
  __shared__ __align__(16) uint32_t sgn[kStages][kWorkers][kM / 32];
  __shared__ __align__(8) uint64_t mbar[kStages];
  __shared__ unsigned int last_flag;
  __shared__ int stalled;
  __shared__ uint32_t tmem_base_s;
  __shared__ __align__(1024) uint32_t h64_s[TC ? 2048 : 4];  // H_64 operand (split-precision mode)
  __shared__ __align__(8) uint64_t mma_bar[2];

  const int tid = threadIdx.x;
  const int w = tid >> 6;
  const int wt = tid & 63;
  const int64_t B = gridDim.x;
  const int64_t bid = blockIdx.x;
  const int64_t s0 = starts[bid];
  const int64_t nsteps = starts[bid + 1] - s0;
  if (nsteps <= 0) return;
  const uint32_t raw_u32 = smem_u32(dyn_smem);
  const uint32_t stage_u32 = (raw_u32 + 1023u) & ~1023u;
  float *stage = dyn_smem + (stage_u32 - raw_u32) / 4;

  if (tid == 0) {
    for (int q = 0; q < kStages; ++q) mbar_init(smem_u32(&mbar[q]), 1);
    if constexpr (TC) {
      mbar_init(smem_u32(&mma_bar[0]), 1);
      mbar_init(smem_u32(&mma_bar[1]), 1);
    }
    fence_mbar_init();
    stalled = 0;
  }
  if constexpr (TC) init_h64(h64_s, tid);
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_s)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tmem_fence_before();
  __syncthreads();
  tmem_fence_after();
  constexpr int kRowCols = TC ? kTcRowSlots : kMaxSlots;  // TC: the last kTcAccCols columns hold pass 1's products
  const uint32_t t_pk = tmem_base_s + ((uint32_t)(32 * ((tid >> 5) & 3)) << 16) + (uint32_t)((tid >> 7) * 2 * kRowCols);
  const uint32_t t_acc = t_pk + kRowCols;
  const uint32_t tc_d = tmem_base_s + (kTmemCols - kTcAccCols) + 64u * (uint32_t)(tid >> 7);
  const uint32_t tc_row = tc_d + ((uint32_t)(32 * ((tid >> 5) & 3)) << 16);
  const uint32_t tc_pair_off = (uint32_t)(2 * (tid >> 7) * kM) * 4u;
  uint32_t tc_phase = 0;
  const uint32_t zero8[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};

  // thread 0: copies of a step (four chunks and their sign words)
  batch_cursor ic;
  ic.init(jobs, njobs, s0);
  int iq = 0;
  int fenced = -1;
  auto issue = [&]() {
    const srht_job &J0 = jobs[ic.ji];
    const uint32_t bar = smem_u32(&mbar[iq]);
    if (!J0.vec) {
      mbar_arrive_expect_tx(bar, 0u);
    } else {
      if (fenced != ic.ji) {
        fence_tensormap_acquire(&J0.tmA);
        fence_tensormap_acquire(&J0.tmB);
        fenced = ic.ji;
      }
      mbar_arrive_expect_tx(bar, (uint32_t)(kWorkers * kM * sizeof(float)) + 2048u);
      bulk_g2s(smem_u32(&sgn[iq][0][0]), J0.signs + 4 * ic.j * (kM / 64), 2048u, bar);
      const CUtensorMap *map = (ic.col < J0.d) ? &J0.tmA : &J0.tmB;
      const int z = (ic.col < J0.d) ? ic.col : 0;
#pragma unroll
      for (int c = 0; c < kWorkers; ++c)
        tma_load_chunk(stage_u32 + (uint32_t)(iq * kStageFloats + c * kM) * 4u, map,
                       (int)((4 * ic.j + c) * (kM / 32)), z, bar);
    }
    ic.next(jobs, njobs);
    iq = (iq + 1 == kStages) ? 0 : iq + 1;
  };
  // thread 0 keeps up to kStages steps loaded or in flight ahead of the
  // last step whose buffer is free (`consumed`; a pair's first step is freed
  // with its second)
  int64_t n_issued = 0, consumed = 0;
  if (tid == 0) {
    issue();
    n_issued = 1;
    if (nsteps > 1) {
      issue();
      n_issued = 2;
    }
  }

  batch_cursor cur;
  cur.init(jobs, njobs, s0);
  int loaded_ji = -1;
  int64_t loaded_kg = -1;
  int q = 0;
  uint32_t phase = 0;
  int pair_q = -1;  // buffer of the pending first step of a step pair, or -1
  for (int64_t ls = 0; ls < nsteps; ++ls) {
    const int ji = cur.ji;
    const int64_t j = cur.j, u = cur.u, kg = cur.kg;
    const int col = cur.col;
    const srht_job &J0 = jobs[ji];
    const int d = J0.d;
    const int slots = J0.slots;
    float *__restrict__ zw = stage + q * kStageFloats + w * kM;
    const uint32_t step_u32 = stage_u32 + (uint32_t)(q * kStageFloats) * 4u;
    if (ji != loaded_ji || kg != loaded_kg) {  // this instance's plan group into TMEM, sums cleared
      tmem_wait_st();
      for (int s8 = 0; s8 < slots; s8 += 8) {
        uint32_t r8[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) r8[e] = J0.pk[((size_t)kg * slots + s8 + e) * kThreads + tid];
        tmem_st8(t_pk + s8, r8);
        tmem_st8(t_acc + s8, zero8);
      }
      loaded_ji = ji;
      loaded_kg = kg;
    }
    __syncthreads();  // the steps before `consumed` are done with their buffers
    if (tid == 0 && n_issued < nsteps && n_issued < consumed + kStages) {
      fence_proxy_async();
      do {
        issue();
        ++n_issued;
      } while (n_issued < nsteps && n_issued < consumed + kStages);
    }
    {
      const uint32_t bar = smem_u32(&mbar[q]);
      const uint32_t limit = *(volatile int *)&stalled ? 64u : kSpinLimit;
      bool ok = false;
      for (uint32_t it = 0; it < limit && !ok; ++it) ok = mbar_try_wait(bar, phase);
      if (!ok) *(volatile int *)&stalled = 1;
    }
    const int vec = J0.vec;
    const int64_t n_raw = J0.n_raw;
    const int64_t nrow32 = n_raw >> 5;
    {
      const float *x = (col < d) ? J0.A + (int64_t)col * J0.lda : J0.B;
      if (!vec) {
        const int64_t row0 = (4 * j + w) * (int64_t)kM;
#pragma unroll 16
        for (int i = wt; i < kM; i += 64) {
          const int64_t row = row0 + i;
          zw[swz128((uint32_t)i)] = (row < n_raw) ? x[row] : 0.0f;
        }
        bar_worker(w);
      } else {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int64_t line = (4 * j + w) * (int64_t)(kM / 32) + 64 * h + wt;
          if (line == nrow32) {
#pragma unroll
            for (int e = 0; e < 32; ++e) {
              const int64_t row = 32 * line + e;
              zw[swz128((uint32_t)((h << 11) | (wt << 5) | e))] = (row < n_raw) ? x[row] : 0.0f;
            }
          }
        }
      }
    }
    uint32_t swv[2];
    if (vec) {
#pragma unroll
      for (int h = 0; h < 2; ++h) swv[h] = sgn[q][w][2 * ((h << 5) | (wt >> 1)) + (wt & 1)];
    } else {
      const uint32_t *t32 = reinterpret_cast<const uint32_t *>(J0.signs + (4 * j + w) * (kM / 64));
#pragma unroll
      for (int h = 0; h < 2; ++h) swv[h] = t32[2 * ((h << 5) | (wt >> 1)) + (wt & 1)];
    }
    float v[64];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint32_t sw = swv[h];
#pragma unroll
      for (int g = 0; g < 8; ++g) {
        const float4 t =
            *reinterpret_cast<const float4 *>(zw + ((h << 11) | (wt << 5) | ((g ^ (wt & 7)) << 2)));
        v[32 * h + 4 * g + 0] = xor_sign(t.x, (sw << (31 - (4 * g + 0))) & 0x80000000u);
        v[32 * h + 4 * g + 1] = xor_sign(t.y, (sw << (31 - (4 * g + 1))) & 0x80000000u);
        v[32 * h + 4 * g + 2] = xor_sign(t.z, (sw << (31 - (4 * g + 2))) & 0x80000000u);
        v[32 * h + 4 * g + 3] = xor_sign(t.w, (sw << (31 - (4 * g + 3))) & 0x80000000u);
      }
    }
    if constexpr (TC) {
      tc_pass1(v, zw, step_u32 + tc_pair_off, smem_u32(h64_s), tc_d, tc_row, smem_u32(&mma_bar[tid >> 7]), tc_phase,
               tid, &stalled);
      tc_phase ^= 1u;
    } else {
      fwht64(v);
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int g = 0; g < 8; ++g)
          *reinterpret_cast<float4 *>(zw + ((h << 11) | (wt << 5) | ((g ^ (wt & 7)) << 2))) =
              make_float4(v[32 * h + 4 * g], v[32 * h + 4 * g + 1], v[32 * h + 4 * g + 2], v[32 * h + 4 * g + 3]);
    }
    bar_worker(w);
    {
      const uint32_t lane = (uint32_t)(wt & 31), hi = (uint32_t)(wt >> 5) << 11;
#pragma unroll
      for (int s = 0; s < 64; ++s) v[s] = zw[hi | ((uint32_t)s << 5) | (lane ^ (((uint32_t)s & 7u) << 2))];
      fwht64(v);
#pragma unroll
      for (int s = 0; s < 64; ++s) zw[hi | ((uint32_t)s << 5) | (lane ^ (((uint32_t)s & 7u) << 2))] = v[s];
    }
    __syncthreads();
    const bool full = slots >= J0.full_min;
    // Step pairs (full-step mode, kPairMinSlots or more rows per thread):
    // steps j (even) and j + 1 of a unit are combined together.  After both
    // are transformed, buffer of j holds z_j + z_(j+1) and buffer of j + 1
    // z_j - z_(j+1), word by word; a row with chunk-group bits h' = h >> 2
    // adds (-1)^popcount(h' & j) times the word of the first buffer if h' is
    // even, of the second if odd (the signs of j and j + 1 differ exactly by
    // h' & 1).  Each row then reads one word per two steps.
    const bool pair_second = pair_q >= 0;
    const bool pair_first = !pair_second && full && slots >= kPairMinSlots && (j & 1) == 0 && j + 1 < J0.J &&
                            ls + 1 < nsteps;
    if (full) {
      if (pair_second)
        cross_chunk_h4_pair(stage + pair_q * kStageFloats, stage + q * kStageFloats, tid);
      else
        cross_chunk_h4(stage + q * kStageFloats, tid);
      __syncthreads();
    }
    if (pair_first) {
      pair_q = q;
      cur.next(jobs, njobs);
      if (++q == kStages) {
        q = 0;
        phase ^= 1u;
      }
      continue;
    }

    const uint32_t jm = (uint32_t)(pair_second ? j - 1 : j) << 16;
    // the first buffer of a pair (or this step's), and the offset of the second
    const uint32_t cb_u32 = pair_second ? stage_u32 + (uint32_t)(pair_q * kStageFloats) * 4u : step_u32;
    const uint32_t cb_delta = pair_second ? step_u32 - cb_u32 : 0u;
    {
      uint32_t pk[8], acc[8], pkn[8], accn[8];
      tmem_wait_st();
      tmem_ld8(t_pk, pk);
      tmem_ld8(t_acc, acc);
      tmem_wait_ld();
      for (int s8 = 0; s8 < slots; s8 += 8) {
        const bool more = s8 + 8 < slots;
        if (more) {
          tmem_ld8(t_pk + s8 + 8, pkn);
          tmem_ld8(t_acc + s8 + 8, accn);
        }
        if (pair_second) {
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const uint32_t p = pk[e];
            const float y = lds_1(cb_u32 + (p & 0xfffcu) + ((p >> 16) & 1u) * cb_delta);
            acc[e] = __float_as_uint(__uint_as_float(acc[e]) + xor_sign(y, (uint32_t)__popc(p & jm) << 31));
          }
        } else if (full) {
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const uint32_t p = pk[e];
            const float y = lds_1(step_u32 + (p & 0xfffcu));
            acc[e] = __float_as_uint(__uint_as_float(acc[e]) + xor_sign(y, (uint32_t)__popc(p & jm) << 31));
          }
        } else {
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const uint32_t p = pk[e];
            float z0, z1, z2, z3;
            lds_x4(step_u32 + (p & 0x3ffcu), z0, z1, z2, z3);
            const float s1 = __int_as_float((int)((p & 0x80000000u) | 0x3f800000u));
            const float s2 = __int_as_float((int)(((p << 1) & 0x80000000u) | 0x3f800000u));
            const float t = fmaf(s2, fmaf(s1, z3, z2), fmaf(s1, z1, z0));
            acc[e] = __float_as_uint(__uint_as_float(acc[e]) + xor_sign(t, (uint32_t)__popc(p & jm) << 31));
          }
        }
        tmem_st8(t_acc + s8, acc);
        if (more) {
          tmem_wait_ld();
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            pk[e] = pkn[e];
            acc[e] = accn[e];
          }
        }
      }
    }
    cur.next(jobs, njobs);
    const int qs = q;  // this step's buffer
    if (++q == kStages) {
      q = 0;
      phase ^= 1u;
    }
    consumed = ls + 1;
    const int qpair = pair_q;  // a finished pair's first buffer (free now), or -1
    pair_q = -1;

    // end of this block's part of (instance ji, unit u)
    if (j == J0.J - 1 || ls == nsteps - 1) {
      const bool poisoned = *(volatile int *)&stalled != 0;
      const int64_t g0 = J0.step0 + u * J0.J;  // the unit's first global step
      const int64_t first = block_of_step(starts, B, g0);
      const int64_t last = block_of_step(starts, B, g0 + J0.J - 1);
      const int64_t nseg = last - first + 1;
      const int64_t seg = bid - first;
      float *pslot = part + (size_t)first * maxseg * rpg_max;  // the unit starting in block `first`
      tmem_wait_st();
      if (nseg == 1) {
        // Whole unit in this block: its rows k0 .. k0 + nk - 1 (a plan group
        // holds consecutive rows) go through this step's buffer (and, after a
        // step pair, the pair's first buffer too), 16384 (32768) at a time,
        // so that the sketch column is written with coalesced stores.  The
        // buffers are refilled only after the next step's first barrier.
        float *ost = stage + qs * kStageFloats;
        float *ost2 = stage + (qpair >= 0 ? qpair : qs) * kStageFloats;
        const int64_t span = (qpair >= 0 ? 2 : 1) * (int64_t)kStageFloats;
        const int64_t k0 = kg * J0.rpg;
        const int64_t nk = min(J0.rpg, (int64_t)J0.r - k0);
        float *dst = ((col < d) ? J0.SA + (int64_t)col * J0.ldsa : J0.SB) + k0;
        // the row indices of 32 rows at a time, the next 32 loaded while
        // these are placed (their latency is then paid once per pass)
        const int32_t *kk_src = J0.pkk + (size_t)kg * slots * kThreads + tid;
        auto load_kk = [&](int s32, int32_t *kk) {
          const int n8 = min(4, (slots - s32) >> 3);
#pragma unroll
          for (int e = 0; e < 32; ++e) kk[e] = (e < 8 * n8) ? __ldg(kk_src + (size_t)(s32 + e) * kThreads) : -1;
        };
        for (int64_t h0 = 0; h0 < nk; h0 += span) {
          __syncthreads();  // the combine (or the previous copy) is done with the buffer
          int32_t kk[32], kn[32];
          load_kk(0, kk);
          for (int s32 = 0; s32 < slots; s32 += 32) {
            const int n8 = min(4, (slots - s32) >> 3);
            uint32_t acc[32];
            if (s32 + 32 < slots) load_kk(s32 + 32, kn);
#pragma unroll
            for (int b8 = 0; b8 < 4; ++b8)
              if (b8 < n8) tmem_ld8(t_acc + s32 + 8 * b8, acc + 8 * b8);
            tmem_wait_ld();
#pragma unroll
            for (int e = 0; e < 32; ++e) {
              const int64_t o = (int64_t)kk[e] - k0 - h0;
              if (kk[e] < 0 || o < 0 || o >= span) continue;
              (o < kStageFloats ? ost : ost2)[o & (kStageFloats - 1)] =
                  poisoned ? __int_as_float(0x7fc00000) : J0.scale * __uint_as_float(acc[e]);
            }
#pragma unroll
            for (int e = 0; e < 32; ++e) kk[e] = kn[e];
          }
          __syncthreads();
          const int64_t cnt = min(span, nk - h0);
          for (int64_t i = tid; i < cnt; i += kThreads) dst[h0 + i] = (i < kStageFloats ? ost : ost2)[i & (kStageFloats - 1)];
        }
        for (int s8 = 0; s8 < slots; s8 += 8) tmem_st8(t_acc + s8, zero8);
      } else {
      // 32 rows at a time: their indices and sums are fetched together
      for (int s32 = 0; s32 < slots; s32 += 32) {
        const int n8 = min(4, (slots - s32) >> 3);
        int32_t kk[32];
        uint32_t acc[32];
#pragma unroll
        for (int e = 0; e < 32; ++e)
          kk[e] = (e < 8 * n8) ? J0.pkk[((size_t)kg * slots + s32 + e) * kThreads + tid] : -1;
#pragma unroll
        for (int b8 = 0; b8 < 4; ++b8)
          if (b8 < n8) tmem_ld8(t_acc + s32 + 8 * b8, acc + 8 * b8);
        tmem_wait_ld();
#pragma unroll
        for (int e = 0; e < 32; ++e) {
          if (kk[e] < 0) continue;
          const float a = poisoned ? __int_as_float(0x7fc00000) : __uint_as_float(acc[e]);
          if (nseg == 1) {
            if (col < d)
              J0.SA[(int64_t)col * J0.ldsa + kk[e]] = J0.scale * a;
            else
              J0.SB[kk[e]] = J0.scale * a;
          } else {
            pslot[(size_t)seg * rpg_max + (size_t)(s32 + e) * kThreads + tid] = a;
          }
        }
#pragma unroll
        for (int b8 = 0; b8 < 4; ++b8)
          if (b8 < n8) tmem_st8(t_acc + s32 + 8 * b8, zero8);
      }
      }
      if (nseg > 1) {
        __threadfence();
        __syncthreads();
        if (tid == 0) last_flag = (atomicAdd(&counters[first], 1u) == (unsigned int)(nseg - 1)) ? 1u : 0u;
        __syncthreads();
        if (last_flag) {
          __threadfence();
          for (int s0b = 0; s0b < slots; s0b += 32) {
            int32_t kk[32];
            float sum[32];
#pragma unroll
            for (int e = 0; e < 32; ++e) {
              kk[e] = (s0b + e < slots) ? J0.pkk[((size_t)kg * slots + s0b + e) * kThreads + tid] : -1;
              sum[e] = 0.0f;
            }
            for (int64_t g = 0; g < nseg; ++g) {
              const float *pg = pslot + (size_t)g * rpg_max + (size_t)s0b * kThreads + tid;
              float t[32];
#pragma unroll
              for (int e = 0; e < 32; ++e) t[e] = (kk[e] >= 0) ? __ldcg(pg + (size_t)e * kThreads) : 0.0f;
#pragma unroll
              for (int e = 0; e < 32; ++e) sum[e] += t[e];
            }
#pragma unroll
            for (int e = 0; e < 32; ++e) {
              if (kk[e] < 0) continue;
              if (col < d)
                J0.SA[(int64_t)col * J0.ldsa + kk[e]] = J0.scale * sum[e];
              else
                J0.SB[kk[e]] = J0.scale * sum[e];
            }
          }
          if (tid == 0) counters[first] = 0u;
        }
      }
    }
  }
  tmem_wait_st();
  tmem_fence_before();
  __syncthreads();
  tmem_fence_after();
  if (tid < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base_s), "r"(kTmemCols)
                 : "memory");
}

// ---------------------------------------------------------------------------
// whole column in shared memory (n <= 2^13), FP32 or FP64
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) sketch_small(const T *__restrict__ A, int64_t lda, const T *__restrict__ b,
                                                    int64_t ldb, int64_t n_raw, int d, int L, uint64_t seed,
                                                    uint64_t inst, const int32_t *__restrict__ idx, int64_t r,
                                                    const int64_t *__restrict__ d_count, T scale, T *__restrict__ SA,
                                                    int64_t ldsa, T *__restrict__ Sb, int64_t ldsb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = 1 << L;
  uint64_t *words = reinterpret_cast<uint64_t *>(smem_raw);  // max(n/64, 4) sign words
  T *buf = reinterpret_cast<T *>(words + (n / 64 > 4 ? n / 64 : 4));
  const int col = blockIdx.x;
  const T *__restrict__ x = (col < d) ? A + (int64_t)col * lda : b + (int64_t)(col - d) * ldb;
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
  T *out = (col < d) ? SA + (int64_t)col * ldsa : Sb + (int64_t)(col - d) * ldsb;
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

// rows of the plan per sketch thread: enough for r rows in one plan group,
// a multiple of 8 (TMEM moves eight at a time), at most kMaxSlots (then
// several groups, each a pass over the data)
int pick_slots(int64_t rows) {
  const int64_t need = (rows + kThreads - 1) / kThreads;
  return (int)std::min<int64_t>(kMaxSlots, std::max<int64_t>(8, (need + 7) / 8 * 8));
}
// the same with the split-precision mode's smaller TMEM share (kTcRowSlots):
// the fewest plan groups, rows spread evenly over them
int pick_slots_tc(int64_t rows) {
  const int64_t need = (rows + kThreads - 1) / kThreads;
  const int64_t groups = std::max<int64_t>(1, (need + kTcRowSlots - 1) / kTcRowSlots);
  const int64_t per = (need + groups - 1) / groups;
  return (int)std::min<int64_t>(kTcRowSlots, std::max<int64_t>(8, (per + 7) / 8 * 8));
}

typedef CUresult (*encode_tiled_fn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                    const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                    CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

encode_tiled_fn tensor_map_encoder() {
  static encode_tiled_fn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<encode_tiled_fn>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

// Column view (32, n_raw / 32, cols) of a column-major FP32 matrix: box
// (32, 128, 1) is one 4096-row chunk of one column, swizzled by 128 bytes;
// lines past the end read as zero.
int column_map(CUtensorMap *m, const float *base, int64_t n_raw, int64_t cols, int64_t ld) {
  encode_tiled_fn enc = tensor_map_encoder();
  if (!enc) return RNNLS_ECUDA;
  const cuuint64_t lines = (cuuint64_t)(n_raw / 32);
  cuuint64_t dims[3] = {32, lines, (cuuint64_t)cols};
  cuuint64_t strides[2] = {128, (cuuint64_t)(cols > 1 ? ld : 32 * (int64_t)lines) * 4};
  cuuint32_t box[3] = {32, kM / 32, 1};
  cuuint32_t es[3] = {1, 1, 1};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(base), dims, strides, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? RNNLS_OK : RNNLS_ECUDA;
}

int launch_srht(cudaStream_t s, const sketch_args_f32 &a, const plan_t &plan, const srht_part &P, int blocks, int vec,
                const uint64_t *signs, float *part, unsigned int *counters) {
  static once_per_device attrs;
  if (attrs.run([] {
        for (auto kern : {sketch_srht_f32<0, false>, sketch_srht_f32<8, false>, sketch_srht_f32<16, false>,
                          sketch_srht_f32<24, false>, sketch_srht_f32<32, false>, sketch_srht_f32<40, false>,
                          sketch_srht_f32<0, true>, sketch_srht_f32<8, true>, sketch_srht_f32<16, true>,
                          sketch_srht_f32<24, true>, sketch_srht_f32<32, true>, sketch_srht_f32<40, true>}) {
          const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     (int)kSketchSmem);
          if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
      }) != cudaSuccess)
    return RNNLS_ECUDA;
  CUtensorMap tmA, tmB;
  memset(&tmA, 0, sizeof(tmA));
  memset(&tmB, 0, sizeof(tmB));
  if (vec) {
    int st = column_map(&tmA, a.A, a.n_raw, a.d, a.lda);
    if (!st) st = column_map(&tmB, a.b, a.n_raw, a.nb, a.ldb);
    if (st) return st;
  }
  // up to 40 rows per thread in registers, beyond that in TMEM
  auto kern = a.tc ? (plan.slots == 8    ? sketch_srht_f32<8, true>
                      : plan.slots == 16 ? sketch_srht_f32<16, true>
                      : plan.slots == 24 ? sketch_srht_f32<24, true>
                      : plan.slots == 32 ? sketch_srht_f32<32, true>
                      : plan.slots == 40 ? sketch_srht_f32<40, true>
                                         : sketch_srht_f32<0, true>)
                   : (plan.slots == 8    ? sketch_srht_f32<8, false>
                      : plan.slots == 16 ? sketch_srht_f32<16, false>
                      : plan.slots == 24 ? sketch_srht_f32<24, false>
                      : plan.slots == 32 ? sketch_srht_f32<32, false>
                      : plan.slots == 40 ? sketch_srht_f32<40, false>
                                         : sketch_srht_f32<0, false>);
  // programmatic dependent of the plan launch before it (the kernel waits for
  // that launch before it reads anything the launch writes)
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = kSketchSmem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e =
      cudaLaunchKernelEx(&cfg, kern, tmA, tmB, a.A, a.lda, a.b, a.ldb, a.n_raw, a.d, a.nb, a.chunk0 / 4, P, vec, a.seed,
                         a.inst, signs, plan.pk, plan.k, plan.slots, plan.rows_per_group, part, a.scale, a.SA, a.ldsa,
                         a.Sb, a.ldsb, counters);
  return (e == cudaSuccess && cudaGetLastError() == cudaSuccess) ? RNNLS_OK : RNNLS_ECUDA;
}

// Launch geometry of the large-n sketch for `sms` usable SMs.
struct srht_geom {
  plan_t plan;
  srht_part P;
  int blocks;
  int vec;
  int64_t maxseg;      // partial-sum segments per unit (0: no unit is split)
  int64_t sign_words;  // sign words of D for the chunks with data
  size_t plan_bytes, part_bytes, sign_bytes;
};

srht_geom plan_geometry(const sketch_args_f32 &a, int sms, bool force_aligned, int full_min = kFullMinSlots) {
  srht_geom g{};
  g.P.full_min = full_min;
  g.plan.slots = a.tc ? pick_slots_tc(a.r) : pick_slots(a.r);
  g.plan.rows_per_group = (int64_t)kThreads * g.plan.slots;
  g.plan.kgroups = (int)((a.r + g.plan.rows_per_group - 1) / g.plan.rows_per_group);
  g.vec = (((uintptr_t)a.A % 16 == 0) && (a.lda % 4 == 0) && ((uintptr_t)a.b % 16 == 0) &&
           (a.nb == 1 || a.ldb % 4 == 0))
              ? 1
              : 0;
  g.P.J = (a.n_raw + 4 * (int64_t)kM - 1) / (4 * (int64_t)kM);
  g.P.U = (int64_t)g.plan.kgroups * (a.d + a.nb);
  g.P.T = g.P.U * g.P.J;
  // many more columns than SMs: whole columns per block balance well enough
  g.P.aligned = (force_aligned || g.P.U >= 8 * (int64_t)sms) ? 1 : 0;
  g.blocks = (int)std::max<int64_t>(1, std::min<int64_t>(sms, g.P.aligned ? g.P.U : g.P.T));
  g.maxseg = 0;
  if (!g.P.aligned) {
    for (int64_t u = 0; u < g.P.U; ++u) {
      const int64_t f = part_block_of(u * g.P.J, g.blocks, g.P), l = part_block_of(u * g.P.J + g.P.J - 1, g.blocks, g.P);
      if (l > f) g.maxseg = std::max<int64_t>(g.maxseg, l - f + 1);
    }
  }
  g.sign_words = 4 * g.P.J * (kM / 64);
  g.sign_bytes = align_up((size_t)g.sign_words * sizeof(uint64_t), 256);
  g.plan_bytes = plan_ws_bytes(g.plan.slots, g.plan.kgroups);
  g.part_bytes = align_up((size_t)g.maxseg * g.P.U * g.plan.rows_per_group * sizeof(float), 256);
  return g;
}

void carve_plan(ws_carver &wc, plan_t &plan) {
  plan.pk = wc.take<uint32_t>((size_t)plan.kgroups * plan.slots * kThreads);
  plan.k = wc.take<int32_t>((size_t)plan.kgroups * plan.slots * kThreads);
}

}  // namespace

int sketch_f32(rnnls_ctx *ctx, const sketch_args_f32 &a, int num_sms) {
  const int64_t n = (int64_t)1 << a.L;
  cudaStream_t s = ctx->stream;
  if (n <= 8192) {
    const size_t smem = (size_t)n * sizeof(float) + (size_t)std::max<int64_t>(n / 64, 4) * sizeof(uint64_t);
    if (ctx->plan_event) RNNLS_CUDA_TRY(cudaEventRecord(ctx->plan_event, s));  // no plan at this size
    prof_scope ps(ctx, K_SKETCH_SMALL);
    sketch_small<float><<<(unsigned)(a.d + a.nb), 256, smem, s>>>(a.A, a.lda, a.b, a.ldb, a.n_raw, a.d, a.L, a.seed,
                                                                  a.inst, a.idx, a.r, a.d_count, a.scale, a.SA,
                                                                  a.ldsa, a.Sb, a.ldsb);
    return cudaGetLastError() == cudaSuccess ? RNNLS_OK : RNNLS_ECUDA;
  }
  const int sms = (ctx->sketch_sms > 0) ? std::min(ctx->sketch_sms, num_sms) : num_sms;
  srht_geom g = plan_geometry(a, sms, false, tune_or(ctx->tune.full_step_min_slots, kFullMinSlots));
  int st = ensure_workspace(ctx, g.part_bytes + g.plan_bytes + g.sign_bytes + 1024);
  if (st) return st;
  ws_carver wc(ctx->ws);
  float *part = g.maxseg ? wc.take<float>((size_t)g.maxseg * g.P.U * g.plan.rows_per_group) : nullptr;
  carve_plan(wc, g.plan);
  uint64_t *signs = wc.take<uint64_t>((size_t)g.sign_words);
  unsigned int *counters = nullptr;
  if (g.maxseg) {
    st = ensure_counters(ctx, (size_t)g.P.U, &counters);
    if (st) return st;
  }
  {
    // one launch: the plan entries, D's sign words and, in iid mode, the
    // rows, which every plan block draws in full for itself
    prof_scope ps(ctx, K_PLAN);
    st = launch_build_plan(s, a.idx, a.r, a.d_count, g.plan, signs, g.sign_words, 16 * a.chunk0, a.seed, a.inst,
                           a.gen_iid ? a.L : 0);
  }
  if (st) return st;
  if (ctx->plan_event) RNNLS_CUDA_TRY(cudaEventRecord(ctx->plan_event, s));
  prof_scope ps_main(ctx, K_SKETCH);
  return launch_srht(s, a, g.plan, g.P, g.blocks, g.vec, signs, part, counters);
}

int sketch_batched_f32(rnnls_ctx *ctx, const rnnls_sketch_job *jobs, int64_t count, int tc) {
  cudaStream_t s = ctx->stream;
  const int num_sms = ctx->num_sms;
  // instances too small for the chunked path go one by one
  std::vector<int64_t> big;
  for (int64_t i = 0; i < count; ++i) {
    const rnnls_sketch_job &jb = jobs[i];
    if (((int64_t)1 << log2_ceil64(jb.n_raw)) > 8192) {
      big.push_back(i);
      continue;
    }
    sketch_args_f32 a{};
    a.A = jb.A; a.lda = jb.lda; a.b = jb.b; a.ldb = jb.n_raw; a.nb = 1; a.n_raw = jb.n_raw; a.d = (int)jb.d;
    a.L = log2_ceil64(jb.n_raw); a.chunk0 = 0; a.r = jb.r; a.d_count = nullptr; a.seed = jb.seed;
    a.inst = jb.instance; a.scale = (float)(1.0 / sqrt((double)jb.r)); a.SA = jb.SA; a.ldsa = jb.ldsa; a.Sb = jb.Sb;
    a.ldsb = jb.ldsa; a.idx = jb.idx; a.gen_iid = 0; a.tc = tc;
    int st = launch_sample_iid(s, jb.seed, jb.instance, a.L, jb.r, jb.idx);
    if (!st) st = sketch_f32(ctx, a, num_sms);
    if (st) return st;
  }
  const int nb = (int)big.size();
  if (nb == 0) return RNNLS_OK;
  // per-instance geometry; global step offsets
  std::vector<srht_job> sj((size_t)nb);
  std::vector<plan_job> pj((size_t)nb);
  std::vector<int64_t> first_s((size_t)nb + 1), first_p((size_t)nb + 1);
  int64_t Ttot = 0, rpg_max = 0, samp_tot = 0, plan_tot = 0;
  size_t plan_bytes = 0;
  for (int t = 0; t < nb; ++t) {
    const rnnls_sketch_job &jb = jobs[big[(size_t)t]];
    srht_job &J = sj[(size_t)t];
    memset(&J, 0, sizeof(J));
    const int slots = tc ? pick_slots_tc(jb.r) : pick_slots(jb.r);
    const int64_t rpg = (int64_t)kThreads * slots;
    const int kgroups = (int)((jb.r + rpg - 1) / rpg);
    J.A = jb.A; J.B = jb.b; J.lda = jb.lda; J.ldb = jb.n_raw; J.ldsa = jb.ldsa; J.ldsb = jb.ldsa;
    J.n_raw = jb.n_raw; J.J = (jb.n_raw + 4 * (int64_t)kM - 1) / (4 * (int64_t)kM);
    J.U = (int64_t)kgroups * (jb.d + 1); J.step0 = Ttot; J.rpg = rpg; J.scale = (float)(1.0 / sqrt((double)jb.r));
    J.d = (int)jb.d; J.slots = slots; J.r = (int)jb.r; J.SA = jb.SA; J.SB = jb.Sb;
    J.full_min = tune_or(ctx->tune.full_step_min_slots, kFullMinSlots);
    J.vec = (((uintptr_t)jb.A % 16 == 0) && (jb.lda % 4 == 0) && ((uintptr_t)jb.b % 16 == 0)) ? 1 : 0;
    Ttot += J.U * J.J;
    rpg_max = std::max(rpg_max, rpg);
    plan_job &P = pj[(size_t)t];
    P.idx = jb.idx; P.r = jb.r; P.slots = slots; P.kgroups = kgroups; P.L = log2_ceil64(jb.n_raw);
    P.rows_per_group = rpg; P.seed = jb.seed; P.inst = jb.instance; P.sign_words = 4 * J.J * (kM / 64);
    plan_bytes += plan_ws_bytes(slots, kgroups) + align_up((size_t)P.sign_words * 8, 256) + 512;
    first_s[(size_t)t] = samp_tot;
    first_p[(size_t)t] = plan_tot;
    samp_tot += sample_blocks(jb.r);
    plan_tot += plan_blocks(P);
  }
  first_s[(size_t)nb] = samp_tot;
  first_p[(size_t)nb] = plan_tot;
  const int sms = (ctx->sketch_sms > 0) ? std::min(ctx->sketch_sms, num_sms) : num_sms;
  const int64_t B = std::max<int64_t>(1, std::min<int64_t>(sms, Ttot));
  // Block ranges of equal estimated cost, in units of about 22 ns: a step
  // costs about 114 + slots (the transform, then the plan rows), plus the
  // unit's write-out (about 6 slots) spread over its J steps.
  std::vector<int64_t> starts((size_t)B + 1);
  {
    std::vector<double> wt((size_t)nb), cum((size_t)nb + 1, 0.0);
    const double step_cost = (double)tune_or(ctx->tune.batch_step_cost, 114);
    for (int t = 0; t < nb; ++t) {
      const srht_job &J = sj[(size_t)t];
      // steps combined in pairs (full-step mode) read each row once per two
      // steps: about half the rows' cost, plus the pair's extra butterfly pass
      const bool pairs = J.slots >= J.full_min && J.slots >= kPairMinSlots && J.J >= 2;
      wt[(size_t)t] = step_cost + (pairs ? 16.0 + 0.55 * J.slots : (double)J.slots) + 6.0 * (double)J.slots / (double)J.J;
      cum[(size_t)t + 1] = cum[(size_t)t] + wt[(size_t)t] * (double)(J.U * J.J);
    }
    int t = 0;
    starts[0] = 0;
    for (int64_t b = 1; b < B; ++b) {
      const double target = cum[(size_t)nb] * (double)b / (double)B;
      while (t + 1 < nb && cum[(size_t)t + 1] <= target) ++t;
      const srht_job &J = sj[(size_t)t];
      int64_t st_b = J.step0 + (int64_t)((target - cum[(size_t)t]) / wt[(size_t)t]);
      // every block keeps at least one step (a split unit then has a segment in
      // every block of its span)
      st_b = std::max(st_b, starts[(size_t)b - 1] + 1);
      starts[(size_t)b] = std::min(st_b, Ttot - (B - b));
    }
    starts[(size_t)B] = Ttot;
  }
  // a unit split between blocks uses the slots of the block where it starts
  int maxseg = 1;
  for (int64_t b = 1; b < B; ++b) {
    const int64_t s_last = starts[(size_t)b] - 1;
    if (s_last < 0) continue;
    int lo = 0, hi = nb - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (sj[(size_t)mid].step0 <= s_last)
        lo = mid;
      else
        hi = mid - 1;
    }
    const srht_job &J = sj[(size_t)lo];
    const int64_t g0 = J.step0 + ((s_last - J.step0) / J.J) * J.J;
    const int64_t f = block_of_step(starts.data(), B, g0), l = block_of_step(starts.data(), B, g0 + J.J - 1);
    maxseg = std::max<int>(maxseg, (int)(l - f + 1));
  }
  const size_t tables = align_up((size_t)nb * sizeof(srht_job), 256) + align_up((size_t)nb * sizeof(plan_job), 256) +
                        2 * align_up((size_t)(nb + 1) * sizeof(int64_t), 256) +
                        align_up((size_t)(B + 1) * sizeof(int64_t), 256);
  const size_t part_bytes = align_up((size_t)B * maxseg * rpg_max * sizeof(float), 256);
  int st = ensure_workspace(ctx, tables + plan_bytes + part_bytes + 4096);
  if (st) return st;
  unsigned int *counters = nullptr;
  st = ensure_counters(ctx, (size_t)B, &counters);
  if (st) return st;
  st = ensure_pinned(ctx, tables);
  if (st) return st;
  ws_carver wc(ctx->ws);
  char *d_tables = wc.take<char>(tables);
  float *part = wc.take<float>((size_t)B * maxseg * rpg_max);
  for (int t = 0; t < nb; ++t) {
    plan_job &P = pj[(size_t)t];
    srht_job &J = sj[(size_t)t];
    plan_t pl;
    pl.slots = P.slots;
    pl.kgroups = P.kgroups;
    pl.rows_per_group = P.rows_per_group;
    carve_plan(wc, pl);
    P.pk = pl.pk;
    P.k = pl.k;
    P.signs = wc.take<uint64_t>((size_t)P.sign_words);
    J.pk = P.pk;
    J.pkk = P.k;
    J.signs = P.signs;
    if (J.vec) {
      st = column_map(&J.tmA, J.A, J.n_raw, J.d, J.lda);
      if (!st) st = column_map(&J.tmB, J.B, J.n_raw, 1, J.n_raw);
      if (st) return st;
    }
  }
  char *h = (char *)ctx->pinned;
  memcpy(h, sj.data(), (size_t)nb * sizeof(srht_job));
  size_t off = align_up((size_t)nb * sizeof(srht_job), 256);
  // plan blocks start with the instances of most rows (a plan block's work
  // grows with r): the last blocks to start are short ones
  {
    std::vector<int> order((size_t)nb);
    for (int t = 0; t < nb; ++t) order[(size_t)t] = t;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return pj[(size_t)a].r > pj[(size_t)b].r; });
    std::vector<plan_job> pj2((size_t)nb);
    samp_tot = 0;
    plan_tot = 0;
    for (int k = 0; k < nb; ++k) {
      pj2[(size_t)k] = pj[(size_t)order[(size_t)k]];
      first_s[(size_t)k] = samp_tot;
      first_p[(size_t)k] = plan_tot;
      samp_tot += sample_blocks(pj2[(size_t)k].r);
      plan_tot += plan_blocks(pj2[(size_t)k]);
    }
    first_s[(size_t)nb] = samp_tot;
    first_p[(size_t)nb] = plan_tot;
    pj.swap(pj2);
  }
  memcpy(h + off, pj.data(), (size_t)nb * sizeof(plan_job));
  const size_t off_p = off;
  off += align_up((size_t)nb * sizeof(plan_job), 256);
  memcpy(h + off, first_s.data(), (size_t)(nb + 1) * sizeof(int64_t));
  const size_t off_fs = off;
  off += align_up((size_t)(nb + 1) * sizeof(int64_t), 256);
  memcpy(h + off, first_p.data(), (size_t)(nb + 1) * sizeof(int64_t));
  const size_t off_fp = off;
  off += align_up((size_t)(nb + 1) * sizeof(int64_t), 256);
  memcpy(h + off, starts.data(), (size_t)(B + 1) * sizeof(int64_t));
  const size_t off_st = off;
  RNNLS_CUDA_TRY(cudaMemcpyAsync(d_tables, h, tables, cudaMemcpyHostToDevice, s));
  RNNLS_CUDA_TRY(cudaEventRecord(ctx->pinned_ready, s));
  {
    prof_scope ps(ctx, K_PLAN);
    st = launch_plan_batched(s, (const plan_job *)(d_tables + off_p), (const int64_t *)(d_tables + off_fs),
                             (const int64_t *)(d_tables + off_fp), nb, samp_tot, plan_tot);
  }
  if (st) return st;
  static smem_attr batch_attr, batch_attr_tc;
  auto kern = tc ? sketch_srht_batch_f32<true> : sketch_srht_batch_f32<false>;
  RNNLS_CUDA_TRY((tc ? batch_attr_tc : batch_attr).ensure((const void *)kern, kSketchSmem));
  prof_scope ps_main(ctx, K_SKETCH);
  kern<<<(unsigned)B, kThreads, kSketchSmem, s>>>((const srht_job *)d_tables, nb, (const int64_t *)(d_tables + off_st),
                                                  part, maxseg, rpg_max, counters);
  return cudaGetLastError() == cudaSuccess ? RNNLS_OK : RNNLS_ECUDA;
}

int sketch_f32_scratch(cudaStream_t s, const sketch_args_f32 &a, int num_sms, void *scratch, size_t bytes) {
  const int64_t n = (int64_t)1 << a.L;
  if (n <= 8192) {
    const size_t smem = (size_t)n * sizeof(float) + (size_t)std::max<int64_t>(n / 64, 4) * sizeof(uint64_t);
    sketch_small<float><<<(unsigned)(a.d + a.nb), 256, smem, s>>>(a.A, a.lda, a.b, a.ldb, a.n_raw, a.d, a.L, a.seed,
                                                                  a.inst, a.idx, a.r, a.d_count, a.scale, a.SA,
                                                                  a.ldsa, a.Sb, a.ldsb);
    return cudaGetLastError() == cudaSuccess ? RNNLS_OK : RNNLS_ECUDA;
  }
  // counters first (zeroed by every call), then the plan, then partial sums;
  // whole columns per block when the partial sums do not fit
  srht_geom g = plan_geometry(a, num_sms, false);
  const size_t cnt_bytes = align_up((size_t)g.P.U * sizeof(unsigned int), 256);
  if (cnt_bytes + g.plan_bytes + g.part_bytes + 768 > bytes) g = plan_geometry(a, num_sms, true);
  if (cnt_bytes + g.plan_bytes + g.part_bytes + 768 > bytes) return RNNLS_EUNSUPPORTED;
  // the sign table when it fits, else the kernel draws D's words itself
  const bool table = cnt_bytes + g.plan_bytes + g.part_bytes + g.sign_bytes + 768 <= bytes;
  ws_carver wc(scratch);
  unsigned int *counters = wc.take<unsigned int>((size_t)g.P.U);
  carve_plan(wc, g.plan);
  uint64_t *signs = table ? wc.take<uint64_t>((size_t)g.sign_words) : nullptr;
  float *part = g.maxseg ? wc.take<float>((size_t)g.maxseg * g.P.U * g.plan.rows_per_group) : nullptr;
  if (g.maxseg && cudaMemsetAsync(counters, 0, (size_t)g.P.U * sizeof(unsigned int), s) != cudaSuccess)
    return RNNLS_ECUDA;
  const int st = launch_build_plan(s, a.idx, a.r, a.d_count, g.plan, signs, g.sign_words, 16 * a.chunk0, a.seed,
                                   a.inst, a.gen_iid ? a.L : 0);
  if (st) return st;
  return launch_srht(s, a, g.plan, g.P, g.blocks, g.vec, signs, part, counters);
}

int sketch_f64(rnnls_ctx *ctx, const sketch_args_f64 &a) {
  const int64_t n = (int64_t)1 << a.L;
  cudaStream_t s = ctx->stream;
  prof_scope ps(ctx, K_SKETCH_F64);
  if (n <= 8192) {
    const size_t smem = (size_t)n * sizeof(double) + (size_t)std::max<int64_t>(n / 64, 4) * sizeof(uint64_t);
    static smem_attr small_attr;
    RNNLS_CUDA_TRY(small_attr.ensure((const void *)sketch_small<double>, 8192 * sizeof(double) + 128 * sizeof(uint64_t)));
    sketch_small<double><<<(unsigned)(a.d + 1), 256, smem, s>>>(a.A, a.lda, a.b, a.n_raw, a.n_raw, a.d, a.L, a.seed,
                                                                a.inst, a.idx, a.r, a.d_count, a.scale, a.SA, a.ldsa,
                                                                a.Sb, a.r);
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
