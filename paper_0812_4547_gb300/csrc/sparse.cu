// sparse.cu -- the sketch H~D[A | b] of Alg. 1 for a sparse A given by
// columns (compressed sparse column: column pointers, row indices, values),
// the form of the paper's term-document data (Sec. 4.1, Sec. 4.2: 2-64 %
// non-zeros).  It computes exactly what the dense sketch computes (same
// Philox rows and signs, same 1/sqrt(r) scale): only the read of A changes.
//
// Work: a unit is (column, range of steps); a step is 16384 consecutive rows
// (four chunks of 4096, fewer when n < 16384).  Per step the block zeroes its
// stage buffer, scatters the column's non-zeros of those rows into it with
// their signs D_ii (a binary search finds them: row indices ascend within a
// column; the dense b is loaded whole), and transforms every chunk in place:
// H_4096 = H_64 (x) H_64, two passes of a 64-point transform held in the
// registers of 64 threads (one chunk per 64 threads).  A chunk is stored as
// a 64 x 64 matrix whose element (i, j) sits at i * 64 + (j ^ (i mod 32)), so
// both passes (a column per thread, then a row per thread) read and write
// 32 different banks per warp.  Then every sampled row i = c * 4096 + l
// gains sum over the step's chunks c' of (-1)^popcount(c & c') z_c'[l]
// (H_n = H_{n/4096} (x) H_4096), kept in shared memory per row.  A column
// split over several units leaves per-unit partial sums that a second launch
// adds in unit order (and scales); otherwise the unit writes SA directly.
//
// The transform costs n log2(4096) additions per column whatever the
// density; what sparsity saves is the read of A (8 bytes per non-zero
// instead of 4 per entry) and the memory to hold it.
#include <math.h>

#include <algorithm>

#include "kernels.h"
#include "launch_attr.h"

namespace rnnls {
namespace {

constexpr int kCscThreads = 256;
constexpr int kChunk = 4096;             // rows per chunk (64 x 64)
constexpr int kMaxChunksPerStep = 4;     // one chunk per 64 threads
constexpr int64_t kCscMaxRows = 16384;   // sampled rows (per-row sums in shared memory)

__device__ __forceinline__ uint32_t cswz(uint32_t pos) {  // position in a chunk -> shared-memory word
  const uint32_t i = pos >> 6, j = pos & 63;
  return (i << 6) | (j ^ (i & 31));
}

__device__ __forceinline__ float sign_of(const uint64_t *__restrict__ signs, int64_t row, float v) {
  const uint64_t w = __ldg(signs + (row >> 6));
  return ((w >> (row & 63)) & 1ull) ? -v : v;
}

// Unnormalised 64-point Walsh-Hadamard transform in registers (natural
// order): the stride-1 stage on scalars, strides 2..32 on packed pairs
// (add/sub.rn.f32x2, the same roundings as scalar code).
__device__ __forceinline__ void fwht64(float *v) {
#pragma unroll
  for (int k = 0; k < 64; k += 2) {
    const float a = v[k], b = v[k + 1];
    v[k] = a + b;
    v[k + 1] = a - b;
  }
  uint64_t w[32];
#pragma unroll
  for (int q = 0; q < 32; ++q) asm("mov.b64 %0, {%1, %2};" : "=l"(w[q]) : "f"(v[2 * q]), "f"(v[2 * q + 1]));
#pragma unroll
  for (int h = 1; h < 32; h <<= 1) {
#pragma unroll
    for (int q = 0; q < 32; ++q) {
      if (q & h) continue;
      uint64_t su, df;
      asm("add.rn.f32x2 %0, %1, %2;" : "=l"(su) : "l"(w[q]), "l"(w[q + h]));
      asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(df) : "l"(w[q]), "l"(w[q + h]));
      w[q] = su;
      w[q + h] = df;
    }
  }
#pragma unroll
  for (int q = 0; q < 32; ++q) asm("mov.b64 {%0, %1}, %2;" : "=f"(v[2 * q]), "=f"(v[2 * q + 1]) : "l"(w[q]));
}

// Sign words of D: word w holds the signs of rows 64 w .. 64 w + 63 (bit set:
// -1); Philox block p gives words 4p .. 4p + 3 (stream of the signs).
__global__ void csc_signs_kernel(uint64_t seed, uint64_t inst, int64_t words, uint64_t *__restrict__ out) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (4 * p >= words) return;
  const u64x4 u = philox4x64_10((uint64_t)p, kStreamSigns, seed, inst);
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (4 * p + q < words) out[4 * p + q] = u.w[q];
}

struct csc_args {
  const int64_t *colptr;  // d + 1 offsets
  const int32_t *rowidx;  // ascending within each column
  const float *val;
  const float *b;         // dense target, n_raw
  int64_t n_raw;
  int d;
  int cps;                // chunks per step
  int64_t nsteps;         // steps of the padded column
  int64_t spu;            // steps per unit
  int units_per_col;
  int64_t r;
  const int32_t *idx;
  const uint64_t *signs;
  float scale;
  float *SA;
  int64_t ldsa;
  float *Sb;
  float *part;            // [units_per_col][d + 1][r] when units_per_col > 1
};

// First position p in [lo, hi) with rowidx[p] >= row.
__device__ __forceinline__ int64_t lower_bound_rows(const int32_t *__restrict__ rowidx, int64_t lo, int64_t hi,
                                                    int64_t row) {
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if ((int64_t)__ldg(rowidx + mid) < row)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(kCscThreads, 2) sketch_csc_kernel(const csc_args a) {
  extern __shared__ __align__(16) float csc_smem[];
  __shared__ int64_t range_s[2];
  const int tid = threadIdx.x;
  const int col = (int)(blockIdx.x % (unsigned)(a.d + 1));
  const int g = (int)(blockIdx.x / (unsigned)(a.d + 1));
  const int64_t s_begin = (int64_t)g * a.spu;
  const int64_t s_end = min(a.nsteps, s_begin + a.spu);
  const int step_rows = a.cps * kChunk;
  float *stage = csc_smem;                                   // cps chunks
  float *acc = csc_smem + (size_t)kMaxChunksPerStep * kChunk;  // r per-row sums
  for (int64_t k = tid; k < a.r; k += kCscThreads) acc[k] = 0.0f;
  const bool is_b = (col == a.d);
  int64_t p = 0, p_end = 0;  // this column's non-zeros from the unit's first row on
  if (!is_b) {
    if (tid == 0) {
      const int64_t c0 = __ldg(a.colptr + col), c1 = __ldg(a.colptr + col + 1);
      range_s[0] = lower_bound_rows(a.rowidx, c0, c1, s_begin * step_rows);
      range_s[1] = c1;
    }
    __syncthreads();
    p = range_s[0];
    p_end = range_s[1];
  }
  const int worker = tid >> 6, t = tid & 63;
  for (int64_t st = s_begin; st < s_end; ++st) {
    const int64_t row0 = st * step_rows;
    // zero the stage buffer, then scatter the step's entries with their signs
    float4 *st4 = reinterpret_cast<float4 *>(stage);
    for (int q = tid; q < step_rows / 4; q += kCscThreads) st4[q] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    __syncthreads();
    if (!is_b) {
      if (tid == 0) range_s[0] = lower_bound_rows(a.rowidx, p, p_end, row0 + step_rows);
      __syncthreads();
      const int64_t q_end = range_s[0];
      for (int64_t q = p + tid; q < q_end; q += kCscThreads) {
        const int64_t row = __ldg(a.rowidx + q);
        const uint32_t off = (uint32_t)(row - row0);
        // rows outside the step (input against the stated order) are skipped, never written
        if (off < (uint32_t)step_rows)
          stage[(off >> 12) * kChunk + cswz(off & (kChunk - 1))] = sign_of(a.signs, row, __ldg(a.val + q));
      }
      p = q_end;
    } else {
      for (int q = tid; q < step_rows; q += kCscThreads) {
        const int64_t row = row0 + q;
        if (row < a.n_raw) stage[(q >> 12) * kChunk + cswz(q & (kChunk - 1))] = sign_of(a.signs, row, __ldg(a.b + row));
      }
    }
    __syncthreads();
    // H_4096 on every chunk: a column of the 64 x 64 matrix per thread, then a row
    if (worker < a.cps) {
      float *z = stage + worker * kChunk;
      float v[64];
#pragma unroll
      for (int i = 0; i < 64; ++i) v[i] = z[(i << 6) | (t ^ (i & 31))];
      fwht64(v);
#pragma unroll
      for (int i = 0; i < 64; ++i) z[(i << 6) | (t ^ (i & 31))] = v[i];
    }
    __syncthreads();
    if (worker < a.cps) {
      float *z = stage + worker * kChunk;
      float v[64];
#pragma unroll
      for (int j = 0; j < 64; ++j) v[j] = z[(t << 6) | (j ^ (t & 31))];
      fwht64(v);
#pragma unroll
      for (int j = 0; j < 64; ++j) z[(t << 6) | (j ^ (t & 31))] = v[j];
    }
    __syncthreads();
    // every sampled row: its chunk's sign pattern against the step's chunks
    const int64_t c0 = st * a.cps;
    for (int64_t k = tid; k < a.r; k += kCscThreads) {
      const int32_t i = __ldg(a.idx + k);
      const uint32_t ci = (uint32_t)(i >> 12), wl = cswz((uint32_t)i & (kChunk - 1));
      float s = acc[k];
      for (int w = 0; w < a.cps; ++w) {
        const float zv = stage[w * kChunk + wl];
        s += (__popc(ci & (uint32_t)(c0 + w)) & 1) ? -zv : zv;
      }
      acc[k] = s;
    }
    __syncthreads();
  }
  if (a.units_per_col == 1) {
    float *out = is_b ? a.Sb : a.SA + (int64_t)col * a.ldsa;
    for (int64_t k = tid; k < a.r; k += kCscThreads) out[k] = a.scale * acc[k];
  } else {
    float *out = a.part + ((int64_t)g * (a.d + 1) + col) * a.r;
    for (int64_t k = tid; k < a.r; k += kCscThreads) out[k] = acc[k];
  }
}

// Units of a column added in unit order, scaled, written to SA / Sb.
__global__ void csc_reduce_kernel(const csc_args a) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)(a.d + 1) * a.r) return;
  const int col = (int)(e / a.r);
  const int64_t k = e % a.r;
  float s = 0.0f;
  for (int g = 0; g < a.units_per_col; ++g) s += a.part[((int64_t)g * (a.d + 1) + col) * a.r + k];
  float *out = (col == a.d) ? a.Sb : a.SA + (int64_t)col * a.ldsa;
  out[k] = a.scale * s;
}

smem_attr g_csc_attr;

}  // namespace

int sketch_csc_f32(rnnls_ctx *ctx, const int64_t *colptr, const int32_t *rowidx, const float *val, const float *b,
                   int64_t n_raw, int64_t d, int64_t r, uint64_t seed, uint64_t instance, float *SA, int64_t ldsa,
                   float *Sb, int32_t *idx) {
  const int L = log2_ceil64(n_raw);
  if (L < 12 || r > kCscMaxRows) return RNNLS_EUNSUPPORTED;
  const int64_t n = (int64_t)1 << L;
  const int cps = (int)std::min<int64_t>(kMaxChunksPerStep, n / kChunk);
  const int64_t nsteps = n / ((int64_t)cps * kChunk);
  // about four units per SM (two resident); a unit covers whole steps of one column
  int64_t upc = std::max<int64_t>(1, (4 * (int64_t)ctx->num_sms + d) / (d + 1));
  upc = std::min(upc, nsteps);
  const int64_t spu = (nsteps + upc - 1) / upc;
  upc = (nsteps + spu - 1) / spu;
  const int64_t words = n / 64;
  const size_t bytes = align_up((size_t)words * 8, 256) + align_up((size_t)r * 4, 256) +
                       (upc > 1 ? align_up((size_t)upc * (d + 1) * r * 4, 256) : 0) + 1024;
  int st = ensure_workspace(ctx, bytes);
  if (st) return st;
  ws_carver wc(ctx->ws);
  uint64_t *signs = wc.take<uint64_t>((size_t)words);
  int32_t *rows = idx ? idx : wc.take<int32_t>((size_t)r);
  float *part = upc > 1 ? wc.take<float>((size_t)upc * (d + 1) * r) : nullptr;
  cudaStream_t s = ctx->stream;
  {
    prof_scope ps(ctx, K_SAMPLE);
    st = launch_sample_iid(s, seed, instance, L, r, rows);
    if (st) return st;
    csc_signs_kernel<<<(unsigned)((words / 4 + 255) / 256 + 1), 256, 0, s>>>(seed, instance, words, signs);
  }
  csc_args a;
  a.colptr = colptr;
  a.rowidx = rowidx;
  a.val = val;
  a.b = b;
  a.n_raw = n_raw;
  a.d = (int)d;
  a.cps = cps;
  a.nsteps = nsteps;
  a.spu = spu;
  a.units_per_col = (int)upc;
  a.r = r;
  a.idx = rows;
  a.signs = signs;
  a.scale = (float)(1.0 / sqrt((double)r));
  a.SA = SA;
  a.ldsa = ldsa;
  a.Sb = Sb;
  a.part = part;
  const size_t smem = (size_t)kMaxChunksPerStep * kChunk * 4 + (size_t)r * 4;
  RNNLS_CUDA_TRY(g_csc_attr.ensure((const void *)sketch_csc_kernel, smem));
  {
    prof_scope ps(ctx, K_SKETCH_CSC);
    sketch_csc_kernel<<<(unsigned)(upc * (d + 1)), kCscThreads, smem, s>>>(a);
  }
  if (upc > 1) {
    prof_scope ps(ctx, K_REDUCE);
    const int64_t total = (d + 1) * r;
    csc_reduce_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(a);
  }
  return cudaGetLastError() == cudaSuccess ? RNNLS_OK : RNNLS_ECUDA;
}

}  // namespace rnnls
