// solve.cu -- the small NNLS of Alg. 1 step 5 on the sketch, by the
// Lawson-Hanson active-set method (Sec. 2.2) on the quadratic-programming
// form Q = SA'SA, q = SA'Sb (Sec. 3.4), plus the full-data objective of
// Definition 1.
//
// Precision plan for GB300 (whose FP64 rate is a small fraction of FP32):
//   - Gram of FP32 sketches: on the tensor cores from an exact split of
//     every column into six 8-bit slices (gram_tc.cu); of FP64 sketches:
//     plain FP64 sums.
//   - Lawson-Hanson: an FP32 inverse of the equilibrated passive block
//     D Q_PP D (D = diag(Q)^-1/2) is kept up to date by bordering (adding a
//     column) and Schur-complement downdates (dropping one); every passive
//     solve is refined in float-float arithmetic against the accurate Q, and
//     the dual vector w = q - Qx is evaluated in float-float.  All decisions
//     (argmax of w, tolerance, sign of z, interpolation step) use these
//     refined values and the same rules as the FP64 reference algorithm.
#include <algorithm>
#include <climits>
#include <cstring>
#include <vector>

#include "kernels.h"
#include "launch_attr.h"

namespace rnnls {

namespace {


constexpr int kGT = 32;         // Gram tile
#ifndef RNNLS_LH_THREADS
#define RNNLS_LH_THREADS 256
#endif
constexpr int kLHThreads = RNNLS_LH_THREADS;  // Lawson-Hanson block

// ---------------------------------------------------------------------------
// FP64 Gram of X = [S | s] (m x (d+1)) in tiles of 32 x 32, split over rows
// (the FP32 Gram runs on the tensor cores, gram_tc.cu).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tile_coords(int t, int T, int &ti, int &tj) {
  ti = 0;
  while (t >= T - ti) {
    t -= T - ti;
    ++ti;
  }
  tj = ti + t;
}

template <typename T>
__device__ __forceinline__ const T *gram_col(const T *S, int64_t lds, const T *s, int d, int g) {
  return (g < d) ? S + (int64_t)g * lds : (g == d ? s : nullptr);
}
__global__ void __launch_bounds__(256) gram_f64_kernel(const double *__restrict__ S, int64_t lds,
                                                       const double *__restrict__ s, int64_t m, int d, int T,
                                                       int64_t rows_per_split, double *__restrict__ part) {
  __shared__ double Xi[kGT][kGT + 1];
  __shared__ double Xj[kGT][kGT + 1];
  int ti, tj;
  tile_coords(blockIdx.x, T, ti, tj);
  const int ntiles = T * (T + 1) / 2;
  const int64_t k0 = (int64_t)blockIdx.y * rows_per_split;
  const int64_t k1 = min(m, k0 + rows_per_split);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  for (int64_t kb = k0; kb < k1; kb += kGT) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = threadIdx.x + 256 * q;
      const int kk = e & 31, cc = e >> 5;
      const int64_t k = kb + kk;
      const double *ci = gram_col(S, lds, s, d, ti * kGT + cc);
      const double *cj = gram_col(S, lds, s, d, tj * kGT + cc);
      Xi[kk][cc] = (ci && k < k1) ? ci[k] : 0.0;
      Xj[kk][cc] = (cj && k < k1) ? cj[k] : 0.0;
    }
    __syncthreads();
    for (int kk = 0; kk < kGT; ++kk) {
      const double a0 = Xi[kk][2 * ty], a1 = Xi[kk][2 * ty + 1];
      const double b0 = Xj[kk][2 * tx], b1 = Xj[kk][2 * tx + 1];
      acc[0][0] += a0 * b0;
      acc[0][1] += a0 * b1;
      acc[1][0] += a1 * b0;
      acc[1][1] += a1 * b1;
    }
    __syncthreads();
  }
  double *out = part + ((int64_t)blockIdx.y * ntiles + blockIdx.x) * (kGT * kGT);
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int c = 0; c < 2; ++c) out[(2 * ty + a) * kGT + 2 * tx + c] = acc[a][c];
}

// Sum the row splits (fixed order), mirror, and split into float pairs.
__global__ void gram_reduce_kernel(const double *__restrict__ part, int splits, int d, int T,
                                   double *__restrict__ Qd, float *__restrict__ Qhi, float *__restrict__ Qlo) {
  const int D1 = d + 1;
  const int ntiles = T * (T + 1) / 2;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)D1 * D1;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / D1), j = (int)(e % D1);
    if (i > j) continue;
    const int ti = i / kGT, tj = j / kGT;
    // index of tile (ti, tj) in the upper-triangular enumeration
    const int t = ti * T - ti * (ti - 1) / 2 + (tj - ti);
    const int pos = (i % kGT) * kGT + (j % kGT);
    double v = 0.0;
    for (int sp = 0; sp < splits; ++sp) v += part[((int64_t)sp * ntiles + t) * (kGT * kGT) + pos];
    const float h = (float)v;
    const float l = (float)(v - (double)h);
    Qd[(int64_t)i * D1 + j] = v;
    Qd[(int64_t)j * D1 + i] = v;
    Qhi[(int64_t)i * D1 + j] = h;
    Qhi[(int64_t)j * D1 + i] = h;
    Qlo[(int64_t)i * D1 + j] = l;
    Qlo[(int64_t)j * D1 + i] = l;
  }
}

// ||S||_1 = max_j sum_k |S_kj| (compensated), one warp per column.
template <typename T>
__global__ void colabs_kernel(const T *__restrict__ S, int64_t lds, int64_t m, int d, double *__restrict__ out) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= d) return;
  const T *c = S + (int64_t)warp * lds;
  double acc = 0.0;
  dot2 a2;
  for (int64_t k = lane; k < m; k += 32) {
    if (sizeof(T) == 8)
      acc += fabs((double)c[k]);
    else
      a2.add(fabsf((float)c[k]));
  }
  if (sizeof(T) == 4) {
    const ff v = a2.value();
    acc = (double)v.hi + (double)v.lo;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) out[warp] = acc;
}

// ---------------------------------------------------------------------------
// Lawson-Hanson block.
// ---------------------------------------------------------------------------
struct lh_job {
  const double *Qd;  // Gram of [S | targets], leading dimension ldq: Q = leading d x d block,
  const float *Qhi;  // q = column qcol, ||s||^2 = entry (qcol, qcol)
  const float *Qlo;
  int ldq, qcol;
  const double *colabs;  // d column 1-norms of the sketch
  int64_t r;
  int d;
  double *x;
  rnnls_info *info;
  int q_smem;  // 1: copy Q into shared memory (it fits); 0: read it from global memory
  float *Bg;   // non-null: the passive-block inverse lives here (global, odd_ld(d) x d), not in shared memory
};

// float-float dot accumulator with float-float inputs (Dot2 on the leading
// products, first-order terms for the low parts).
struct dotff {
  float s, c;
  __device__ __forceinline__ dotff() : s(0.0f), c(0.0f) {}
  __device__ __forceinline__ void init(ff a) {
    s = a.hi;
    c = a.lo;
  }
  __device__ __forceinline__ void add_prod(ff a, ff b) {
    const ff p = two_prod(a.hi, b.hi);
    const ff t = two_sum(s, p.hi);
    s = t.hi;
    float e = __fadd_rn(t.lo, p.lo);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    c = __fadd_rn(c, e);
  }
  __device__ __forceinline__ void sub_prod(ff a, ff b) { add_prod(ff_neg(a), b); }
  __device__ __forceinline__ ff value() const { return fast_two_sum(s, c); }
};

struct lh_shared {
  uint32_t wkey[kLHThreads / 32];  // per-warp candidate keys / partial sums (fast path)
  int widx[kLHThreads / 32];
  float wsum[kLHThreads / 32];
  int p;       // passive count
  int t;       // candidate / chosen index
  int status;
  int flag;
  float fscal;
  ff ffscal;
  int ired[kLHThreads / 32];
  ff vred[kLHThreads / 32];
  float fred[kLHThreads / 32];
};

// block sum of floats (all threads get the result)
template <int NT>
__device__ float block_sum_f(float v, lh_shared &sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh.fred[warp] = v;
  __syncthreads();
  float t = 0.0f;
#pragma unroll
  for (int q = 0; q < NT / 32; ++q) t += sh.fred[q];
  return t;
}

template <int NT>
__device__ ff block_sum_ff(ff v, lh_shared &sh) {
  for (int o = 16; o > 0; o >>= 1) {
    ff u{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
    v = ff_add(v, u);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh.vred[warp] = v;
  __syncthreads();
  ff t{0.0f, 0.0f};
#pragma unroll
  for (int q = 0; q < NT / 32; ++q) t = ff_add(t, sh.vred[q]);
  return t;
}

// argmax of (valid, value) with ties to the smallest index; returns -1 if none
template <int NT>
__device__ int block_argmax_ff(bool valid, ff v, int idx, lh_shared &sh, ff &best) {
  int bi = valid ? idx : -1;
  ff bv = v;
  for (int o = 16; o > 0; o >>= 1) {
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    const ff ov{__shfl_xor_sync(0xffffffffu, bv.hi, o), __shfl_xor_sync(0xffffffffu, bv.lo, o)};
    if (oi >= 0 && (bi < 0 || ff_gt(ov, bv) || (!ff_gt(bv, ov) && oi < bi))) {
      bi = oi;
      bv = ov;
    }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) {
    sh.ired[warp] = bi;
    sh.vred[warp] = bv;
  }
  __syncthreads();
  bi = -1;
#pragma unroll
  for (int q = 0; q < NT / 32; ++q) {
    const int oi = sh.ired[q];
    const ff ov = sh.vred[q];
    if (oi >= 0 && (bi < 0 || ff_gt(ov, bv) || (!ff_gt(bv, ov) && oi < bi))) {
      bi = oi;
      bv = ov;
    }
  }
  best = bv;
  return bi;
}

// Order-preserving map of a float onto unsigned integers.
__device__ __forceinline__ uint32_t fkey(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// Warp-wide argmax of float-float values with ties to the smallest index
// (lanes without a candidate pass idx < 0); -1 if no lane has one.
__device__ __forceinline__ int warp_argmax_ff(ff v, int idx, ff &best) {
  const bool valid = idx >= 0;
  const uint32_t kh = valid ? fkey(v.hi) : 0u;
  const uint32_t mh = __reduce_max_sync(0xffffffffu, kh);
  const uint32_t kl = (valid && kh == mh) ? fkey(v.lo) : 0u;
  const uint32_t ml = __reduce_max_sync(0xffffffffu, kl);
  const uint32_t ci = (valid && kh == mh && kl == ml) ? (uint32_t)idx : 0xffffffffu;
  const uint32_t mi = __reduce_min_sync(0xffffffffu, ci);
  const uint32_t win = __ballot_sync(0xffffffffu, ci == mi && mi != 0xffffffffu);
  const int src = win ? __ffs(win) - 1 : 0;
  best.hi = __shfl_sync(0xffffffffu, v.hi, src);
  best.lo = __shfl_sync(0xffffffffu, v.lo, src);
  return (mi == 0xffffffffu) ? -1 : (int)mi;
}

struct lh_vecs {
  float *B;           // FP32 inverse of D Q_PP D, slot indexed, leading dimension ldB (odd)
  int ldB;
  const float *Qh, *Ql;  // Q (d+1 x d+1) as float pairs, leading dimension ldQ (shared memory when it fits)
  int ldQ;
  float *Dsc;         // d: D_jj = Q_jj^(-1/2)
  float *qh;          // d: D q in FP32
  ff *qv;             // d: q
  ff *w;              // d: dual w = q - Q x
  int *varslot;       // d: slot of variable j, or -1
  unsigned char *rej; // d: rejected in the current selection
  int *slotvar;       // d+1: variable of slot s
  ff *xs, *zs, *res;  // d+1: x, z and residual per slot
  float *f1, *f2, *f3;  // d+1 FP32 temporaries
};

__host__ __device__ __forceinline__ int odd_ld(int d) { return (d % 2 == 1) ? d : d + 1; }

// Threads cooperating on one output of a length-n dot product (power of 2,
// consecutive lanes of one warp): more threads for shorter outputs.
__device__ __forceinline__ int lanes_per_row(int rows) {
  return (rows <= 32) ? 8 : (rows <= 64 ? 4 : (rows <= 128 ? 2 : 1));
}

// y[s] = sum_q B[s][q] g[q] for s < p (B symmetric: lanes of row s read
// column s, rows of B at odd stride, so a warp touches distinct banks)
template <int NT>
__device__ __forceinline__ void apply_B(const lh_vecs &V, int p, const float *g, float *y) {
  const int tpr = lanes_per_row(p);
  const int part = threadIdx.x & (tpr - 1);
  for (int base = 0; base < p; base += NT / tpr) {
    const int s = base + threadIdx.x / tpr;
    const bool ok = s < p;
    float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
    if (ok) {
      int q = part;
      for (; q + 3 * tpr < p; q += 4 * tpr) {
        a0 = fmaf(V.B[q * V.ldB + s], g[q], a0);
        a1 = fmaf(V.B[(q + tpr) * V.ldB + s], g[q + tpr], a1);
        a2 = fmaf(V.B[(q + 2 * tpr) * V.ldB + s], g[q + 2 * tpr], a2);
        a3 = fmaf(V.B[(q + 3 * tpr) * V.ldB + s], g[q + 3 * tpr], a3);
      }
      for (; q < p; q += tpr) a0 = fmaf(V.B[q * V.ldB + s], g[q], a0);
    }
    float a = (a0 + a1) + (a2 + a3);
    for (int o = 1; o < tpr; o <<= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (ok && part == 0) y[s] = a;
  }
}

// w_j = q_j - sum_s Q[j][slotvar[s]] x_s for every j (float-float)
template <int NT>
__device__ __noinline__ void compute_w(const lh_vecs &V, int d, int p) {
  const int tpj = lanes_per_row(d);
  const int part = threadIdx.x & (tpj - 1);
  for (int base = 0; base < d; base += NT / tpj) {
    const int j = base + threadIdx.x / tpj;
    const bool ok = j < d;
    dotff a0, a1;
    if (ok) {
      if (part == 0) a0.init(V.qv[j]);
      int s = part;
      for (; s + tpj < p; s += 2 * tpj) {
        const int e0 = V.slotvar[s] * V.ldQ + j, e1 = V.slotvar[s + tpj] * V.ldQ + j;
        a0.sub_prod(ff{V.Qh[e0], V.Ql[e0]}, V.xs[s]);
        a1.sub_prod(ff{V.Qh[e1], V.Ql[e1]}, V.xs[s + tpj]);
      }
      if (s < p) {
        const int e0 = V.slotvar[s] * V.ldQ + j;
        a0.sub_prod(ff{V.Qh[e0], V.Ql[e0]}, V.xs[s]);
      }
    }
    ff a = ff_add(a0.value(), a1.value());
    for (int o = 1; o < tpj; o <<= 1) {
      const ff u{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
      a = ff_add(a, u);
    }
    if (ok && part == 0) V.w[j] = a;
  }
}

// Fast path, phase 1: FP32 dual for every j and each warp's best candidate
// (largest w_j outside P, ties to the smallest j) into sh.wkey / sh.widx.
template <int NT>
__device__ __forceinline__ void dual_and_warp_best(const lh_vecs &V, int d, int p, lh_shared &sh) {
  const int tpj = lanes_per_row(d);
  const int part = threadIdx.x & (tpj - 1);
  uint32_t bkey = 0u;
  uint32_t bidx = 0xffffffffu;
  for (int base = 0; base < d; base += NT / tpj) {
    const int j = base + threadIdx.x / tpj;
    const bool ok = j < d;
    float a[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    if (ok) {
      // eight independent loads in flight (Q sits in L2 for large d)
      int s = part;
      for (; s + 7 * tpj < p; s += 8 * tpj) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int su = s + u * tpj;
          a[u] = fmaf(-V.Qh[V.slotvar[su] * V.ldQ + j], V.xs[su].hi, a[u]);
        }
      }
      for (; s < p; s += tpj) a[0] = fmaf(-V.Qh[V.slotvar[s] * V.ldQ + j], V.xs[s].hi, a[0]);
    }
    float acc = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
    for (int o = 1; o < tpj; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (ok && part == 0) {
      const float wj = V.qv[j].hi + acc;
      V.w[j] = ff{wj, 0.0f};
      if (V.varslot[j] < 0) {
        const uint32_t k = fkey(wj);
        if (bidx == 0xffffffffu || k > bkey) {  // j increases along this lane: first wins ties
          bkey = k;
          bidx = (uint32_t)j;
        }
      }
    }
  }
  const uint32_t mk = __reduce_max_sync(0xffffffffu, bidx != 0xffffffffu ? bkey : 0u);
  const uint32_t mi = __reduce_min_sync(0xffffffffu, (bidx != 0xffffffffu && bkey == mk) ? bidx : 0xffffffffu);
  if ((threadIdx.x & 31) == 0) {
    sh.wkey[threadIdx.x >> 5] = mk;
    sh.widx[threadIdx.x >> 5] = (int)mi;
  }
}

// After the barrier: the block's candidate from the per-warp winners.
template <int NT>
__device__ __forceinline__ int merge_warp_best(const lh_shared &sh) {
  uint32_t bk = 0u;
  int bi = -1;
  for (int q = 0; q < NT / 32; ++q) {
    const int i = sh.widx[q];
    if (i < 0) continue;
    const uint32_t k = sh.wkey[q];
    if (bi < 0 || k > bk || (k == bk && i < bi)) {
      bk = k;
      bi = i;
    }
  }
  return bi;
}

// Fast path, phase 2: v = B u with u_s = D_s Q[v_s][t] D_t, v into f3,
// per-warp partial sums of u'v into sh.wsum.  D_s Q[v_s][t] is formed once
// per slot into f1 (row t of Q may sit in L2; f1 is free here), so the
// product reads shared memory only.
template <int NT>
__device__ __forceinline__ void bordered_v(const lh_vecs &V, int p, int t, float dt, lh_shared &sh) {
  const int tpr = lanes_per_row(p);
  const int part = threadIdx.x & (tpr - 1);
  const float *qt = V.Qh + t * V.ldQ;
  for (int q = threadIdx.x; q < p; q += NT) {
    const int v = V.slotvar[q];
    V.f1[q] = qt[v] * V.Dsc[v];
  }
  __syncthreads();
  const float *u = V.f1;
  float uv = 0.0f;
  for (int base = 0; base < p; base += NT / tpr) {
    const int s = base + threadIdx.x / tpr;
    const bool ok = s < p;
    float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
    if (ok) {
      int q = part;
      for (; q + 3 * tpr < p; q += 4 * tpr) {
        a0 = fmaf(V.B[q * V.ldB + s], u[q], a0);
        a1 = fmaf(V.B[(q + tpr) * V.ldB + s], u[q + tpr], a1);
        a2 = fmaf(V.B[(q + 2 * tpr) * V.ldB + s], u[q + 2 * tpr], a2);
        a3 = fmaf(V.B[(q + 3 * tpr) * V.ldB + s], u[q + 3 * tpr], a3);
      }
      for (; q < p; q += tpr) a0 = fmaf(V.B[q * V.ldB + s], u[q], a0);
    }
    float a = ((a0 + a1) + (a2 + a3)) * dt;
    for (int o = 1; o < tpr; o <<= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (ok && part == 0) {
      V.f3[s] = a;
      uv = fmaf(u[s] * dt, a, uv);
    }
  }
  for (int o = 16; o > 0; o >>= 1) uv += __shfl_xor_sync(0xffffffffu, uv, o);
  if ((threadIdx.x & 31) == 0) sh.wsum[threadIdx.x >> 5] = uv;
}

// The entering candidate: argmax of w over j outside P and not rejected
// (ties to the smallest j).  Warp 0 decides; everyone gets the result.
template <int NT>
__device__ __noinline__ int select_candidate(const lh_vecs &V, int d, lh_shared &sh, ff &best) {
  if (threadIdx.x < 32) {
    ff bv{0.0f, 0.0f};
    int bj = -1;
    for (int j = threadIdx.x; j < d; j += 32) {
      if (V.varslot[j] < 0 && !V.rej[j]) {
        const ff wj = V.w[j];
        if (bj < 0 || ff_gt(wj, bv)) {
          bv = wj;
          bj = j;
        }
      }
    }
    ff b;
    const int t = warp_argmax_ff(bv, bj, b);
    if (threadIdx.x == 0) {
      sh.t = t;
      sh.ffscal = b;
    }
  }
  __syncthreads();
  best = sh.ffscal;
  return sh.t;
}

// The interpolation step: over slots with z <= 0, the minimum of
// x/(x - z) (ties to the smallest variable).  Warp 0 decides.
template <int NT>
__device__ __noinline__ int select_alpha(const lh_vecs &V, int p, lh_shared &sh, ff &amin) {
  if (threadIdx.x < 32) {
    ff bv{0.0f, 0.0f};
    int bj = -1;
    for (int s = threadIdx.x; s < p; s += 32) {
      if (ff_le0(V.zs[s])) {
        const int v = V.slotvar[s];
        const ff xv = V.xs[s];
        const ff a = ff_div(xv, ff_sub(xv, V.zs[s]));
        if (bj < 0 || ff_lt(a, bv) || (!ff_gt(a, bv) && v < bj)) {
          bv = a;
          bj = v;
        }
      }
    }
    ff b;
    const int t = warp_argmax_ff(ff_neg(bv), bj, b);
    if (threadIdx.x == 0) {
      sh.t = t;
      sh.ffscal = ff_neg(b);
    }
  }
  __syncthreads();
  amin = sh.ffscal;
  return sh.t;
}

// res_i = q_{v_i} - sum_q Q[v_i][v_q] z_q for slots i < np (float-float).
// Q is stored bitwise symmetric, so slot i reads column v_i of the rows v_q:
// the slots of one warp then read within the same rows.
template <int NT>
__device__ __noinline__ void residual_slots(const lh_vecs &V, int np) {
  const int tpr = lanes_per_row(np);
  const int part = threadIdx.x & (tpr - 1);
  for (int base = 0; base < np; base += NT / tpr) {
    const int i = base + threadIdx.x / tpr;
    const bool ok = i < np;
    dotff a0, a1;
    if (ok) {
      const int vi = V.slotvar[i];
      if (part == 0) a0.init(V.qv[vi]);
      int q = part;
      for (; q + tpr < np; q += 2 * tpr) {
        const int e0 = V.slotvar[q] * V.ldQ + vi, e1 = V.slotvar[q + tpr] * V.ldQ + vi;
        a0.sub_prod(ff{V.Qh[e0], V.Ql[e0]}, V.zs[q]);
        a1.sub_prod(ff{V.Qh[e1], V.Ql[e1]}, V.zs[q + tpr]);
      }
      if (q < np) {
        const int e0 = V.slotvar[q] * V.ldQ + vi;
        a0.sub_prod(ff{V.Qh[e0], V.Ql[e0]}, V.zs[q]);
      }
    }
    ff a = ff_add(a0.value(), a1.value());
    for (int o = 1; o < tpr; o <<= 1) {
      const ff u{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
      a = ff_add(a, u);
    }
    if (ok && part == 0) V.res[i] = a;
  }
}

// Passive solve z = Q_PP^{-1} q_P for slots 0..np-1.  Without bordering, B
// is the inverse of D Q_PP D.  With bordering, B covers slots 0..np-2 and
// the candidate in slot np-1 enters through v = f3 = B u and the Schur
// value sc.  Unless `have_initial` (zs already holds an FP32 estimate), one
// FP32 solve comes first; then `iters` float-float refinement steps, and
// (iters > 0) more while the largest relative correction over the slots
// still halves from one step to the next and exceeds 2^-44 (at most 60
// more: the FP32 inverse contracts the error by about cond(D Q_PP D) 2^-24
// per step, so ill-conditioned blocks need more; once the corrections stop
// shrinking, float-float rounding has been reached).
constexpr int kMaxExtraRefine = 60;
template <int NT>
__device__ __noinline__ void passive_solve(const lh_vecs &V, lh_shared &sh, int np, bool bordered, float sc,
                                           int iters, bool have_initial = false) {
  __shared__ unsigned int corr_max[3];  // per step (rotating): largest |dz| / |z| as float bits
  const int pb = bordered ? np - 1 : np;
  const int cap = iters > 0 ? iters + kMaxExtraRefine : 0;
  if (threadIdx.x == 0) corr_max[0] = corr_max[1] = corr_max[2] = 0u;
  float prev = INFINITY;
  for (int step = have_initial ? 1 : 0; step <= cap; ++step) {
    if (step > 0) {
      residual_slots<NT>(V, np);
      __syncthreads();
    }
    for (int s = threadIdx.x; s < np; s += NT) {
      const int v = V.slotvar[s];
      V.f1[s] = (step == 0) ? V.qh[v] : V.res[s].hi * V.Dsc[v];
    }
    __syncthreads();
    apply_B<NT>(V, pb, V.f1, V.f2);
    __syncthreads();
    if (bordered) {
      float part = 0.0f;
      for (int s = threadIdx.x; s < pb; s += NT) part = fmaf(V.f3[s], V.f1[s], part);
      const float vg = block_sum_f<NT>(part, sh);
      const float yt = (V.f1[pb] - vg) / sc;
      for (int s = threadIdx.x; s < pb; s += NT) V.f2[s] = fmaf(-V.f3[s], yt, V.f2[s]);
      if (threadIdx.x == 0) V.f2[pb] = yt;
      __syncthreads();
    }
    float mx = 0.0f;
    for (int s = threadIdx.x; s < np; s += NT) {
      const float dz = V.f2[s] * V.Dsc[V.slotvar[s]];
      V.zs[s] = (step == 0) ? ff_make(dz) : ff_add(V.zs[s], ff_make(dz));
      mx = fmaxf(mx, fabsf(dz) / fmaxf(fabsf(V.zs[s].hi), 1e-30f));
    }
    // the slot two steps ahead was last read two barriers ago: clear it now
    if (threadIdx.x == 0) corr_max[(step + 1) % 3] = 0u;
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&corr_max[step % 3], __float_as_uint(mx));
    __syncthreads();
    const float cm = __uint_as_float(corr_max[step % 3]);
    // past the fixed steps: stop once converged or no longer converging
    if (step >= iters && step > 0 && (cm <= 0x1p-44f || cm > 0.5f * prev)) break;
    prev = cm;
  }
  __syncthreads();  // every thread has read the last step's maximum before a later call clears it
}

// Drop slot s (Schur-complement downdate of B), then move the last slot
// into s (B row/column, Q row, x, slot maps).  p = count before the drop.
template <int NT>
__device__ __noinline__ void drop_slot(const lh_vecs &V, int d, int s, int p) {
  const float bss = V.B[(int64_t)s * V.ldB + s];
  for (int q = threadIdx.x; q < p; q += NT) V.f1[q] = V.B[(int64_t)q * V.ldB + s];
  __syncthreads();
  const float ibss = 1.0f / bss;
  {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int a = warp; a < p; a += NT / 32) {
      const float fa = V.f1[a] * ibss;
      for (int c = lane; c < p; c += 32) V.B[a * V.ldB + c] = fmaf(-fa, V.f1[c], V.B[a * V.ldB + c]);
    }
  }
  __syncthreads();
  const int last = p - 1;
  if (s != last) {
    for (int q = threadIdx.x; q < p; q += NT) V.f1[q] = V.B[(int64_t)last * V.ldB + q];
    __syncthreads();
    for (int q = threadIdx.x; q < p; q += NT) {
      if (q == s) continue;
      const float val = V.f1[q];
      const int qq = (q == last) ? s : q;
      V.B[(int64_t)s * V.ldB + qq] = val;
      V.B[(int64_t)qq * V.ldB + s] = val;
    }
    if (threadIdx.x == 0) {
      const int v = V.slotvar[last];
      V.slotvar[s] = v;
      V.varslot[v] = s;
      V.xs[s] = V.xs[last];
    }
  }
  __syncthreads();
}

struct lh_layout {
  size_t bytes;
  size_t off_B, off_Qh, off_Ql, off_Dsc, off_qh, off_qv, off_w, off_varslot, off_rej, off_slotvar, off_xs, off_zs,
      off_res, off_f1, off_f2, off_f3;
};

__host__ __device__ inline lh_layout lh_make_layout(int d, bool q_smem, bool b_smem = true) {
  lh_layout L;
  size_t o = 0;
  auto take = [&](size_t b) {
    const size_t at = o;
    o += (b + 15) & ~(size_t)15;
    return at;
  };
  const int ldB = odd_ld(d), ldQ = odd_ld(d + 1);
  L.off_B = b_smem ? take((size_t)ldB * d * 4) : 0;
  L.off_Qh = q_smem ? take((size_t)(d + 1) * ldQ * 4) : 0;
  L.off_Ql = q_smem ? take((size_t)(d + 1) * ldQ * 4) : 0;
  L.off_Dsc = take((size_t)d * 4);
  L.off_qh = take((size_t)d * 4);
  L.off_qv = take((size_t)d * 8);
  L.off_w = take((size_t)d * 8);
  L.off_varslot = take((size_t)d * 4);
  L.off_rej = take((size_t)d);
  L.off_slotvar = take((size_t)(d + 1) * 4);
  L.off_xs = take((size_t)(d + 1) * 8);
  L.off_zs = take((size_t)(d + 1) * 8);
  L.off_res = take((size_t)(d + 1) * 8);
  L.off_f1 = take((size_t)(d + 1) * 4);
  L.off_f2 = take((size_t)(d + 1) * 4);
  L.off_f3 = take((size_t)(d + 1) * 4);
  L.bytes = o;
  return L;
}

template <int NT>
__device__ void lh_block(const lh_job &jb, unsigned char *smem_raw, lh_shared &sh, int max_outer, int max_inner) {
  const int d = jb.d;
  const int D1 = d + 1;
  const int tid = threadIdx.x;
  const bool q_smem = jb.q_smem;
  const lh_layout L = lh_make_layout(d, q_smem, jb.Bg == nullptr);
  lh_vecs V;
  V.ldB = odd_ld(d);
  V.B = jb.Bg ? jb.Bg : (float *)(smem_raw + L.off_B);
  if (q_smem) {
    float *qh = (float *)(smem_raw + L.off_Qh);
    float *ql = (float *)(smem_raw + L.off_Ql);
    const int ld = odd_ld(D1);
    for (int e = tid; e < D1 * D1; e += NT) {
      const int i = e / D1, j = e - i * D1;
      const int64_t src = (int64_t)(i < d ? i : jb.qcol) * jb.ldq + (j < d ? j : jb.qcol);
      qh[i * ld + j] = jb.Qhi[src];
      ql[i * ld + j] = jb.Qlo[src];
    }
    V.Qh = qh;
    V.Ql = ql;
    V.ldQ = ld;
  } else {
    V.Qh = jb.Qhi;  // read at rows and columns < d only
    V.Ql = jb.Qlo;
    V.ldQ = jb.ldq;
  }
  V.Dsc = (float *)(smem_raw + L.off_Dsc);
  V.qh = (float *)(smem_raw + L.off_qh);
  V.qv = (ff *)(smem_raw + L.off_qv);
  V.w = (ff *)(smem_raw + L.off_w);
  V.varslot = (int *)(smem_raw + L.off_varslot);
  V.rej = (unsigned char *)(smem_raw + L.off_rej);
  V.slotvar = (int *)(smem_raw + L.off_slotvar);
  V.xs = (ff *)(smem_raw + L.off_xs);
  V.zs = (ff *)(smem_raw + L.off_zs);
  V.res = (ff *)(smem_raw + L.off_res);
  V.f1 = (float *)(smem_raw + L.off_f1);
  V.f2 = (float *)(smem_raw + L.off_f2);
  V.f3 = (float *)(smem_raw + L.off_f3);

  // tolerance 10 eps ||S||_1 max(r, d) ||s||_2 (FP64 scalar work, once)
  __shared__ double tol_d;
  if (tid == 0) {
    double n1 = 0.0;
    for (int j = 0; j < d; ++j) n1 = fmax(n1, jb.colabs[j]);
    const double ss = jb.Qd[(int64_t)jb.qcol * jb.ldq + jb.qcol];
    tol_d = 10.0 * 2.220446049250313e-16 * n1 * (double)max(jb.r, (int64_t)d) * sqrt(fmax(ss, 0.0));
    sh.p = 0;
    sh.status = RNNLS_OK;
  }
  __syncthreads();
  const ff tol = ff_from_double(tol_d);
  {
    int bad = 0;
    for (int64_t e = tid; e < (int64_t)D1 * D1; e += NT) {
      const int64_t i = e / D1, j = e - i * D1;
      bad |= !isfinite(jb.Qd[(i < d ? i : jb.qcol) * jb.ldq + (j < d ? j : jb.qcol)]);
    }
    if (__syncthreads_or(bad)) {
      for (int j = tid; j < d; j += NT) jb.x[j] = 0.0;
      if (tid == 0 && jb.info) {
        rnnls_info inf;
        inf.status = RNNLS_ENONFINITE;
        inf.outer_iters = inf.inner_iters = inf.passive_count = 0;
        inf.tol = tol_d;
        inf.dual_max = 0.0;
        inf.objective = 0.0;
        inf.accurate_mode = 0;
        inf.reserved = 0;
        *jb.info = inf;
      }
      return;
    }
  }
  for (int j = tid; j < d; j += NT) {
    const double qjj = jb.Qd[(int64_t)j * jb.ldq + j];
    const float dj = (qjj > 0.0) ? (float)(1.0 / sqrt(qjj)) : 0.0f;
    V.Dsc[j] = dj;
    const ff qj{jb.Qhi[(int64_t)j * jb.ldq + jb.qcol], jb.Qlo[(int64_t)j * jb.ldq + jb.qcol]};
    V.qv[j] = qj;
    V.qh[j] = qj.hi * dj;
    V.varslot[j] = -1;
  }
  __syncthreads();

  // Iterations run in FP32 (inverse of the equilibrated passive block,
  // FP32 dual).  When they stop, the result is verified in float-float: a
  // refined passive solve must be positive and the float-float dual must
  // not exceed tol off the passive set.  If either check fails the method
  // continues from there with every passive solve refined and the dual in
  // float-float, exactly as the FP64 algorithm would.
  int outer = 0, inner = 0;
  bool accurate = false;
  int accurate_mode = 0;  // which end-point check switched to the accurate mode
  bool go_inner = false;
  for (;;) {
    bool need_inner = true;
    if (!go_inner) {
      bool accepted = false;
      int t = -1;
      ff best{0.0f, 0.0f};
      if (accurate) {
        compute_w<NT>(V, d, sh.p);
        for (int j = tid; j < d; j += NT) V.rej[j] = 0;
        __syncthreads();
        t = select_candidate<NT>(V, d, sh, best);
      } else {
        dual_and_warp_best<NT>(V, d, sh.p, sh);
        for (int j = tid; j < d; j += NT) V.rej[j] = 0;
        __syncthreads();
        t = merge_warp_best<NT>(sh);
        if (t >= 0) best = V.w[t];
      }
      for (;;) {
        if (t < 0 || !ff_gt(best, tol)) break;
        const int p = sh.p;
        const float dt = V.Dsc[t];
        // v = B u and the Schur value sc = 1 - u'v (fixed summation order)
        bordered_v<NT>(V, p, t, dt, sh);
        __syncthreads();
        float uv = 0.0f;
        for (int q = 0; q < NT / 32; ++q) uv += sh.wsum[q];
        const float sc = 1.0f - uv;
        if (!(sc > 1e-13f) || dt == 0.0f) {
          if (tid == 0) V.rej[t] = 1;
          __syncthreads();
          t = select_candidate<NT>(V, d, sh, best);
          continue;
        }
        // x_P solves the current passive set, so the bordered solution is
        // z_t = D_t^2 w_t / sc > 0 and z_P = x_P - D_P v (D_t w_t / sc)
        const float yt = dt * best.hi / sc;
        const float isc = 1.0f / sc;
        int neg = 0;
        for (int s2 = tid; s2 < p; s2 += NT) {
          const float zf = fmaf(-V.Dsc[V.slotvar[s2]] * V.f3[s2], yt, V.xs[s2].hi);
          V.zs[s2] = ff_make(zf);
          neg |= (zf <= 0.0f) ? 1 : 0;
        }
        if (tid == 0) {
          V.zs[p] = ff_make(dt * yt);
          V.slotvar[p] = t;
        }
        if (accurate) {
          __syncthreads();
          passive_solve<NT>(V, sh, p + 1, true, sc, 2, true);
          if (!ff_gt0(V.zs[p])) {
            if (tid == 0) V.rej[t] = 1;
            __syncthreads();
            t = select_candidate<NT>(V, d, sh, best);
            continue;
          }
          neg = 0;
          for (int s2 = tid; s2 < p; s2 += NT) neg |= ff_le0(V.zs[s2]) ? 1 : 0;
        }
        // commit the bordered inverse: B += v v'/sc, new row/col -v/sc, corner 1/sc
        {
          const int warp = tid >> 5, lane = tid & 31;
          for (int a = warp; a < p; a += NT / 32) {
            const float fa = V.f3[a] * isc;
            for (int c = lane; c < p; c += 32) V.B[a * V.ldB + c] = fmaf(fa, V.f3[c], V.B[a * V.ldB + c]);
          }
        }
        for (int s2 = tid; s2 < p; s2 += NT) {
          V.B[s2 * V.ldB + p] = -V.f3[s2] * isc;
          V.B[p * V.ldB + s2] = -V.f3[s2] * isc;
        }
        if (tid == 0) {
          V.B[p * V.ldB + p] = isc;
          V.varslot[t] = p;
          V.xs[p] = ff{0.0f, 0.0f};
          sh.p = p + 1;
        }
        neg = __syncthreads_or(neg);
        accepted = true;
        need_inner = (neg != 0);
        if (!neg) {
          // x = z on the new passive set: swap the vectors instead of copying
          ff *tmp = V.xs;
          V.xs = V.zs;
          V.zs = tmp;
        }
        break;
      }
      if (!accepted) {
        if (accurate) break;
        // verify the FP32 end point
        const int p = sh.p;
        if (p > 0) passive_solve<NT>(V, sh, p, false, 0.0f, 3);
        int neg = 0;
        for (int s = tid; s < p; s += NT) neg |= ff_le0(V.zs[s]) ? 1 : 0;
        if (__syncthreads_or(neg)) {
          accurate = true;
          accurate_mode = 1;
          go_inner = true;
          continue;
        }
        for (int s = tid; s < p; s += NT) V.xs[s] = V.zs[s];
        __syncthreads();
        compute_w<NT>(V, d, p);
        __syncthreads();
        int up = 0;
        for (int j = tid; j < d; j += NT) up |= (V.varslot[j] < 0 && ff_gt(V.w[j], tol)) ? 1 : 0;
        if (__syncthreads_or(up)) {
          accurate = true;
          accurate_mode = 2;
          continue;
        }
        break;
      }
      if (outer >= max_outer) {
        if (tid == 0) sh.status = RNNLS_EMAXITER;
        __syncthreads();
        break;
      }
      ++outer;
      if (!need_inner) {
        ++inner;  // the interpolation loop's check found every z_j > 0
        continue;
      }
    }
    go_inner = false;
    for (;;) {
      ++inner;
      const int p = sh.p;
      ff amin;
      const int jmin = select_alpha<NT>(V, p, sh, amin);
      if (jmin < 0) {
        for (int s = tid; s < p; s += NT) V.xs[s] = V.zs[s];
        __syncthreads();
        break;
      }
      if (inner > max_inner) {
        if (tid == 0) sh.status = RNNLS_EMAXITER;
        __syncthreads();
        break;
      }
      for (int s = tid; s < p; s += NT) V.xs[s] = ff_add(V.xs[s], ff_mul(amin, ff_sub(V.zs[s], V.xs[s])));
      __syncthreads();
      if (tid == 0) V.xs[V.varslot[jmin]] = ff{0.0f, 0.0f};
      __syncthreads();
      for (int s = p - 1; s >= 0; --s) {
        if (ff_le0(V.xs[s])) {
          const int v = V.slotvar[s];
          __syncthreads();
          if (tid == 0) V.varslot[v] = -1;
          drop_slot<NT>(V, d, s, sh.p);
          if (tid == 0) sh.p = sh.p - 1;
          __syncthreads();
        }
      }
      if (sh.p == 0) break;
      passive_solve<NT>(V, sh, sh.p, false, 0.0f, accurate ? 2 : 0);
    }
    if (sh.status != RNNLS_OK) break;
  }

  // outputs: x, dual maximum over the active set, objective
  compute_w<NT>(V, d, sh.p);
  __syncthreads();
  for (int j = tid; j < d; j += NT) {
    const int s = V.varslot[j];
    jb.x[j] = (s >= 0) ? ff_to_double(V.xs[s]) : 0.0;
  }
  ff dmax{0.0f, 0.0f};
  int dj = -1;
  for (int j = tid; j < d; j += NT)
    if (V.varslot[j] < 0 && (dj < 0 || ff_gt(V.w[j], dmax))) {
      dmax = V.w[j];
      dj = j;
    }
  ff dbest;
  const int dbi = block_argmax_ff<NT>(dj >= 0, dmax, dj, sh, dbest);
  // objective = s's - sum over P of x_j (q_j + w_j)   (w = q - Qx)
  ff part{0.0f, 0.0f};
  for (int s = tid; s < sh.p; s += NT) {
    const int v = V.slotvar[s];
    part = ff_add(part, ff_mul(V.xs[s], ff_add(V.qv[v], V.w[v])));
  }
  const ff qxpxw = block_sum_ff<NT>(part, sh);
  if (tid == 0 && jb.info) {
    rnnls_info inf;
    inf.status = sh.status;
    inf.outer_iters = outer;
    inf.inner_iters = inner;
    inf.passive_count = sh.p;
    inf.tol = tol_d;
    inf.dual_max = (dbi >= 0) ? ff_to_double(dbest) : 0.0;
    inf.objective = jb.Qd[(int64_t)jb.qcol * jb.ldq + jb.qcol] - ff_to_double(qxpxw);
    inf.accurate_mode = accurate_mode;
    inf.reserved = 0;
    *jb.info = inf;
  }
}

template <int NT>
__global__ void __launch_bounds__(NT, NT == 32 ? 16 : 2) lh_kernel(const lh_job *__restrict__ jobs, int max_outer_mul,
                                                                  int max_inner_mul, int warp_max_d) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ lh_shared sh;
  const lh_job jb = jobs[blockIdx.x];
  if (jb.d <= 0) return;  // a problem the device-side plan refused (its info says so)
  // problems up to warp_max_d unknowns run as one-warp blocks, the others as
  // 256-thread blocks: each launch skips the other kind
  if ((NT == 32) != (jb.d <= warp_max_d)) return;
  lh_block<NT>(jb, smem_raw, sh, max_outer_mul * jb.d, max_inner_mul * jb.d);
}

template <int NT>
__global__ void __launch_bounds__(NT, 1) lh_kernel_one(const lh_job jb, int max_outer_mul, int max_inner_mul) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ lh_shared sh;
  lh_block<NT>(jb, smem_raw, sh, max_outer_mul * jb.d, max_inner_mul * jb.d);
}

// ||A x - b||^2 in FP64 (evaluation of Definition 1's objective)
__global__ void residual_kernel(const float *__restrict__ A, int64_t lda, const float *__restrict__ b, int64_t n,
                                int d, const double *__restrict__ x, double *__restrict__ partial) {
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double v = -(double)b[i];
    for (int j = 0; j < d; ++j) v += (double)A[(int64_t)j * lda + i] * x[j];
    acc += v * v;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
    partial[blockIdx.x] = t;
  }
}

__global__ void sum_partials_kernel(const double *__restrict__ partial, int nb, double *__restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < nb; ++q) t += partial[q];
    *out = t;
  }
}

struct gram_plan {
  int T, ntiles, splits;
  int64_t rows_per_split;
};

gram_plan plan_gram(int64_t m, int d, int num_sms) {
  gram_plan g;
  g.T = (d + 1 + kGT - 1) / kGT;
  g.ntiles = g.T * (g.T + 1) / 2;
  // about six blocks per SM (blocks of 256 threads and 80 registers, three
  // resident per SM): enough warps to keep the FP32 pipe busy
  int64_t want = std::max<int64_t>(1, (6 * (int64_t)num_sms + g.ntiles - 1) / g.ntiles);
  want = std::min<int64_t>(want, std::max<int64_t>(1, (m + 255) / 256));
  int64_t rps = (m + want - 1) / want;
  rps = std::max<int64_t>(kGT, (rps + kGT - 1) / kGT * kGT);
  g.rows_per_split = rps;
  g.splits = (int)((m + rps - 1) / rps);
  if (g.splits < 1) g.splits = 1;
  return g;
}

struct solve_ws {
  double *part;
  double *part_abs;
  double *Qd;
  float *Qhi, *Qlo;
  double *colabs;
  lh_job *jobs;
};

size_t solve_ws_bytes(const gram_plan &g, int d, int64_t njobs) {
  const size_t D1 = d + 1;
  return align_up((size_t)g.splits * g.ntiles * kGT * kGT * 8, 256) + align_up((size_t)g.splits * g.T * kGT * 8, 256) +
         align_up(D1 * D1 * 8, 256) +
         2 * align_up(D1 * D1 * 4, 256) + align_up((size_t)d * 8, 256) + align_up((size_t)njobs * sizeof(lh_job), 256) +
         1024;
}

// Shared memory a Lawson-Hanson block needs, and whether its passive Q rows
// fit there (else the block reads Q from global memory).
constexpr size_t kLHStaticSmem = 2048;
bool lh_q_fits(rnnls_ctx *ctx, int d) {
  return lh_make_layout(d, true).bytes + kLHStaticSmem <= (size_t)ctx->max_smem_optin;
}
// Whether the passive-block inverse fits in shared memory (Q read from global
// memory); for larger d it lives in the workspace and is read through L1/L2.
bool lh_b_fits(rnnls_ctx *ctx, int d) {
  return lh_make_layout(d, false, true).bytes + kLHStaticSmem <= (size_t)ctx->max_smem_optin;
}
size_t lh_smem_for(rnnls_ctx *ctx, int d) {
  return lh_make_layout(d, lh_q_fits(ctx, d), lh_b_fits(ctx, d)).bytes;
}
size_t lh_bg_bytes(rnnls_ctx *ctx, int d) {
  return lh_b_fits(ctx, d) ? 0 : align_up((size_t)odd_ld(d) * d * sizeof(float), 256);
}

// Problems with up to lh_warp_max_d unknowns can run as one-warp blocks (one
// warp per problem: the block's barriers and reductions stay inside the
// warp, and many problems share an SM); by default every problem runs as a
// 256-thread block.  Measured on GB300 (term-document sketches, one solve):
// d = 16: 88 vs 55 us, d = 64: 482 vs 148 us, d = 128: 1982 vs 451 us for
// one warp vs 256 threads; the per-iteration dot products and inverse
// updates, not the block barriers, set a solve's time, so eight times the
// work per thread costs more than the barriers save.
int lh_warp_max_d(const rnnls_ctx *ctx) { return ctx->tune.lh_warp_max_d; }

// d_jobs: `count` jobs with d in [min_d, max_d] (bounds; device-made job
// tables pass 1 and their bound), smem: the largest block's shared memory.
int lh_launch(rnnls_ctx *ctx, const lh_job *d_jobs, int64_t count, size_t smem, int min_d, int max_d) {
  prof_scope ps(ctx, K_LH);
  if (smem + kLHStaticSmem > (size_t)ctx->max_smem_optin) return RNNLS_EUNSUPPORTED;
  const int wmd = lh_warp_max_d(ctx);
  if (min_d <= wmd) {
    // the one-warp blocks' problems have d <= wmd: their shared memory is at most that of d = wmd
    const size_t s32 = std::min(smem, lh_make_layout(std::min(wmd, max_d), true, true).bytes);
    static smem_attr lh_attr32;
    RNNLS_CUDA_TRY(lh_attr32.ensure((const void *)lh_kernel<32>, s32));
    lh_kernel<32><<<(unsigned)count, 32, s32, ctx->stream>>>(d_jobs, 3, 30, wmd);
    if (cudaGetLastError() != cudaSuccess) return RNNLS_ECUDA;
  }
  if (max_d > wmd) {
    static smem_attr lh_attr;
    RNNLS_CUDA_TRY(lh_attr.ensure((const void *)lh_kernel<kLHThreads>, smem));
    lh_kernel<kLHThreads><<<(unsigned)count, kLHThreads, smem, ctx->stream>>>(d_jobs, 3, 30, wmd);
  }
  return cudaGetLastError() == cudaSuccess ? RNNLS_OK : RNNLS_ECUDA;
}

int lh_launch_one(rnnls_ctx *ctx, const lh_job &jb) {
  prof_scope ps(ctx, K_LH);
  const size_t smem = lh_make_layout(jb.d, jb.q_smem != 0, jb.Bg == nullptr).bytes;
  if (smem + kLHStaticSmem > (size_t)ctx->max_smem_optin) return RNNLS_EUNSUPPORTED;
  if (jb.d <= lh_warp_max_d(ctx)) {
    static smem_attr one_attr32;
    RNNLS_CUDA_TRY(one_attr32.ensure((const void *)lh_kernel_one<32>, smem));
    lh_kernel_one<32><<<1, 32, smem, ctx->stream>>>(jb, 3, 30);
  } else {
    static smem_attr one_attr;
    RNNLS_CUDA_TRY(one_attr.ensure((const void *)lh_kernel_one<kLHThreads>, smem));
    lh_kernel_one<kLHThreads><<<1, kLHThreads, smem, ctx->stream>>>(jb, 3, 30);
  }
  return cudaGetLastError() == cudaSuccess ? RNNLS_OK : RNNLS_ECUDA;
}

// One problem: the FP32 Gram on the tensor cores (column statistics, then
// the exact sliced products), the FP64 Gram as a plain two-pass reduction.
template <typename T>
int solve_one(rnnls_ctx *ctx, const T *SA, int64_t ldsa, const T *Sb, int64_t r, int64_t d, double *x,
              rnnls_info *info) {
  const bool fits = lh_q_fits(ctx, (int)d);
  const size_t D1 = d + 1;
  cudaStream_t s = ctx->stream;
  int st = RNNLS_OK;
  solve_ws w;
  float *Bg = nullptr;
  if (sizeof(T) == 4) {
    gram_tc_job gj = gram_tc_plan((const float *)SA, ldsa, (const float *)Sb, r, 1, r, (int)d, 0, ctx->num_sms,
                                  (int64_t)1 << 40, gram_min_chunks(ctx), gram_max_splits(ctx));
    const size_t bytes = align_up(D1 * D1 * 8, 256) + 2 * align_up(D1 * D1 * 4, 256) + align_up((size_t)d * 8, 256) +
                         gram_tc_ws_bytes(gj) + lh_bg_bytes(ctx, (int)d) + 1024;
    st = ensure_workspace(ctx, bytes);
    if (st) return st;
    unsigned int *counters = nullptr;
    st = ensure_counters(ctx, (size_t)gj.tiles, &counters);
    if (st) return st;
    ws_carver wc(ctx->ws);
    w.Qd = wc.take<double>(D1 * D1);
    w.Qhi = wc.take<float>(D1 * D1);
    w.Qlo = wc.take<float>(D1 * D1);
    w.colabs = wc.take<double>((size_t)d);
    gram_tc_carve(gj, wc, counters, w.Qd, w.Qhi, w.Qlo, w.colabs);
    Bg = lh_b_fits(ctx, (int)d) ? nullptr : wc.take<float>((size_t)odd_ld((int)d) * d);
    st = gram_tc_launch_one(ctx, gj);
    if (st) return st;
  } else {
    const gram_plan g = plan_gram(r, (int)d, ctx->num_sms);
    const size_t bytes = solve_ws_bytes(g, (int)d, 1) + lh_bg_bytes(ctx, (int)d);
    st = ensure_workspace(ctx, bytes);
    if (st) return st;
    ws_carver wc(ctx->ws);
    w.part = wc.take<double>((size_t)g.splits * g.ntiles * kGT * kGT);
    w.Qd = wc.take<double>(D1 * D1);
    w.Qhi = wc.take<float>(D1 * D1);
    w.Qlo = wc.take<float>(D1 * D1);
    w.colabs = wc.take<double>((size_t)d);
    Bg = lh_b_fits(ctx, (int)d) ? nullptr : wc.take<float>((size_t)odd_ld((int)d) * d);
    dim3 grid((unsigned)g.ntiles, (unsigned)g.splits);
    {
      prof_scope ps(ctx, K_GRAM);
      gram_f64_kernel<<<grid, 256, 0, s>>>((const double *)SA, ldsa, (const double *)Sb, r, (int)d, g.T,
                                           g.rows_per_split, w.part);
    }
    {
      prof_scope ps(ctx, K_GRAM_REDUCE);
      gram_reduce_kernel<<<(unsigned)std::min<int64_t>((D1 * D1 + 255) / 256, 1024), 256, 0, s>>>(
          w.part, g.splits, (int)d, g.T, w.Qd, w.Qhi, w.Qlo);
    }
    {
      prof_scope ps(ctx, K_COLABS);
      colabs_kernel<T><<<(unsigned)((d * 32 + 255) / 256), 256, 0, s>>>(SA, ldsa, r, (int)d, w.colabs);
    }
  }
  lh_job jb;
  jb.Qd = w.Qd;
  jb.Qhi = w.Qhi;
  jb.Qlo = w.Qlo;
  jb.ldq = (int)d + 1;
  jb.qcol = (int)d;
  jb.colabs = w.colabs;
  jb.r = r;
  jb.d = (int)d;
  jb.x = x;
  jb.info = info;
  jb.q_smem = fits ? 1 : 0;
  jb.Bg = Bg;
  if (cudaGetLastError() != cudaSuccess) return RNNLS_ECUDA;
  return lh_launch_one(ctx, jb);
}

}  // namespace

int solve_f32(rnnls_ctx *ctx, const float *SA, int64_t ldsa, const float *Sb, int64_t r, int64_t d, double *x,
              rnnls_info *info) {
  return solve_one<float>(ctx, SA, ldsa, Sb, r, d, x, info);
}

int solve_f64(rnnls_ctx *ctx, const double *SA, int64_t ldsa, const double *Sb, int64_t r, int64_t d, double *x,
              rnnls_info *info) {
  return solve_one<double>(ctx, SA, ldsa, Sb, r, d, x, info);
}

// Default maximum of 32-row chunks per Gram CTA in a batched launch (4096
// rows), so that the CTAs of a batch of uneven problems carry comparable work.
constexpr int64_t kBatchChunksPerCta = 128;

int solve_batched(rnnls_ctx *ctx, const rnnls_problem *probs, int64_t count) {
  // one launch for every problem's column statistics, one for every Gram,
  // then one Lawson-Hanson launch over all
  std::vector<gram_tc_job> gjs((size_t)count);
  const size_t tab_jobs = align_up((size_t)count * sizeof(gram_tc_job), 256);
  const size_t tab_first = align_up((size_t)(count + 1) * sizeof(int64_t), 256);
  const size_t tbytes = tab_jobs + 2 * tab_first + align_up((size_t)count * sizeof(lh_job), 256);
  size_t bytes = tbytes + 256;
  size_t smem = 0;
  int64_t tiles = 0;
  int min_d = INT_MAX, max_d = 0;
  for (int64_t i = 0; i < count; ++i) {
    const rnnls_problem &pb = probs[i];
    const int di = (int)pb.d;
    min_d = std::min(min_d, di);
    max_d = std::max(max_d, di);
    gjs[(size_t)i] = gram_tc_plan(pb.SA, pb.ldsa, pb.Sb, pb.r, 1, pb.r, di, 0, 1,
                                  tune_or(ctx->tune.batch_gram_chunks, kBatchChunksPerCta), gram_min_chunks(ctx),
                                  gram_max_splits(ctx));
    const size_t D1 = di + 1;
    bytes += align_up(D1 * D1 * 8, 256) + 2 * align_up(D1 * D1 * 4, 256) + align_up((size_t)di * 8, 256) +
             gram_tc_ws_bytes(gjs[(size_t)i]) + lh_bg_bytes(ctx, di) + 1024;
    smem = std::max(smem, lh_smem_for(ctx, di));
    tiles += gjs[(size_t)i].tiles;
  }
  int st = ensure_workspace(ctx, bytes);
  if (st) return st;
  unsigned int *counters = nullptr;
  st = ensure_counters(ctx, (size_t)tiles, &counters);
  if (st) return st;
  st = ensure_pinned(ctx, tbytes);
  if (st) return st;
  ws_carver wc(ctx->ws);
  char *d_tables = wc.take<char>(tbytes);
  char *h_tables = (char *)ctx->pinned;
  gram_tc_job *gj = (gram_tc_job *)h_tables;
  int64_t *first_col = (int64_t *)(h_tables + tab_jobs);
  int64_t *first_cta = (int64_t *)(h_tables + tab_jobs + tab_first);
  lh_job *jobs = (lh_job *)(h_tables + tab_jobs + 2 * tab_first);
  // Lawson-Hanson blocks start in order of decreasing d (longest first: the
  // blocks of the last wave are the short ones, so the launch ends sooner)
  std::vector<int64_t> lh_pos((size_t)count);
  {
    std::vector<int64_t> order((size_t)count);
    for (int64_t i = 0; i < count; ++i) order[(size_t)i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return probs[a].d > probs[b].d; });
    for (int64_t k = 0; k < count; ++k) lh_pos[(size_t)order[(size_t)k]] = k;
  }
  int64_t ctas = 0, cols = 0;
  for (int64_t i = 0; i < count; ++i) {
    const rnnls_problem &pb = probs[i];
    const size_t D1 = pb.d + 1;
    gram_tc_job q = gjs[(size_t)i];
    double *Qd = wc.take<double>(D1 * D1);
    float *Qhi = wc.take<float>(D1 * D1);
    float *Qlo = wc.take<float>(D1 * D1);
    double *colabs = wc.take<double>((size_t)pb.d);
    gram_tc_carve(q, wc, counters, Qd, Qhi, Qlo, colabs);
    counters += q.tiles;
    gj[i] = q;
    first_col[i] = cols;
    cols += q.c;
    first_cta[i] = ctas;
    ctas += (int64_t)q.tiles * q.splits;
    lh_job &jb = jobs[lh_pos[(size_t)i]];
    jb.Qd = Qd;
    jb.Qhi = Qhi;
    jb.Qlo = Qlo;
    jb.ldq = (int)D1;
    jb.qcol = (int)pb.d;
    jb.colabs = colabs;
    jb.r = pb.r;
    jb.d = (int)pb.d;
    jb.x = pb.x;
    jb.info = pb.info;
    jb.q_smem = lh_q_fits(ctx, (int)pb.d) ? 1 : 0;
    jb.Bg = lh_b_fits(ctx, (int)pb.d) ? nullptr : wc.take<float>((size_t)odd_ld((int)pb.d) * pb.d);
  }
  first_col[count] = cols;
  first_cta[count] = ctas;
  {
    // the Gram CTAs of the problems with most rows (the longest K-splits)
    // start first; a job's CTAs and columns stay contiguous
    std::vector<int64_t> order((size_t)count);
    for (int64_t i = 0; i < count; ++i) order[(size_t)i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return probs[a].r > probs[b].r; });
    std::vector<gram_tc_job> g2((size_t)count);
    for (int64_t k = 0; k < count; ++k) g2[(size_t)k] = gj[order[(size_t)k]];
    int64_t c2 = 0, t2 = 0;
    for (int64_t k = 0; k < count; ++k) {
      gj[k] = g2[(size_t)k];
      first_col[k] = c2;
      first_cta[k] = t2;
      c2 += gj[k].c;
      t2 += (int64_t)gj[k].tiles * gj[k].splits;
    }
  }
  cudaStream_t s = ctx->stream;
  // tables staged through the context's pinned buffer (ensure_pinned waited
  // for the previous call's copy out of it)
  RNNLS_CUDA_TRY(cudaMemcpyAsync(d_tables, h_tables, tbytes, cudaMemcpyHostToDevice, s));
  RNNLS_CUDA_TRY(cudaEventRecord(ctx->pinned_ready, s));
  const gram_tc_job *d_gj = (const gram_tc_job *)d_tables;
  const int64_t *d_first_col = (const int64_t *)(d_tables + tab_jobs);
  const int64_t *d_first_cta = (const int64_t *)(d_tables + tab_jobs + tab_first);
  const lh_job *d_jobs = (const lh_job *)(d_tables + tab_jobs + 2 * tab_first);
  st = gram_tc_launch_batched(ctx, d_gj, d_first_col, d_first_cta, (int)count, cols, ctas);
  if (st) return st;
  return lh_launch(ctx, d_jobs, count, smem, min_d, max_d);
}

// ---------------------------------------------------------------------------
// Batched solve from a device-resident descriptor array: the plan (tiles,
// K-splits, CTA and column offsets, workspace slots) is made on the device,
// within host-given bounds max_r, max_d; every problem owns a workspace slot
// of the bound's size.
// ---------------------------------------------------------------------------
namespace {

struct dev_plan_args {
  const rnnls_problem *probs;
  int64_t count, max_r;
  int max_d;
  int qfit_max, bfit_max;      // largest d whose Q / passive inverse fits in shared memory
  int min_chunks, max_splits;  // the context's Gram choices
  int64_t batch_chunks;
  char *slots;                 // count slots of slot_bytes
  size_t slot_bytes, off_qhi, off_qlo, off_colabs, off_cs, off_cu, off_part, off_bg;
  unsigned int *counters;      // count x tiles_max
  int tiles_max;
  gram_tc_job *gjobs;
  lh_job *ljobs;
  int64_t *first_col, *first_cta;  // count + 1 each
  int64_t *tmp;                    // 2 count scratch: columns and CTAs per problem
};

// One block: validate and plan every problem, then prefix sums in order.
__global__ void __launch_bounds__(256) plan_batched_device_kernel(const dev_plan_args a) {
  for (int64_t p = threadIdx.x; p < a.count; p += 256) {
    const rnnls_problem pb = a.probs[p];
    const bool ok = pb.SA && pb.Sb && pb.x && pb.r >= 1 && pb.r <= a.max_r && pb.d >= 1 && pb.d <= a.max_d &&
                    pb.ldsa >= pb.r;
    char *slot = a.slots + (size_t)p * a.slot_bytes;
    const int d = ok ? (int)pb.d : 0;
    const int c = d + 1;
    gram_tc_job j{};
    lh_job l{};
    if (ok) {
      j.S = pb.SA;
      j.s = pb.Sb;
      j.lds = pb.ldsa;
      j.ldt = pb.r;
      j.nb = 1;
      j.m = pb.r;
      j.d = d;
      j.c = c;
      j.multi = 0;
      j.tiles = gram_tc_tile_count(c, d, 0);
      gram_tc_splits(pb.r, j.tiles, 1, a.batch_chunks, a.min_chunks, a.max_splits, j.splits, j.chunks_per_split);
      j.vec4 = ((((uintptr_t)pb.SA) & 15u) == 0 && (pb.ldsa % 4) == 0 && (((uintptr_t)pb.Sb) & 15u) == 0) ? 1 : 0;
      j.Qd = (double *)slot;
      j.Qhi = (float *)(slot + a.off_qhi);
      j.Qlo = (float *)(slot + a.off_qlo);
      j.colabs = (double *)(slot + a.off_colabs);
      j.colscale = (float *)(slot + a.off_cs);
      j.colunscale = (float *)(slot + a.off_cu);
      j.part = j.splits > 1 ? (double *)(slot + a.off_part) : nullptr;
      j.counters = a.counters + (size_t)p * a.tiles_max;
      l.Qd = j.Qd;
      l.Qhi = j.Qhi;
      l.Qlo = j.Qlo;
      l.ldq = c;
      l.qcol = d;
      l.colabs = j.colabs;
      l.r = pb.r;
      l.d = d;
      l.x = pb.x;
      l.info = pb.info;
      l.q_smem = d <= a.qfit_max ? 1 : 0;
      l.Bg = d > a.bfit_max ? (float *)(slot + a.off_bg) : nullptr;
    } else if (pb.info) {
      rnnls_info inf{};
      inf.status = RNNLS_EINVAL;
      *pb.info = inf;
    }
    a.gjobs[p] = j;
    a.ljobs[p] = l;
    a.tmp[p] = ok ? c : 0;
    a.tmp[a.count + p] = ok ? (int64_t)j.tiles * j.splits : 0;
  }
  __syncthreads();
  // exclusive prefix sums of columns and CTAs, in problem order
  __shared__ int64_t carry[2];
  __shared__ int64_t warp_tot[2][8];
  if (threadIdx.x < 2) carry[threadIdx.x] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t base = 0; base < a.count; base += 256) {
    const int64_t p = base + threadIdx.x;
    int64_t v[2], inc[2];
    for (int k = 0; k < 2; ++k) {
      v[k] = p < a.count ? a.tmp[k * a.count + p] : 0;
      inc[k] = v[k];
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t u = __shfl_up_sync(0xffffffffu, inc[k], o);
        if (lane >= o) inc[k] += u;
      }
      if (lane == 31) warp_tot[k][warp] = inc[k];
    }
    __syncthreads();
    for (int k = 0; k < 2; ++k) {
      int64_t before = carry[k];
      for (int w = 0; w < warp; ++w) before += warp_tot[k][w];
      if (p < a.count) (k == 0 ? a.first_col : a.first_cta)[p] = before + inc[k] - v[k];
    }
    __syncthreads();
    if (threadIdx.x < 2) {
      int64_t t = 0;
      for (int w = 0; w < 8; ++w) t += warp_tot[threadIdx.x][w];
      carry[threadIdx.x] += t;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    a.first_col[a.count] = carry[0];
    a.first_cta[a.count] = carry[1];
  }
}

}  // namespace

int solve_batched_device(rnnls_ctx *ctx, const rnnls_problem *d_probs, int64_t count, int64_t max_r, int64_t max_d) {
  if (count == 0) return RNNLS_OK;
  const int md = (int)max_d, D1 = md + 1;
  const int min_chunks = gram_min_chunks(ctx), max_splits = gram_max_splits(ctx);
  const int64_t batch_chunks = tune_or(ctx->tune.batch_gram_chunks, kBatchChunksPerCta);
  // bounds over every problem the plan may see (tiles grow with d, splits with r)
  const int tiles_max = gram_tc_tile_count(D1, md, 0);
  int splits_max = 1;
  int64_t cps_unused = 0;
  gram_tc_splits(max_r, tiles_max, 1, batch_chunks, min_chunks, max_splits, splits_max, cps_unused);
  int qfit_max = 0, bfit_max = 0;
  size_t smem = 0;
  for (int dd = 1; dd <= md; ++dd) {
    if (lh_q_fits(ctx, dd)) qfit_max = dd;
    if (lh_b_fits(ctx, dd)) bfit_max = dd;
    smem = std::max(smem, lh_smem_for(ctx, dd));
  }
  dev_plan_args a{};
  size_t o = 0;
  auto take = [&](size_t b) {
    const size_t at = o;
    o = align_up(o + b, 256);
    return at;
  };
  take((size_t)D1 * D1 * 8);  // Qd at 0
  a.off_qhi = take((size_t)D1 * D1 * 4);
  a.off_qlo = take((size_t)D1 * D1 * 4);
  a.off_colabs = take((size_t)md * 8);
  a.off_cs = take((size_t)2 * D1 * 4);
  a.off_cu = take((size_t)D1 * 4);
  a.off_part = take(splits_max > 1 ? (size_t)splits_max * tiles_max * kGramTileM * kGramTileN * 8 : 0);
  a.off_bg = take(md > bfit_max ? (size_t)odd_ld(md) * md * 4 : 0);
  a.slot_bytes = align_up(o, 256);
  const size_t tables = align_up((size_t)count * sizeof(gram_tc_job), 256) +
                        align_up((size_t)count * sizeof(lh_job), 256) +
                        2 * align_up((size_t)(count + 1) * 8, 256) + align_up((size_t)2 * count * 8, 256);
  int st = ensure_workspace(ctx, tables + (size_t)count * a.slot_bytes + 1024);
  if (st) return st;
  unsigned int *counters = nullptr;
  st = ensure_counters(ctx, (size_t)count * tiles_max, &counters);
  if (st) return st;
  ws_carver wc(ctx->ws);
  a.probs = d_probs;
  a.count = count;
  a.max_r = max_r;
  a.max_d = md;
  a.qfit_max = qfit_max;
  a.bfit_max = bfit_max;
  a.min_chunks = min_chunks;
  a.max_splits = max_splits;
  a.batch_chunks = batch_chunks;
  a.gjobs = wc.take<gram_tc_job>((size_t)count);
  a.ljobs = wc.take<lh_job>((size_t)count);
  a.first_col = wc.take<int64_t>((size_t)count + 1);
  a.first_cta = wc.take<int64_t>((size_t)count + 1);
  a.tmp = wc.take<int64_t>((size_t)2 * count);
  a.slots = wc.take<char>((size_t)count * a.slot_bytes);
  a.counters = counters;
  a.tiles_max = tiles_max;
  cudaStream_t s = ctx->stream;
  plan_batched_device_kernel<<<1, 256, 0, s>>>(a);
  if (cudaGetLastError() != cudaSuccess) return RNNLS_ECUDA;
  st = gram_tc_launch_batched(ctx, a.gjobs, a.first_col, a.first_cta, (int)count, count * D1,
                              count * (int64_t)tiles_max * splits_max);
  if (st) return st;
  return lh_launch(ctx, a.ljobs, count, smem, 1, md);
}

int solve_multi(rnnls_ctx *ctx, const float *SA, int64_t ldsa, const float *SB, int64_t ldsb, int64_t r, int64_t d,
                int64_t nrhs, double *X, int64_t ldx, rnnls_info *infos) {
  // one Gram of [SA | SB] (the target-by-target block only on its diagonal),
  // then one Lawson-Hanson block per target, all reading the same Q
  const int64_t D1 = d + nrhs;
  gram_tc_job gj = gram_tc_plan(SA, ldsa, SB, ldsb, (int)nrhs, r, (int)d, 1, ctx->num_sms, (int64_t)1 << 40,
                                gram_min_chunks(ctx), gram_max_splits(ctx));
  const bool bfit = lh_b_fits(ctx, (int)d);
  const size_t bytes = align_up((size_t)(D1 * D1) * 8, 256) + 2 * align_up((size_t)(D1 * D1) * 4, 256) +
                       align_up((size_t)D1 * 8, 256) + gram_tc_ws_bytes(gj) +
                       align_up((size_t)nrhs * sizeof(lh_job), 256) + (size_t)nrhs * lh_bg_bytes(ctx, (int)d) + 1024;
  int st = ensure_workspace(ctx, bytes);
  if (st) return st;
  unsigned int *counters = nullptr;
  st = ensure_counters(ctx, (size_t)gj.tiles, &counters);
  if (st) return st;
  ws_carver wc(ctx->ws);
  solve_ws w;
  w.Qd = wc.take<double>((size_t)(D1 * D1));
  w.Qhi = wc.take<float>((size_t)(D1 * D1));
  w.Qlo = wc.take<float>((size_t)(D1 * D1));
  w.colabs = wc.take<double>((size_t)D1);
  gram_tc_carve(gj, wc, counters, w.Qd, w.Qhi, w.Qlo, w.colabs);
  lh_job *d_jobs = wc.take<lh_job>((size_t)nrhs);
  cudaStream_t s = ctx->stream;
  st = gram_tc_launch_one(ctx, gj);
  if (st) return st;
  std::vector<lh_job> jobs((size_t)nrhs);
  for (int64_t t = 0; t < nrhs; ++t) {
    lh_job &jb = jobs[(size_t)t];
    jb.Qd = w.Qd;
    jb.Qhi = w.Qhi;
    jb.Qlo = w.Qlo;
    jb.ldq = (int)D1;
    jb.qcol = (int)(d + t);
    jb.colabs = w.colabs;
    jb.r = r;
    jb.d = (int)d;
    jb.x = X + t * ldx;
    jb.info = infos ? infos + t : nullptr;
    jb.q_smem = 0;  // every target reads the shared Q from global memory (L1/L2), so two blocks fit per SM
    jb.Bg = bfit ? nullptr : wc.take<float>((size_t)odd_ld((int)d) * d);
  }
  const size_t jbytes = (size_t)nrhs * sizeof(lh_job);
  st = ensure_pinned(ctx, jbytes);
  if (st) return st;
  memcpy(ctx->pinned, jobs.data(), jbytes);
  RNNLS_CUDA_TRY(cudaMemcpyAsync(d_jobs, ctx->pinned, jbytes, cudaMemcpyHostToDevice, s));
  RNNLS_CUDA_TRY(cudaEventRecord(ctx->pinned_ready, s));
  return lh_launch(ctx, d_jobs, nrhs, lh_make_layout((int)d, false, bfit).bytes, (int)d, (int)d);
}

int residual_f32(rnnls_ctx *ctx, const float *A, int64_t lda, const float *b, int64_t n, int64_t d,
                 const double *x, double *out) {
  const int nb = std::min<int64_t>(std::max<int64_t>((n + 255) / 256, 1), 4 * (int64_t)ctx->num_sms);
  int st = ensure_workspace(ctx, (size_t)nb * sizeof(double) + 256);
  if (st) return st;
  double *partial = (double *)ctx->ws;
  prof_scope ps(ctx, K_RESIDUAL);
  residual_kernel<<<nb, 256, 0, ctx->stream>>>(A, lda, b, n, (int)d, x, partial);
  sum_partials_kernel<<<1, 32, 0, ctx->stream>>>(partial, nb, out);
  return cudaGetLastError() == cudaSuccess ? RNNLS_OK : RNNLS_ECUDA;
}

}  // namespace rnnls

