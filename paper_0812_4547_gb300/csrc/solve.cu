// solve.cu -- the small NNLS of Alg. 1 step 5 on the sketch, by the
// Lawson-Hanson active-set method (Sec. 2.2) on the quadratic-programming
// form Q = SA'SA, q = SA'Sb (Sec. 3.4), plus the full-data objective of
// Definition 1.
//
// Precision plan for GB300 (whose FP64 rate is a small fraction of FP32):
//   - Gram: products of FP32 entries are exact as float pairs (FMA), sums
//     are compensated (Ogita-Rump-Oishi Dot2), partial sums combined in FP64.
//   - Lawson-Hanson: an FP32 inverse of the equilibrated passive block
//     D Q_PP D (D = diag(Q)^-1/2) is kept up to date by bordering (adding a
//     column) and Schur-complement downdates (dropping one); every passive
//     solve is refined in float-float arithmetic against the accurate Q, and
//     the dual vector w = q - Qx is evaluated in float-float.  All decisions
//     (argmax of w, tolerance, sign of z, interpolation step) use these
//     refined values and the same rules as the FP64 reference algorithm.
#include <algorithm>
#include <cstring>
#include <vector>

#include "kernels.h"

namespace rnnls {

namespace {

constexpr int kGT = 32;         // Gram tile
constexpr int kLHThreads = 256; // Lawson-Hanson block

// ---------------------------------------------------------------------------
// Gram of X = [S | s] (m x (d+1)) in tiles of 32 x 32, split over rows.
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

__global__ void __launch_bounds__(256) gram_f32_kernel(const float *__restrict__ S, int64_t lds,
                                                       const float *__restrict__ s, int64_t m, int d, int T,
                                                       int64_t rows_per_split, double *__restrict__ part) {
  __shared__ float Xi[kGT][kGT + 1];
  __shared__ float Xj[kGT][kGT + 1];
  int ti, tj;
  tile_coords(blockIdx.x, T, ti, tj);
  const int ntiles = T * (T + 1) / 2;
  const int64_t k0 = (int64_t)blockIdx.y * rows_per_split;
  const int64_t k1 = min(m, k0 + rows_per_split);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  dot2 acc[2][2];
  for (int64_t kb = k0; kb < k1; kb += kGT) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = threadIdx.x + 256 * q;
      const int kk = e & 31, cc = e >> 5;
      const int64_t k = kb + kk;
      const float *ci = gram_col(S, lds, s, d, ti * kGT + cc);
      const float *cj = gram_col(S, lds, s, d, tj * kGT + cc);
      Xi[kk][cc] = (ci && k < k1) ? ci[k] : 0.0f;
      Xj[kk][cc] = (cj && k < k1) ? cj[k] : 0.0f;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < kGT; ++kk) {
      const float a0 = Xi[kk][2 * ty], a1 = Xi[kk][2 * ty + 1];
      const float b0 = Xj[kk][2 * tx], b1 = Xj[kk][2 * tx + 1];
      acc[0][0].add_prod(a0, b0);
      acc[0][1].add_prod(a0, b1);
      acc[1][0].add_prod(a1, b0);
      acc[1][1].add_prod(a1, b1);
    }
    __syncthreads();
  }
  double *out = part + ((int64_t)blockIdx.y * ntiles + blockIdx.x) * (kGT * kGT);
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const ff v = acc[a][c].value();
      out[(2 * ty + a) * kGT + 2 * tx + c] = (double)v.hi + (double)v.lo;
    }
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
  const double *Qd;  // (d+1) x (d+1): Q, q = column d, ||s||^2 = entry (d, d)
  const float *Qhi;
  const float *Qlo;
  const double *colabs;  // d column 1-norms of the sketch
  int64_t r;
  int d;
  double *x;
  rnnls_info *info;
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

__device__ __forceinline__ ff qld(const lh_job &jb, int i, int j) {
  const int64_t e = (int64_t)i * (jb.d + 1) + j;
  return ff{jb.Qhi[e], jb.Qlo[e]};
}

// block sum of floats (all threads get the result)
__device__ float block_sum_f(float v, lh_shared &sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh.fred[warp] = v;
  __syncthreads();
  float t = 0.0f;
#pragma unroll
  for (int q = 0; q < kLHThreads / 32; ++q) t += sh.fred[q];
  return t;
}

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
  for (int q = 0; q < kLHThreads / 32; ++q) t = ff_add(t, sh.vred[q]);
  return t;
}

// argmax of (valid, value) with ties to the smallest index; returns -1 if none
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
  for (int q = 0; q < kLHThreads / 32; ++q) {
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

// argmin with ties to the smallest index
__device__ int block_argmin_ff(bool valid, ff v, int idx, lh_shared &sh, ff &best) {
  return block_argmax_ff(valid, ff_neg(v), idx, sh, best);
}

struct lh_vecs {
  float *B;     // ldB x p FP32 inverse of D Q_PP D, slot indexed
  int ldB;
  float *Dsc;   // d: D_jj = Q_jj^(-1/2)
  float *qh;    // d: D q in FP32
  float *f1, *f2, *f3;  // d+1 FP32 temporaries
  ff *x, *z, *w, *res;  // d float-float vectors
  int *slotvar;  // p: variable at slot
  int *varslot;  // d: slot of variable or -1
  unsigned char *rej;
};

// y[s] = sum_s' B[s][s'] g[s'] for s < p (B symmetric: read column s)
__device__ __forceinline__ void apply_B(const lh_vecs &V, int p, const float *g, float *y) {
  for (int s = threadIdx.x; s < p; s += kLHThreads) {
    float acc = 0.0f;
    for (int q = 0; q < p; ++q) acc = fmaf(V.B[(int64_t)q * V.ldB + s], g[q], acc);
    y[s] = acc;
  }
}

// Accurate passive solve for the current slots 0..np-1 (variables slotvar),
// z = Q_PP^{-1} q_P.  B holds the inverse of D Q_PP D when `bordered` is
// false; when true, slots 0..np-2 use B and slot np-1 is the candidate added
// by the bordering formulas with vector v = f3 (B u) and Schur value sc.
__device__ void passive_solve(const lh_job &jb, const lh_vecs &V, lh_shared &sh, int np, bool bordered, float sc,
                              int iters) {
  const int d = jb.d;
  const int pb = bordered ? np - 1 : np;
  // initial FP32 solve in scaled variables: g = D q_P
  // step 0 uses g = qh; subsequent steps use g = D res
  for (int step = 0; step <= iters; ++step) {
    // g into f1
    for (int s = threadIdx.x; s < np; s += kLHThreads) {
      const int v = V.slotvar[s];
      V.f1[s] = (step == 0) ? V.qh[v] : V.res[s].hi * V.Dsc[v];
    }
    __syncthreads();
    // y = B g on the first pb slots -> f2
    apply_B(V, pb, V.f1, V.f2);
    __syncthreads();
    if (bordered) {
      // y_t = (g_t - v'g_P) / sc ; y_P = B g_P - v y_t
      float part = 0.0f;
      for (int s = threadIdx.x; s < pb; s += kLHThreads) part = fmaf(V.f3[s], V.f1[s], part);
      const float vg = block_sum_f(part, sh);
      const float yt = (V.f1[pb] - vg) / sc;
      for (int s = threadIdx.x; s < pb; s += kLHThreads) V.f2[s] = fmaf(-V.f3[s], yt, V.f2[s]);
      if (threadIdx.x == 0) V.f2[pb] = yt;
      __syncthreads();
    }
    // z (+)= D y
    for (int s = threadIdx.x; s < np; s += kLHThreads) {
      const int v = V.slotvar[s];
      const float dz = V.f2[s] * V.Dsc[v];
      V.z[s] = (step == 0) ? ff_make(dz) : ff_add(V.z[s], ff_make(dz));
    }
    __syncthreads();
    if (step == iters) break;
    // residual res = q_P - Q_PP z (float-float)
    for (int s = threadIdx.x; s < np; s += kLHThreads) {
      const int vi = V.slotvar[s];
      dotff acc;
      acc.init(qld(jb, vi, d));
      for (int q = 0; q < np; ++q) acc.sub_prod(qld(jb, V.slotvar[q], vi), V.z[q]);
      V.res[s] = acc.value();
    }
    __syncthreads();
  }
}

__device__ void compute_w(const lh_job &jb, const lh_vecs &V, int p) {
  const int d = jb.d;
  for (int j = threadIdx.x; j < d; j += kLHThreads) {
    dotff acc;
    acc.init(qld(jb, j, d));
    for (int s = 0; s < p; ++s) {
      const int v = V.slotvar[s];
      acc.sub_prod(qld(jb, v, j), V.x[v]);
    }
    V.w[j] = acc.value();
  }
}

// Remove slot s from the inverse (Schur complement) and move the last slot
// into its place.  p is the count before removal.
__device__ void downdate(const lh_vecs &V, lh_shared &sh, int s, int p) {
  const float bss = V.B[(int64_t)s * V.ldB + s];
  // save column s
  for (int q = threadIdx.x; q < p; q += kLHThreads) V.f1[q] = V.B[(int64_t)q * V.ldB + s];
  __syncthreads();
  for (int64_t e = threadIdx.x; e < (int64_t)p * p; e += kLHThreads) {
    const int a = (int)(e / p), c = (int)(e % p);
    V.B[(int64_t)a * V.ldB + c] -= V.f1[a] * V.f1[c] / bss;
  }
  __syncthreads();
  const int last = p - 1;
  if (s != last) {
    // move row/column `last` into s
    for (int q = threadIdx.x; q < p; q += kLHThreads) V.f1[q] = V.B[(int64_t)last * V.ldB + q];
    __syncthreads();
    for (int q = threadIdx.x; q < p; q += kLHThreads) {
      if (q == s) continue;  // the removed slot's own entries are dropped
      const float val = V.f1[q];
      const int qq = (q == last) ? s : q;
      V.B[(int64_t)s * V.ldB + qq] = val;
      V.B[(int64_t)qq * V.ldB + s] = val;
    }
    if (threadIdx.x == 0) {
      const int v = V.slotvar[last];
      V.slotvar[s] = v;
      V.varslot[v] = s;
    }
  }
  __syncthreads();
}

__device__ void lh_block(const lh_job &jb, unsigned char *smem_raw, lh_shared &sh, int max_outer, int max_inner) {
  const int d = jb.d;
  const int tid = threadIdx.x;
  lh_vecs V;
  V.ldB = (d % 2 == 0) ? d + 1 : d + 2;
  char *ptr = (char *)smem_raw;
  auto take = [&](size_t bytes) {
    char *q = ptr;
    ptr += (bytes + 15) & ~(size_t)15;
    return (void *)q;
  };
  V.B = (float *)take((size_t)V.ldB * d * sizeof(float));
  V.Dsc = (float *)take(d * sizeof(float));
  V.qh = (float *)take(d * sizeof(float));
  V.f1 = (float *)take((d + 1) * sizeof(float));
  V.f2 = (float *)take((d + 1) * sizeof(float));
  V.f3 = (float *)take((d + 1) * sizeof(float));
  V.x = (ff *)take(d * sizeof(ff));
  V.z = (ff *)take((d + 1) * sizeof(ff));
  V.w = (ff *)take(d * sizeof(ff));
  V.res = (ff *)take((d + 1) * sizeof(ff));
  V.slotvar = (int *)take((d + 1) * sizeof(int));
  V.varslot = (int *)take(d * sizeof(int));
  V.rej = (unsigned char *)take(d);

  // tolerance 10 eps ||S||_1 max(r, d) ||s||_2 (FP64 scalar work, once)
  __shared__ double tol_d;
  if (tid == 0) {
    double n1 = 0.0;
    for (int j = 0; j < d; ++j) n1 = fmax(n1, jb.colabs[j]);
    const double ss = jb.Qd[(int64_t)d * (d + 1) + d];
    tol_d = 10.0 * 2.220446049250313e-16 * n1 * (double)max(jb.r, (int64_t)d) * sqrt(fmax(ss, 0.0));
    sh.p = 0;
    sh.status = RNNLS_OK;
    sh.flag = 0;
  }
  __syncthreads();
  const ff tol = ff_from_double(tol_d);
  // finiteness of Q, q
  {
    int bad = 0;
    for (int64_t e = tid; e < (int64_t)(d + 1) * (d + 1); e += kLHThreads) bad |= !isfinite(jb.Qd[e]);
    if (__syncthreads_or(bad)) {
      for (int j = tid; j < d; j += kLHThreads) jb.x[j] = 0.0;
      if (tid == 0 && jb.info) {
        rnnls_info inf;
        inf.status = RNNLS_ENONFINITE;
        inf.outer_iters = inf.inner_iters = inf.passive_count = 0;
        inf.tol = tol_d;
        inf.dual_max = 0.0;
        inf.objective = 0.0;
        *jb.info = inf;
      }
      return;
    }
  }
  for (int j = tid; j < d; j += kLHThreads) {
    const double qjj = jb.Qd[(int64_t)j * (d + 1) + j];
    const float dj = (qjj > 0.0) ? (float)(1.0 / sqrt(qjj)) : 0.0f;
    V.Dsc[j] = dj;
    V.qh[j] = (float)jb.Qd[(int64_t)j * (d + 1) + d] * dj;
    V.x[j] = ff{0.0f, 0.0f};
    V.varslot[j] = -1;
  }
  __syncthreads();

  int outer = 0, inner = 0;
  const int refine = 2;
  for (;;) {
    // dual vector
    compute_w(jb, V, sh.p);
    for (int j = tid; j < d; j += kLHThreads) V.rej[j] = 0;
    __syncthreads();
    bool accepted = false;
    for (;;) {
      // candidate: argmax over j not in P, not rejected
      bool valid = false;
      ff wv{0.0f, 0.0f};
      int jj = -1;
      ff bestl{-3.0e38f, 0.0f};
      int bi = -1;
      for (int j = tid; j < d; j += kLHThreads) {
        if (V.varslot[j] < 0 && !V.rej[j]) {
          const ff wj = V.w[j];
          if (jj < 0 || ff_gt(wj, bestl)) {
            bestl = wj;
            jj = j;
          }
        }
      }
      valid = jj >= 0;
      wv = bestl;
      ff best;
      bi = block_argmax_ff(valid, wv, jj, sh, best);
      if (bi < 0 || !ff_gt(best, tol)) break;
      const int t = bi;
      const int p = sh.p;
      // bordering: u = D Q[P, t] D_t, v = B u, sc = 1 - u'v
      for (int s = tid; s < p; s += kLHThreads) {
        const int v = V.slotvar[s];
        V.f1[s] = jb.Qhi[(int64_t)v * (d + 1) + t] * V.Dsc[v] * V.Dsc[t];
      }
      __syncthreads();
      apply_B(V, p, V.f1, V.f3);
      __syncthreads();
      float part = 0.0f;
      for (int s = tid; s < p; s += kLHThreads) part = fmaf(V.f1[s], V.f3[s], part);
      const float uv = block_sum_f(part, sh);
      const float sc = 1.0f - uv;
      if (!(sc > 1e-13f) || V.Dsc[t] == 0.0f) {
        if (tid == 0) V.rej[t] = 1;
        __syncthreads();
        continue;
      }
      if (tid == 0) V.slotvar[p] = t;
      __syncthreads();
      passive_solve(jb, V, sh, p + 1, true, sc, refine);
      if (!ff_gt0(V.z[p])) {
        if (tid == 0) V.rej[t] = 1;
        __syncthreads();
        continue;
      }
      // commit the bordered inverse: B += v v'/sc, new row/col -v/sc, corner 1/sc
      for (int64_t e = tid; e < (int64_t)p * p; e += kLHThreads) {
        const int a = (int)(e / p), c = (int)(e % p);
        V.B[(int64_t)a * V.ldB + c] += V.f3[a] * V.f3[c] / sc;
      }
      for (int s = tid; s < p; s += kLHThreads) {
        V.B[(int64_t)s * V.ldB + p] = -V.f3[s] / sc;
        V.B[(int64_t)p * V.ldB + s] = -V.f3[s] / sc;
      }
      if (tid == 0) {
        V.B[(int64_t)p * V.ldB + p] = 1.0f / sc;
        V.varslot[t] = p;
        sh.p = p + 1;
      }
      __syncthreads();
      accepted = true;
      break;
    }
    if (!accepted) break;
    if (outer >= max_outer) {
      if (tid == 0) sh.status = RNNLS_EMAXITER;
      __syncthreads();
      break;
    }
    ++outer;
    // interpolation loop; z holds the passive solution for the current slots
    for (;;) {
      ++inner;
      const int p = sh.p;
      // alpha = min over slots with z <= 0 of x/(x - z), ties -> smallest variable
      bool valid = false;
      ff aval{0.0f, 0.0f};
      int jv = -1;
      for (int s = tid; s < p; s += kLHThreads) {
        const int v = V.slotvar[s];
        if (ff_le0(V.z[s])) {
          const ff xv = V.x[v];
          const ff a = ff_div(xv, ff_sub(xv, V.z[s]));
          if (jv < 0 || ff_lt(a, aval) || (!ff_gt(a, aval) && v < jv)) {
            aval = a;
            jv = v;
          }
        }
      }
      valid = jv >= 0;
      ff amin;
      const int jmin = block_argmin_ff(valid, aval, jv, sh, amin);
      if (jmin < 0) {
        for (int s = tid; s < p; s += kLHThreads) V.x[V.slotvar[s]] = V.z[s];
        __syncthreads();
        break;
      }
      if (inner > max_inner) {
        if (tid == 0) sh.status = RNNLS_EMAXITER;
        __syncthreads();
        break;
      }
      const ff alpha = ff_neg(amin);  // argmin returned the negated value
      for (int s = tid; s < p; s += kLHThreads) {
        const int v = V.slotvar[s];
        V.x[v] = ff_add(V.x[v], ff_mul(alpha, ff_sub(V.z[s], V.x[v])));
      }
      __syncthreads();
      if (tid == 0) V.x[jmin] = ff{0.0f, 0.0f};
      __syncthreads();
      // drop every passive variable with x <= 0 (highest slot first keeps
      // the slot moves simple)
      for (int s = p - 1; s >= 0; --s) {
        const int v = V.slotvar[s];
        if (ff_le0(V.x[v])) {
          __syncthreads();
          if (tid == 0) {
            V.x[v] = ff{0.0f, 0.0f};
            V.varslot[v] = -1;
          }
          downdate(V, sh, s, sh.p);
          if (tid == 0) sh.p = sh.p - 1;
          __syncthreads();
        }
      }
      if (sh.p == 0) break;
      passive_solve(jb, V, sh, sh.p, false, 0.0f, refine);
    }
    if (sh.status != RNNLS_OK) break;
  }

  // outputs
  compute_w(jb, V, sh.p);
  __syncthreads();
  for (int j = tid; j < d; j += kLHThreads) jb.x[j] = ff_to_double(V.x[j]);
  // dual max over the active set and objective x'Qx - 2q'x + s's
  ff dmax{-3.0e38f, 0.0f};
  int dj = -1;
  for (int j = tid; j < d; j += kLHThreads)
    if (V.varslot[j] < 0 && (dj < 0 || ff_gt(V.w[j], dmax))) {
      dmax = V.w[j];
      dj = j;
    }
  ff dbest;
  const int dbi = block_argmax_ff(dj >= 0, dmax, dj, sh, dbest);
  // objective = s's - q'x - x'w  (since w = q - Qx: x'Qx = q'x - x'w)
  ff part{0.0f, 0.0f};
  for (int j = tid; j < d; j += kLHThreads) {
    const ff xj = V.x[j];
    const ff qj = qld(jb, j, d);
    part = ff_add(part, ff_mul(xj, ff_add(qj, V.w[j])));
  }
  const ff qxpxw = block_sum_ff(part, sh);
  if (tid == 0 && jb.info) {
    rnnls_info inf;
    inf.status = sh.status;
    inf.outer_iters = outer;
    inf.inner_iters = inner;
    inf.passive_count = sh.p;
    inf.tol = tol_d;
    inf.dual_max = (dbi >= 0) ? ff_to_double(dbest) : 0.0;
    inf.objective = jb.Qd[(int64_t)d * (d + 1) + d] - ff_to_double(qxpxw);
    *jb.info = inf;
  }
}

size_t lh_smem_bytes(int d) {
  const int ldB = (d % 2 == 0) ? d + 1 : d + 2;
  auto r16 = [](size_t b) { return (b + 15) & ~(size_t)15; };
  size_t b = r16((size_t)ldB * d * 4) + 2 * r16(d * 4) + 3 * r16((d + 1) * 4) + r16(d * 8) + r16((d + 1) * 8) +
             r16(d * 8) + r16((d + 1) * 8) + r16((d + 1) * 4) + r16(d * 4) + r16(d);
  return b;
}

__global__ void __launch_bounds__(kLHThreads, 1) lh_kernel(const lh_job *__restrict__ jobs, int max_outer_mul,
                                                           int max_inner_mul) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ lh_shared sh;
  const lh_job jb = jobs[blockIdx.x];
  lh_block(jb, smem_raw, sh, max_outer_mul * jb.d, max_inner_mul * jb.d);
}

__global__ void __launch_bounds__(kLHThreads, 1) lh_kernel_one(const lh_job jb, int max_outer_mul,
                                                               int max_inner_mul) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ lh_shared sh;
  lh_block(jb, smem_raw, sh, max_outer_mul * jb.d, max_inner_mul * jb.d);
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
  int64_t want = std::max<int64_t>(1, (2 * (int64_t)num_sms + g.ntiles - 1) / g.ntiles);
  int64_t rps = (m + want - 1) / want;
  rps = std::max<int64_t>(kGT, (rps + kGT - 1) / kGT * kGT);
  g.rows_per_split = rps;
  g.splits = (int)((m + rps - 1) / rps);
  if (g.splits < 1) g.splits = 1;
  return g;
}

struct solve_ws {
  double *part;
  double *Qd;
  float *Qhi, *Qlo;
  double *colabs;
  lh_job *jobs;
};

size_t solve_ws_bytes(const gram_plan &g, int d, int64_t njobs) {
  const size_t D1 = d + 1;
  return align_up((size_t)g.splits * g.ntiles * kGT * kGT * 8, 256) + align_up(D1 * D1 * 8, 256) +
         2 * align_up(D1 * D1 * 4, 256) + align_up((size_t)d * 8, 256) + align_up((size_t)njobs * sizeof(lh_job), 256) +
         1024;
}

int lh_launch(rnnls_ctx *ctx, const lh_job *d_jobs, int64_t count, int dmax) {
  prof_scope ps(ctx, K_LH);
  const size_t smem = lh_smem_bytes(dmax);
  if (smem > (size_t)ctx->max_smem_optin) return RNNLS_EUNSUPPORTED;
  RNNLS_CUDA_TRY(cudaFuncSetAttribute(lh_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  lh_kernel<<<(unsigned)count, kLHThreads, smem, ctx->stream>>>(d_jobs, 3, 30);
  return cudaGetLastError() == cudaSuccess ? RNNLS_OK : RNNLS_ECUDA;
}

int lh_launch_one(rnnls_ctx *ctx, const lh_job &jb) {
  prof_scope ps(ctx, K_LH);
  const size_t smem = lh_smem_bytes(jb.d);
  if (smem > (size_t)ctx->max_smem_optin) return RNNLS_EUNSUPPORTED;
  static int attr_bytes = 0;
  if ((int)smem > attr_bytes) {
    RNNLS_CUDA_TRY(cudaFuncSetAttribute(lh_kernel_one, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr_bytes = (int)smem;
  }
  lh_kernel_one<<<1, kLHThreads, smem, ctx->stream>>>(jb, 3, 30);
  return cudaGetLastError() == cudaSuccess ? RNNLS_OK : RNNLS_ECUDA;
}

template <typename T>
int solve_one(rnnls_ctx *ctx, const T *SA, int64_t ldsa, const T *Sb, int64_t r, int64_t d, double *x,
              rnnls_info *info) {
  const gram_plan g = plan_gram(r, (int)d, ctx->num_sms);
  const size_t bytes = solve_ws_bytes(g, (int)d, 1);
  int st = ensure_workspace(ctx, bytes);
  if (st) return st;
  ws_carver wc(ctx->ws);
  solve_ws w;
  const size_t D1 = d + 1;
  w.part = wc.take<double>((size_t)g.splits * g.ntiles * kGT * kGT);
  w.Qd = wc.take<double>(D1 * D1);
  w.Qhi = wc.take<float>(D1 * D1);
  w.Qlo = wc.take<float>(D1 * D1);
  w.colabs = wc.take<double>((size_t)d);
  cudaStream_t s = ctx->stream;
  dim3 grid((unsigned)g.ntiles, (unsigned)g.splits);
  {
    prof_scope ps(ctx, K_GRAM);
    if (sizeof(T) == 4)
      gram_f32_kernel<<<grid, 256, 0, s>>>((const float *)SA, ldsa, (const float *)Sb, r, (int)d, g.T,
                                           g.rows_per_split, w.part);
    else
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
  lh_job jb;
  jb.Qd = w.Qd;
  jb.Qhi = w.Qhi;
  jb.Qlo = w.Qlo;
  jb.colabs = w.colabs;
  jb.r = r;
  jb.d = (int)d;
  jb.x = x;
  jb.info = info;
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

int solve_batched(rnnls_ctx *ctx, const rnnls_problem *probs, int64_t count) {
  // Gram per problem (tile kernels), then one Lawson-Hanson launch over all
  int dmax = 1;
  int64_t rmax = 1;
  for (int64_t i = 0; i < count; ++i) {
    dmax = std::max<int>(dmax, (int)probs[i].d);
    rmax = std::max<int64_t>(rmax, probs[i].r);
  }
  std::vector<gram_plan> plans((size_t)count);
  size_t bytes = align_up((size_t)count * sizeof(lh_job), 256) + 256;
  for (int64_t i = 0; i < count; ++i) {
    plans[(size_t)i] = plan_gram(probs[i].r, (int)probs[i].d, std::max(1, ctx->num_sms / 8));
    bytes += solve_ws_bytes(plans[(size_t)i], (int)probs[i].d, 0);
  }
  int st = ensure_workspace(ctx, bytes);
  if (st) return st;
  ws_carver wc(ctx->ws);
  lh_job *d_jobs = wc.take<lh_job>((size_t)count);
  std::vector<lh_job> jobs((size_t)count);
  cudaStream_t s = ctx->stream;
  for (int64_t i = 0; i < count; ++i) {
    const rnnls_problem &pb = probs[i];
    const gram_plan &g = plans[(size_t)i];
    const size_t D1 = pb.d + 1;
    double *part = wc.take<double>((size_t)g.splits * g.ntiles * kGT * kGT);
    double *Qd = wc.take<double>(D1 * D1);
    float *Qhi = wc.take<float>(D1 * D1);
    float *Qlo = wc.take<float>(D1 * D1);
    double *colabs = wc.take<double>((size_t)pb.d);
    dim3 grid((unsigned)g.ntiles, (unsigned)g.splits);
    gram_f32_kernel<<<grid, 256, 0, s>>>(pb.SA, pb.ldsa, pb.Sb, pb.r, (int)pb.d, g.T, g.rows_per_split, part);
    gram_reduce_kernel<<<(unsigned)std::min<int64_t>((D1 * D1 + 255) / 256, 1024), 256, 0, s>>>(part, g.splits,
                                                                                               (int)pb.d, g.T, Qd,
                                                                                               Qhi, Qlo);
    colabs_kernel<float><<<(unsigned)((pb.d * 32 + 255) / 256), 256, 0, s>>>(pb.SA, pb.ldsa, pb.r, (int)pb.d, colabs);
    lh_job &jb = jobs[(size_t)i];
    jb.Qd = Qd;
    jb.Qhi = Qhi;
    jb.Qlo = Qlo;
    jb.colabs = colabs;
    jb.r = pb.r;
    jb.d = (int)pb.d;
    jb.x = pb.x;
    jb.info = pb.info;
  }
  if (cudaGetLastError() != cudaSuccess) return RNNLS_ECUDA;
  // job table: staged through the context's pinned buffer (the previous
  // batched call's copy must have finished before it is overwritten)
  const size_t jbytes = (size_t)count * sizeof(lh_job);
  st = ensure_pinned(ctx, jbytes);
  if (st) return st;
  memcpy(ctx->pinned, jobs.data(), jbytes);
  RNNLS_CUDA_TRY(cudaMemcpyAsync(d_jobs, ctx->pinned, jbytes, cudaMemcpyHostToDevice, s));
  RNNLS_CUDA_TRY(cudaEventRecord(ctx->pinned_ready, s));
  return lh_launch(ctx, d_jobs, count, dmax);
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
