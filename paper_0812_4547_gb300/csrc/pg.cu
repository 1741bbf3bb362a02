// pg.cu -- an iterative solver for the small problem of Alg. 1 step 5 on
// the quadratic-programming form of Sec. 3.4 (min x'Qx - 2q'x over x >= 0,
// Q = SA'SA, q = SA'Sb): accelerated projected gradient, the alternative to
// the active-set solve for large d (Sec. 2.2 names iterative methods as the
// second family of NNLS solvers; Sec. 3.4 notes that on the sketch each
// iteration costs O(d^2) on Q~ instead of O(n d) on A).
//
// Method: FISTA (Beck & Teboulle, SIAM J. Imaging Sci. 2, 2009) with the
// gradient-based adaptive restart of O'Donoghue & Candes (Found. Comput.
// Math. 15, 2015), on the equilibrated problem y = x / D, D = diag(Q)^-1/2,
// Q' = D Q D (unit diagonal), q' = D q:
//   g = Q' z - q';   y+ = max(0, z - g / L);   G = L (z - y+)   (gradient map)
//   restart (t = 1, z = y+) when (z - y+)'(y+ - y) > 0, otherwise
//   t+ = (1 + sqrt(1 + 4 t^2)) / 2,   z = y+ + ((t - 1) / t+) (y+ - y).
// L is a bound on the largest eigenvalue of Q': the power-iteration value
// (60 steps from the all-ones vector) with a 25 % margin, never above the
// Gershgorin bound.  The solve stops when
// max_j |G_j| <= tol max_j |q'_j| (the projected-gradient KKT residual of the
// equilibrated problem) or after max_iter iterations (RNNLS_EMAXITER).
//
// GPU shape: one persistent cooperative launch.  Block b owns a contiguous
// range of rows; per iteration every warp forms its rows' gradients as
// float-float dot products of Q (the float pairs the Gram writes) with
// u = D z (float pairs, republished every iteration), the block updates its
// rows of y and z in FP64, and all blocks meet twice at a grid barrier (to
// combine the restart test and the residual, and to publish z).  Block
// partials are combined in block order, so the result is deterministic.  The
// barrier's wait is bounded: a barrier that gives up ends the solve with
// RNNLS_ETIMEOUT instead of hanging.
#include <math.h>

#include <algorithm>

#include "kernels.h"

namespace rnnls {
namespace {

constexpr int kPgThreads = 256;
constexpr int kPgWarps = kPgThreads / 32;
constexpr uint32_t kBarrierPolls = 1u << 24;  // about a second with the back-off below
constexpr int kPowerIters = 60;

struct pg_job {
  const double *Qd;
  const float *Qhi, *Qlo;
  int ldq, d;  // q in column d, ||Sb||^2 at (d, d)
  double *x;
  rnnls_info *info;
  double *Ds, *qp, *y, *z, *part;  // part: [blocks][4]
  float *uh, *ul;
  unsigned int *bar;  // [0] arrivals, [1] generation (zeroed before the launch)
  double tol;
  int max_iter;
};

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int *p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier over co-resident blocks (cooperative launch).  Returns
// false in every thread if the wait of this block gave up.
__device__ bool grid_barrier(const pg_job &jb, unsigned int &gen, int *ok_s) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    const unsigned int g = gen;
    if (atomicAdd(&jb.bar[0], 1u) == gridDim.x - 1) {
      atomicExch(&jb.bar[0], 0u);
      __threadfence();
      atomicExch(&jb.bar[1], g + 1);
    } else {
      uint32_t polls = 0;
      while (ld_acquire(&jb.bar[1]) == g) {
        if (++polls > kBarrierPolls) {
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    gen = g + 1;
    *ok_s = ok;
  }
  __syncthreads();
  return *ok_s != 0;
}

// acc_j = sum_k Q_jk u_k for the rows of this block (float-float products,
// FP64 warp sums), written to out[j - r0].
__device__ void matvec_rows(const pg_job &jb, int r0, int r1, double *out) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int j = r0 + warp; j < r1; j += kPgWarps) {
    const float *qh = jb.Qhi + (int64_t)j * jb.ldq;
    const float *ql = jb.Qlo + (int64_t)j * jb.ldq;
    float s = 0.0f, c = 0.0f;
    for (int k = lane; k < jb.d; k += 32) {
      const float ah = qh[k], al = ql[k];
      const float bh = __ldcg(jb.uh + k), bl = __ldcg(jb.ul + k);
      const ff p = two_prod(ah, bh);
      const ff t = two_sum(s, p.hi);
      s = t.hi;
      float e = __fadd_rn(t.lo, p.lo);
      e = __fmaf_rn(ah, bl, e);
      e = __fmaf_rn(al, bh, e);
      c = __fadd_rn(c, e);
    }
    double v = (double)s + (double)c;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) out[j - r0] = v;
  }
}

// Block sums of (a, b) and block maximum of m (thread 0 holds the results).
__device__ void block_reduce(double &a, double &b, double &m, double (*sh)[3]) {
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  }
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    sh[warp][0] = a;
    sh[warp][1] = b;
    sh[warp][2] = m;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    a = b = 0.0;
    m = -INFINITY;
    for (int w = 0; w < kPgWarps; ++w) {
      a += sh[w][0];
      b += sh[w][1];
      m = fmax(m, sh[w][2]);
    }
  }
  __syncthreads();
}

// Every block combines the blocks' partials (columns 0, 1 summed, 2 maxed):
// lane l of warp 0 takes blocks l, l + 32, ... in order, then a fixed
// shuffle tree, so every block gets the same bits; results in out[3].
__device__ void combine_partials(const pg_job &jb, double *out) {
  if (threadIdx.x < 32) {
    double a = 0.0, b = 0.0, m = -INFINITY;
    for (unsigned int q = threadIdx.x; q < gridDim.x; q += 32) {
      a += __ldcg(jb.part + 4 * q + 0);
      b += __ldcg(jb.part + 4 * q + 1);
      m = fmax(m, __ldcg(jb.part + 4 * q + 2));
    }
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
      m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    }
    if (threadIdx.x == 0) {
      out[0] = a;
      out[1] = b;
      out[2] = m;
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kPgThreads) pg_kernel(const pg_job jb) {
  extern __shared__ __align__(16) double pg_smem[];
  __shared__ double red[kPgWarps][3];
  __shared__ double comb[3];
  __shared__ int ok_s;
  const int d = jb.d;
  const int per = (d + (int)gridDim.x - 1) / (int)gridDim.x;
  const int r0 = min(d, (int)blockIdx.x * per), r1 = min(d, r0 + per);
  double *g = pg_smem;         // [per] gradients of this block's rows
  double *yn = pg_smem + per;  // [per] new iterate of this block's rows
  unsigned int gen = 0;
  bool alive = true;
  auto publish_u = [&](const double *v) {  // u = D v as float pairs, this block's rows
    for (int j = r0 + threadIdx.x; j < r1; j += kPgThreads) {
      const ff u = ff_from_double(jb.Ds[j] * v[j]);
      __stcg(jb.uh + j, u.hi);
      __stcg(jb.ul + j, u.lo);
    }
  };

  // ---- set-up: D, q', the start point, max |q'|, the Gershgorin bound ----
  double a = 0.0, b = 0.0, m = 0.0;
  int bad = 0;
  for (int j = r0 + threadIdx.x; j < r1; j += kPgThreads) {
    const double qjj = jb.Qd[(int64_t)j * jb.ldq + j], qj = jb.Qd[(int64_t)j * jb.ldq + d];
    bad |= !(isfinite(qjj) && isfinite(qj));
    const double Dj = (qjj > 0.0 && isfinite(qjj)) ? 1.0 / sqrt(qjj) : 0.0;
    jb.Ds[j] = Dj;
    jb.qp[j] = Dj * qj;
    jb.y[j] = 0.0;
    jb.z[j] = 0.0;
    m = fmax(m, fabs(Dj * qj));
  }
  b = bad ? 1.0 : 0.0;  // a NaN or an infinity in Q's diagonal or in q
  block_reduce(a, b, m, red);
  if (threadIdx.x == 0) {
    jb.part[4 * blockIdx.x + 0] = 0.0;
    jb.part[4 * blockIdx.x + 1] = b;
    jb.part[4 * blockIdx.x + 2] = m;
  }
  alive = grid_barrier(jb, gen, &ok_s);
  combine_partials(jb, comb);
  const double qmax = comb[2];
  int status = RNNLS_OK;
  if (!alive) status = RNNLS_ETIMEOUT;
  else if (comb[1] > 0.0 || !isfinite(qmax)) status = RNNLS_ENONFINITE;

  // Gershgorin: max_j sum_k |Q'_jk| (rows of this block), then the power iteration
  double gersh = 0.0;
  if (status == RNNLS_OK) {
    for (int j = r0 + (threadIdx.x >> 5); j < r1; j += kPgWarps) {
      double s = 0.0;
      for (int k = threadIdx.x & 31; k < d; k += 32) s += fabs(jb.Qd[(int64_t)j * jb.ldq + k]) * jb.Ds[k];
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if ((threadIdx.x & 31) == 0) g[j - r0] = s * jb.Ds[j];
    }
    __syncthreads();
    double gm = 0.0;
    for (int j = r0 + threadIdx.x; j < r1; j += kPgThreads) gm = fmax(gm, g[j - r0]);
    a = b = 0.0;
    block_reduce(a, b, gm, red);
    // power iteration start: v = 1 / sqrt(d) (kept in z)
    for (int j = r0 + threadIdx.x; j < r1; j += kPgThreads) jb.z[j] = rsqrt((double)d);
    publish_u(jb.z);
    if (threadIdx.x == 0) {
      jb.part[4 * blockIdx.x + 0] = 0.0;
      jb.part[4 * blockIdx.x + 1] = 0.0;
      jb.part[4 * blockIdx.x + 2] = gm;
    }
    alive = grid_barrier(jb, gen, &ok_s);
    combine_partials(jb, comb);
    gersh = comb[2];
  }
  double lam = 0.0;
  for (int it = 0; it < kPowerIters && alive && status == RNNLS_OK; ++it) {
    matvec_rows(jb, r0, r1, g);
    __syncthreads();
    double s2 = 0.0;
    for (int j = r0 + threadIdx.x; j < r1; j += kPgThreads) {
      g[j - r0] *= jb.Ds[j];  // (Q' v)_j
      s2 += g[j - r0] * g[j - r0];
    }
    b = 0.0;
    m = 0.0;
    block_reduce(s2, b, m, red);
    if (threadIdx.x == 0) {
      jb.part[4 * blockIdx.x + 0] = s2;
      jb.part[4 * blockIdx.x + 1] = 0.0;
      jb.part[4 * blockIdx.x + 2] = 0.0;
    }
    alive = grid_barrier(jb, gen, &ok_s);
    combine_partials(jb, comb);
    lam = sqrt(comb[0]);  // ||Q' v|| with ||v|| = 1
    const double inv = lam > 0.0 ? 1.0 / lam : 0.0;
    for (int j = r0 + threadIdx.x; j < r1; j += kPgThreads) jb.z[j] = g[j - r0] * inv;
    publish_u(jb.z);
    alive = alive && grid_barrier(jb, gen, &ok_s);
  }
  const double L = fmin(1.25 * lam, gersh);

  // ---- FISTA with gradient restart ----------------------------------------
  int iters = 0, restarts = 0;
  double t = 1.0;
  if (status == RNNLS_OK && alive) {
    for (int j = r0 + threadIdx.x; j < r1; j += kPgThreads) jb.z[j] = 0.0;
    publish_u(jb.z);
    alive = grid_barrier(jb, gen, &ok_s);
  }
  const double thr = jb.tol * qmax;
  bool done = !(status == RNNLS_OK && alive && L > 0.0 && qmax > 0.0);
  while (!done) {
    matvec_rows(jb, r0, r1, g);
    __syncthreads();
    double S = 0.0, M = 0.0;
    for (int j = r0 + threadIdx.x; j < r1; j += kPgThreads) {
      const double zj = jb.z[j], yj = jb.y[j];
      const double gj = jb.Ds[j] * g[j - r0] - jb.qp[j];
      const double ynj = fmax(0.0, zj - gj / L);
      yn[j - r0] = ynj;
      S += (zj - ynj) * (ynj - yj);
      M = fmax(M, L * fabs(zj - ynj));
    }
    b = 0.0;
    block_reduce(S, b, M, red);
    if (threadIdx.x == 0) {
      jb.part[4 * blockIdx.x + 0] = S;
      jb.part[4 * blockIdx.x + 1] = 0.0;
      jb.part[4 * blockIdx.x + 2] = M;
    }
    alive = grid_barrier(jb, gen, &ok_s);
    combine_partials(jb, comb);
    ++iters;
    if (!alive) {
      status = RNNLS_ETIMEOUT;
      break;
    }
    const bool conv = comb[2] <= thr;
    const bool restart = comb[0] > 0.0;
    double beta = 0.0;
    if (restart) {
      t = 1.0;
      ++restarts;
    } else {
      const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
      beta = (t - 1.0) / tn;
      t = tn;
    }
    for (int j = r0 + threadIdx.x; j < r1; j += kPgThreads) {
      const double ynj = yn[j - r0];
      jb.z[j] = conv ? ynj : ynj + beta * (ynj - jb.y[j]);
      jb.y[j] = ynj;
    }
    if (conv || iters >= jb.max_iter) {
      if (!conv) status = RNNLS_EMAXITER;
      done = true;
    }
    publish_u(done ? jb.y : jb.z);
    alive = grid_barrier(jb, gen, &ok_s);
    if (!alive) {
      status = RNNLS_ETIMEOUT;
      break;
    }
  }

  // ---- outputs: x = D y, the dual w = q - Q x, the objective ---------------
  // u holds D y (published above) unless the set-up failed
  const bool have = (status == RNNLS_OK || status == RNNLS_EMAXITER) && alive;
  if (have) {
    matvec_rows(jb, r0, r1, g);
    __syncthreads();
  }
  double obj = 0.0, npos = 0.0, wmax = -INFINITY;
  for (int j = r0 + threadIdx.x; j < r1; j += kPgThreads) {
    const double xj = have ? jb.Ds[j] * jb.y[j] : 0.0;
    jb.x[j] = xj;
    if (have) {
      const double qj = jb.Qd[(int64_t)j * jb.ldq + d];
      const double wj = qj - g[j - r0];
      obj += xj * (qj + wj);
      if (xj > 0.0)
        npos += 1.0;
      else
        wmax = fmax(wmax, wj);
    }
  }
  block_reduce(obj, npos, wmax, red);
  if (threadIdx.x == 0) {
    jb.part[4 * blockIdx.x + 0] = obj;
    jb.part[4 * blockIdx.x + 1] = npos;
    jb.part[4 * blockIdx.x + 2] = wmax;
  }
  const bool fin = grid_barrier(jb, gen, &ok_s);
  if (blockIdx.x == 0 && jb.info) {
    combine_partials(jb, comb);
    if (threadIdx.x == 0) {
      rnnls_info inf;
      inf.status = fin ? status : RNNLS_ETIMEOUT;
      inf.outer_iters = iters;
      inf.inner_iters = restarts;
      inf.passive_count = (int32_t)comb[1];
      inf.tol = thr;
      inf.dual_max = (comb[2] == -INFINITY) ? 0.0 : comb[2];
      inf.objective = have ? jb.Qd[(int64_t)d * jb.ldq + d] - comb[0] : 0.0;
      inf.accurate_mode = 0;
      inf.reserved = 0;
      *jb.info = inf;
    }
  }
}

}  // namespace

int solve_pg_f32(rnnls_ctx *ctx, const float *SA, int64_t ldsa, const float *Sb, int64_t r, int64_t d, double *x,
                 rnnls_info *info, double tol, int max_iter) {
  gram_tc_job gj = gram_tc_plan(SA, ldsa, Sb, r, 1, r, (int)d, 0, ctx->num_sms, (int64_t)1 << 40,
                                gram_min_chunks(ctx), gram_max_splits(ctx));
  const size_t D1 = (size_t)d + 1;
  int per_sm = 0;
  RNNLS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pg_kernel, kPgThreads,
                                                               2 * (((size_t)d + ctx->num_sms - 1) / ctx->num_sms) *
                                                                   sizeof(double)));
  // blocks: all co-resident, at least four rows each
  int nblocks = std::max(1, std::min(std::min(per_sm, 1) * ctx->num_sms, (int)((d + 3) / 4)));
  const int per = (int)((d + nblocks - 1) / nblocks);
  nblocks = (int)((d + per - 1) / per);
  const size_t smem = 2 * (size_t)per * sizeof(double);
  const size_t bytes = align_up(D1 * D1 * 8, 256) + 2 * align_up(D1 * D1 * 4, 256) + align_up((size_t)d * 8, 256) +
                       gram_tc_ws_bytes(gj) + 4 * align_up((size_t)d * 8, 256) + 2 * align_up((size_t)d * 4, 256) +
                       align_up((size_t)nblocks * 4 * 8, 256) + 256 + 1024;
  int st = ensure_workspace(ctx, bytes);
  if (st) return st;
  unsigned int *counters = nullptr;
  st = ensure_counters(ctx, (size_t)gj.tiles, &counters);
  if (st) return st;
  ws_carver wc(ctx->ws);
  double *Qd = wc.take<double>(D1 * D1);
  float *Qhi = wc.take<float>(D1 * D1);
  float *Qlo = wc.take<float>(D1 * D1);
  double *colabs = wc.take<double>((size_t)d);
  gram_tc_carve(gj, wc, counters, Qd, Qhi, Qlo, colabs);
  pg_job jb;
  jb.Qd = Qd;
  jb.Qhi = Qhi;
  jb.Qlo = Qlo;
  jb.ldq = (int)D1;
  jb.d = (int)d;
  jb.x = x;
  jb.info = info;
  jb.Ds = wc.take<double>((size_t)d);
  jb.qp = wc.take<double>((size_t)d);
  jb.y = wc.take<double>((size_t)d);
  jb.z = wc.take<double>((size_t)d);
  jb.uh = wc.take<float>((size_t)d);
  jb.ul = wc.take<float>((size_t)d);
  jb.part = wc.take<double>((size_t)nblocks * 4);
  jb.bar = wc.take<unsigned int>(2);
  jb.tol = tol;
  jb.max_iter = max_iter;
  st = gram_tc_launch_one(ctx, gj);
  if (st) return st;
  RNNLS_CUDA_TRY(cudaMemsetAsync(jb.bar, 0, 2 * sizeof(unsigned int), ctx->stream));
  prof_scope ps(ctx, K_PG);
  void *args[] = {(void *)&jb};
  RNNLS_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)pg_kernel, dim3((unsigned)nblocks), dim3(kPgThreads), args,
                                             smem, ctx->stream));
  return RNNLS_OK;
}

}  // namespace rnnls
