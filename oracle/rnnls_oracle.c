/*
 * rnnls_oracle.c -- plain, slow, FP64 CPU oracle for RandomizedNNLS
 * (Boutsidis & Drineas, "Random Projections for the Nonnegative
 * Least-Squares Problem").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header, table or constant
 * generator with the CUDA library: every routine here is written out from
 * its definition.
 *
 * What it computes, and where each piece comes from:
 *   - Philox4x64-10 counter-based generator: Salmon, Moraes, Dror & Shaw,
 *     "Parallel random numbers: as easy as 1, 2, 3" (SC'11), Sec. 4.  The
 *     paper under test leaves the generator for D and S unspecified
 *     (Alg. 1 steps 2 and 4); this stream layout is the project's reading.
 *   - Walsh-Hadamard matrix: Sylvester recursion H_2n = [[H,H],[H,-H]] of
 *     Sec. 2, natural order, H[i][j] = (-1)^popcount(i & j); normalised by
 *     1/sqrt(n); zero-row padding to a power of two (Sec. 2).
 *   - Sketch H~ D [A b]: Alg. 1 steps 1-5.  Bernoulli row selection with
 *     probability r/n (Alg. 1 step 2), or r uniform draws with replacement
 *     (fixed-size reading), each kept row scaled by sqrt(n/r); with the
 *     1/sqrt(n) normalisation the combined factor is 1/sqrt(r).  For r >= n
 *     in Bernoulli mode every row is kept with factor 1/sqrt(n) (Alg. 2,
 *     min{1, r p_i} with p_i = 1/n).
 *   - Small NNLS: Lawson & Hanson active-set method (the solver the paper
 *     cites in Sec. 2.2, used as Matlab's lsqnonneg), run on the quadratic
 *     programming form x'Qx - 2q'x with Q = S'S, q = S'Sb (Sec. 3.4).
 *     Each passive-set least-squares subproblem is solved from scratch by a
 *     dense Cholesky factorisation of Q_PP.
 *   - Objective ||Ax - b||^2 of Definition 1 and the residual ratio of
 *     Theorem 1.
 *
 * Parity status: every exported function is pinned by CPU tests against a
 * library routine, a closed form or brute force (see tests/test_oracle_*.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ECAPACITY 2
#define ORC_ESINGULAR 4
#define ORC_EMAXITER 5

#define ORC_MODE_IID 0
#define ORC_MODE_BERNOULLI 1

/* ------------------------------------------------------------------------ */
/* Philox4x64-10 (SC'11 paper, Sec. 4: multiplier and Weyl constants of the  */
/* 4x64 variant, 10 rounds).                                                 */
/* ------------------------------------------------------------------------ */
static void mul128(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo) {
  unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
  *hi = (uint64_t)(p >> 64);
  *lo = (uint64_t)p;
}

void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
  uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint64_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += W0;
      k1 += W1;
    }
    uint64_t hi0, lo0, hi1, lo1;
    mul128(M0, x0, &hi0, &lo0);
    mul128(M1, x2, &hi1, &lo1);
    uint64_t y0 = hi1 ^ x1 ^ k0;
    uint64_t y1 = lo1;
    uint64_t y2 = hi0 ^ x3 ^ k1;
    uint64_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* One 64-bit word of stream `stream`: call j = word_index / 4, word
 * word_index % 4, key (seed, instance), counter (j, stream, 0, 0). */
static uint64_t stream_word(uint64_t seed, uint64_t instance, uint64_t stream, uint64_t word_index) {
  uint64_t ctr[4] = {word_index >> 2, stream, 0, 0};
  uint64_t key[2] = {seed, instance};
  uint64_t out[4];
  orc_philox4x64_10(ctr, key, out);
  return out[word_index & 3];
}

/* D_ii of Alg. 1 step 4: bit (i mod 64) of word (i / 64) of stream 0;
 * a set bit means -1. */
int orc_sign(uint64_t seed, uint64_t instance, uint64_t i) {
  uint64_t w = stream_word(seed, instance, 0, i >> 6);
  return ((w >> (i & 63)) & 1ULL) ? -1 : 1;
}

void orc_signs(uint64_t seed, uint64_t instance, int64_t n, int8_t *D) {
  for (int64_t i = 0; i < n; ++i) D[i] = (int8_t)orc_sign(seed, instance, (uint64_t)i);
}

static int log2_pow2(int64_t n) {
  int L = 0;
  while (((int64_t)1 << L) < n) ++L;
  return L;
}

/* Sampled rows.  iid: draw k takes word k of stream 2, row = top L bits.
 * Bernoulli (Alg. 1 step 2): row i is kept iff word i of stream 1 is below
 * r * 2^(64-L), i.e. with probability exactly r/n; every row if r >= n.
 * Returns the number of rows written (or -1 if cap is too small). */
int64_t orc_sample(uint64_t seed, uint64_t instance, int64_t n, int64_t r, int mode, int32_t *idx,
                   int64_t cap) {
  int L = log2_pow2(n);
  if (mode == ORC_MODE_IID) {
    if (r > cap) return -1;
    for (int64_t k = 0; k < r; ++k) {
      uint64_t u = stream_word(seed, instance, 2, (uint64_t)k);
      idx[k] = (L == 0) ? 0 : (int32_t)(u >> (64 - L));
    }
    return r;
  }
  int64_t cnt = 0;
  for (int64_t i = 0; i < n; ++i) {
    int keep;
    if (r >= n) {
      keep = 1;
    } else {
      uint64_t u = stream_word(seed, instance, 1, (uint64_t)i);
      uint64_t thresh = (uint64_t)r << (64 - L); /* r < n = 2^L so no overflow */
      keep = u < thresh;
    }
    if (keep) {
      if (cnt >= cap) return -1;
      idx[cnt++] = (int32_t)i;
    }
  }
  return cnt;
}

/* Combined scale of the kept rows: (1/sqrt(n)) * sqrt(n/r) = 1/sqrt(r),
 * or 1/sqrt(n) when Bernoulli mode keeps every row (r >= n). */
double orc_scale(int64_t n, int64_t r, int mode) {
  if (mode == ORC_MODE_BERNOULLI && r >= n) return 1.0 / sqrt((double)n);
  return 1.0 / sqrt((double)r);
}

/* ------------------------------------------------------------------------ */
/* Walsh-Hadamard transform (Sec. 2).                                         */
/* ------------------------------------------------------------------------ */
static int popcount64(uint64_t v) {
  int c = 0;
  while (v) {
    v &= v - 1;
    ++c;
  }
  return c;
}

/* Dense unnormalised Sylvester matrix, row-major n x n. */
void orc_hadamard_dense(int64_t n, double *H) {
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j) H[i * n + j] = (popcount64((uint64_t)(i & j)) & 1) ? -1.0 : 1.0;
}

/* In-place unnormalised transform y <- H_n y, iterative butterflies
 * (a, b) -> (a + b, a - b) for h = 1, 2, 4, ..., n/2. */
void orc_fwht(double *y, int64_t n) {
  for (int64_t h = 1; h < n; h <<= 1) {
    for (int64_t i = 0; i < n; i += 2 * h) {
      for (int64_t j = i; j < i + h; ++j) {
        double a = y[j], b = y[j + h];
        y[j] = a + b;
        y[j + h] = a - b;
      }
    }
  }
}

/* y <- H_n y by explicit matrix-vector product with the dense matrix. */
static void fwht_dense(double *y, int64_t n, double *tmp) {
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t j = 0; j < n; ++j) s += ((popcount64((uint64_t)(i & j)) & 1) ? -y[j] : y[j]);
    tmp[i] = s;
  }
  memcpy(y, tmp, (size_t)n * sizeof(double));
}

/* ------------------------------------------------------------------------ */
/* The sketch of Alg. 1: SX = scale * (rows idx of H_n) * D * [A b].          */
/* A: col-major n_raw x d (leading dimension lda); b: n_raw; rows n_raw..n-1  */
/* are the zero padding of Sec. 2.  SA: col-major r_out x d, ld ldsa.         */
/* ------------------------------------------------------------------------ */
int64_t orc_sketch(const double *A, int64_t lda, const double *b, int64_t n_raw, int64_t d, int64_t r,
                   uint64_t seed, uint64_t instance, int mode, double *SA, int64_t ldsa, double *Sb,
                   int32_t *idx, int64_t cap, int nthreads) {
  if (n_raw < 1 || d < 1 || r < 1 || lda < n_raw) return -ORC_EINVAL;
  int L = log2_pow2(n_raw);
  int64_t n = (int64_t)1 << L;
  int64_t rr = orc_sample(seed, instance, n, r, mode, idx, cap);
  if (rr < 0) return -ORC_ECAPACITY;
  if (ldsa < rr) return -ORC_EINVAL;
  double scale = orc_scale(n, r, mode);
  int8_t *D = (int8_t *)malloc((size_t)n);
  orc_signs(seed, instance, n, D);
  (void)nthreads;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
#endif
  for (int64_t col = 0; col <= d; ++col) {
    const double *x = (col < d) ? A + col * lda : b;
    double *y = (double *)malloc((size_t)n * sizeof(double));
    for (int64_t i = 0; i < n; ++i) y[i] = (i < n_raw) ? D[i] * x[i] : 0.0;
    if (n <= 1024) {
      double *tmp = (double *)malloc((size_t)n * sizeof(double));
      fwht_dense(y, n, tmp);
      free(tmp);
    } else {
      orc_fwht(y, n);
    }
    double *out = (col < d) ? SA + col * ldsa : Sb;
    for (int64_t k = 0; k < rr; ++k) out[k] = scale * y[idx[k]];
    free(y);
  }
  free(D);
  return rr;
}

/* One entry of the sketch straight from the definition, O(n):
 * scale * sum_i (-1)^popcount(row & i) * D_i * X[i].  Used to check
 * full-size GPU results at sampled positions. */
double orc_sketch_entry(const double *x, int64_t n_raw, uint64_t seed, uint64_t instance, int64_t row,
                        double scale) {
  double s = 0.0;
  for (int64_t i = 0; i < n_raw; ++i) {
    double v = orc_sign(seed, instance, (uint64_t)i) * x[i];
    s += (popcount64((uint64_t)(row & i)) & 1) ? -v : v;
  }
  return scale * s;
}

/* ------------------------------------------------------------------------ */
/* Quadratic-programming form of Sec. 3.4: Q = S'S, q = S's.                  */
/* ------------------------------------------------------------------------ */
void orc_gram(const double *S, int64_t lds, const double *s, int64_t m, int64_t d, double *Q, double *q,
              double *ss) {
  for (int64_t i = 0; i < d; ++i) {
    for (int64_t j = 0; j <= i; ++j) {
      double acc = 0.0;
      for (int64_t k = 0; k < m; ++k) acc += S[i * lds + k] * S[j * lds + k];
      Q[i * d + j] = acc;
      Q[j * d + i] = acc;
    }
    double acc = 0.0;
    for (int64_t k = 0; k < m; ++k) acc += S[i * lds + k] * s[k];
    q[i] = acc;
  }
  if (ss) {
    double acc = 0.0;
    for (int64_t k = 0; k < m; ++k) acc += s[k] * s[k];
    *ss = acc;
  }
}

/* Lawson-Hanson tolerance on the dual vector (Matlab lsqnonneg style,
 * 10 * eps * ||S||_1 * max(m, d), times ||s||_2 to make it scale with the
 * right-hand side). */
double orc_lh_tol(const double *S, int64_t lds, const double *s, int64_t m, int64_t d) {
  double norm1 = 0.0;
  for (int64_t j = 0; j < d; ++j) {
    double c = 0.0;
    for (int64_t k = 0; k < m; ++k) c += fabs(S[j * lds + k]);
    if (c > norm1) norm1 = c;
  }
  double s2 = 0.0;
  for (int64_t k = 0; k < m; ++k) s2 += s[k] * s[k];
  const double eps = 2.220446049250313e-16;
  double mx = (double)(m > d ? m : d);
  return 10.0 * eps * norm1 * mx * sqrt(s2);
}

/* Solve Q_PP z_P = q_P by a dense Cholesky of Q_PP (P listed in `pl`,
 * p entries).  A pivot counts as zero when its square is not above
 * ORC_PIVOT_REL * Q_jj (the column is then numerically dependent on the
 * earlier passive columns: the angle to their span is below ~3e-7 rad).
 * Returns 0, or the position of the first zero pivot plus one. */
#define ORC_PIVOT_REL 1e-13
static int passive_solve(const double *Q, const double *q, int64_t d, const int64_t *pl, int64_t p, double *R,
                         double *z) {
  /* R: upper triangular, row-major p x p, Q_PP = R'R. */
  for (int64_t i = 0; i < p; ++i) {
    for (int64_t j = i; j < p; ++j) {
      double v = Q[pl[i] * d + pl[j]];
      for (int64_t k = 0; k < i; ++k) v -= R[k * p + i] * R[k * p + j];
      if (j == i) {
        if (!(v > ORC_PIVOT_REL * Q[pl[i] * d + pl[i]])) return (int)(i + 1);
        R[i * p + i] = sqrt(v);
      } else {
        R[i * p + j] = v / R[i * p + i];
      }
    }
  }
  /* R' u = q_P */
  for (int64_t i = 0; i < p; ++i) {
    double v = q[pl[i]];
    for (int64_t k = 0; k < i; ++k) v -= R[k * p + i] * z[k];
    z[i] = v / R[i * p + i];
  }
  /* R z = u */
  for (int64_t i = p - 1; i >= 0; --i) {
    double v = z[i];
    for (int64_t k = i + 1; k < p; ++k) v -= R[i * p + k] * z[k];
    z[i] = v / R[i * p + i];
  }
  return 0;
}

typedef struct {
  int32_t status;
  int32_t outer_iters;
  int32_t inner_iters;
  int32_t passive_count;
  int64_t trace_len;
} orc_lh_info;

/* Lawson-Hanson NNLS (Lawson & Hanson 1974, ch. 23) on the QP form.
 * Rules (shared with the GPU solver by specification, not by code):
 *   - start from x = 0, P empty (the paper initialises every solve with the
 *     all-zeros vector, Sec. 4.1);
 *   - outer step: w = q - Qx; stop when P is full or max_{j not in P} w_j
 *     <= tol; otherwise take t = argmax (ties -> smallest j);
 *   - the candidate t is rejected (w_t set to 0 for this selection) if the
 *     passive solve with t has z_t <= 0 or a non-positive Cholesky pivot,
 *     as in the original NNLS routine; the next largest w_j is tried;
 *   - inner step while some z_j <= 0 on P: alpha = min x_j/(x_j - z_j) over
 *     those j (ties -> smallest j), x <- x + alpha (z - x), the minimising
 *     index is set to exactly 0, every j in P with x_j <= 0 leaves P;
 *   - caps: max_outer accepted additions, max_inner passive solves in the
 *     inner loops; exceeding either returns ORC_EMAXITER with the current x.
 */
static double qp_objective(const double *Q, const double *q, int64_t d, const double *x) {
  double f = 0.0;
  for (int64_t i = 0; i < d; ++i) {
    double v = 0.0;
    for (int64_t k = 0; k < d; ++k) v += Q[i * d + k] * x[k];
    f += x[i] * (0.5 * v - q[i]);
  }
  return f;
}

/* `trace` (nullable, capacity trace_cap) receives the objective
 * x'Qx/2 - q'x after every update of x, in order; the count is returned in
 * info->trace_len. */
int orc_nnls_lh_traced(const double *Q, const double *q, int64_t d, double tol, int64_t max_outer,
                       int64_t max_inner, double *x, orc_lh_info *info, double *trace, int64_t trace_cap) {
  int8_t *inP = (int8_t *)calloc((size_t)d, 1);
  int8_t *rej = (int8_t *)calloc((size_t)d, 1);
  int64_t *pl = (int64_t *)malloc((size_t)d * sizeof(int64_t));
  double *w = (double *)malloc((size_t)d * sizeof(double));
  double *z = (double *)malloc((size_t)d * sizeof(double));
  double *zp = (double *)malloc((size_t)d * sizeof(double));
  double *R = (double *)malloc((size_t)d * (size_t)d * sizeof(double));
  int status = ORC_OK;
  int64_t outer = 0, inner = 0, p = 0, ntr = 0;
  for (int64_t j = 0; j < d; ++j) x[j] = 0.0;
#define ORC_TRACE()                                                              \
  do {                                                                           \
    if (trace && ntr < trace_cap) trace[ntr] = qp_objective(Q, q, d, x);         \
    ++ntr;                                                                       \
  } while (0)

  for (;;) {
    /* dual vector */
    for (int64_t j = 0; j < d; ++j) {
      double v = q[j];
      for (int64_t k = 0; k < d; ++k) v -= Q[j * d + k] * x[k];
      w[j] = v;
      rej[j] = 0;
    }
    int accepted = 0;
    for (;;) {
      int64_t t = -1;
      double best = 0.0;
      for (int64_t j = 0; j < d; ++j) {
        if (inP[j] || rej[j]) continue;
        if (t < 0 || w[j] > best) {
          best = w[j];
          t = j;
        }
      }
      if (t < 0 || !(best > tol)) break; /* optimal: no candidate above tol */
      /* try t */
      p = 0;
      inP[t] = 1;
      for (int64_t j = 0; j < d; ++j)
        if (inP[j]) pl[p++] = j;
      int bad = passive_solve(Q, q, d, pl, p, R, zp);
      int64_t tpos = -1;
      for (int64_t i = 0; i < p; ++i)
        if (pl[i] == t) tpos = i;
      if (bad || !(zp[tpos] > 0.0)) {
        inP[t] = 0;
        rej[t] = 1;
        continue;
      }
      accepted = 1;
      break;
    }
    if (!accepted) break;
    if (outer >= max_outer) {
      status = ORC_EMAXITER;
      break;
    }
    ++outer;
    /* zp holds the passive solution for the current P (listed in pl) */
    for (;;) {
      ++inner;
      for (int64_t j = 0; j < d; ++j) z[j] = 0.0;
      for (int64_t i = 0; i < p; ++i) z[pl[i]] = zp[i];
      int64_t jmin = -1;
      double alpha = 0.0;
      for (int64_t i = 0; i < p; ++i) {
        int64_t j = pl[i];
        if (z[j] <= 0.0) {
          double a = x[j] / (x[j] - z[j]);
          if (jmin < 0 || a < alpha) {
            alpha = a;
            jmin = j;
          }
        }
      }
      if (jmin < 0) {
        for (int64_t j = 0; j < d; ++j) x[j] = z[j];
        ORC_TRACE();
        break;
      }
      if (inner > max_inner) {
        status = ORC_EMAXITER;
        break;
      }
      for (int64_t i = 0; i < p; ++i) {
        int64_t j = pl[i];
        x[j] = x[j] + alpha * (z[j] - x[j]);
      }
      x[jmin] = 0.0;
      for (int64_t i = 0; i < p; ++i) {
        int64_t j = pl[i];
        if (x[j] <= 0.0) {
          x[j] = 0.0;
          inP[j] = 0;
        }
      }
      ORC_TRACE();
      p = 0;
      for (int64_t j = 0; j < d; ++j)
        if (inP[j]) pl[p++] = j;
      if (p == 0) {
        break;
      }
      int bad = passive_solve(Q, q, d, pl, p, R, zp);
      if (bad) {
        status = ORC_ESINGULAR;
        break;
      }
    }
    if (status != ORC_OK) break;
  }
  int64_t pc = 0;
  for (int64_t j = 0; j < d; ++j) pc += inP[j];
  if (info) {
    info->status = status;
    info->outer_iters = (int32_t)outer;
    info->inner_iters = (int32_t)inner;
    info->passive_count = (int32_t)pc;
    info->trace_len = ntr;
  }
#undef ORC_TRACE
  free(inP);
  free(rej);
  free(pl);
  free(w);
  free(z);
  free(zp);
  free(R);
  return status;
}

int orc_nnls_lh(const double *Q, const double *q, int64_t d, double tol, int64_t max_outer, int64_t max_inner,
                double *x, orc_lh_info *info) {
  return orc_nnls_lh_traced(Q, q, d, tol, max_outer, max_inner, x, info, NULL, 0);
}

/* NNLS of min_{x>=0} ||S x - s||^2 through the QP form, with the default
 * tolerance and caps (3d accepted additions, 30d passive solves). */
int orc_nnls(const double *S, int64_t lds, const double *s, int64_t m, int64_t d, double *x, orc_lh_info *info) {
  double *Q = (double *)malloc((size_t)d * (size_t)d * sizeof(double));
  double *q = (double *)malloc((size_t)d * sizeof(double));
  orc_gram(S, lds, s, m, d, Q, q, NULL);
  double tol = orc_lh_tol(S, lds, s, m, d);
  int st = orc_nnls_lh(Q, q, d, tol, 3 * d, 30 * d, x, info);
  free(Q);
  free(q);
  return st;
}

/* ||A x - b||^2 (Definition 1's objective), FP64, rows in order. */
double orc_residual_sq(const double *A, int64_t lda, const double *b, int64_t n, int64_t d, const double *x) {
  double acc = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double v = -b[i];
    for (int64_t j = 0; j < d; ++j) v += A[j * lda + i] * x[j];
    acc += v * v;
  }
  return acc;
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
