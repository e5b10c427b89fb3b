/*
 * ndg_oracle.c -- plain, slow FP64 CPU oracle for the N-dimensional Gaussian
 * mixture of "N-Dimensional Gaussians for Fitting of High Dimensional
 * Functions" (SIGGRAPH 2024).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header or constant with the CUDA path.
 *
 * Every floating-point input arrives as double (the caller widens its FP32
 * arrays exactly), every computation is FP64 unless a function says it
 * follows the FP32 cull contract, and every loop runs in the order the
 * definition is written in.  Compile with -ffp-contract=off so that no FMA
 * is introduced behind the code's back.
 *
 * Layouts (row-major, one row per Gaussian):
 *   mean   [G][N]        theta  [G][P]  packed lower triangle, row i holds
 *                                       entries (i,0..i); P = N(N+1)/2
 *   alpha  [G]           color  [G][3]
 *   children (one per parent, same shapes): u_theta, m_u, c_alpha, c_color
 * Evaluated Gaussians: e < G is parent e, e >= G is the child of parent e-G
 * (present only when has_children != 0).
 *
 * Parity status of each function is stated in its comment; all of them are
 * pinned by tests against closed forms, brute force or finite differences.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OMAXN 16
#define PIDX(i, j) ((i) * ((i) + 1) / 2 + (j))

static double sigm(double v) { return 1.0 / (1.0 + exp(-v)); }

/* Section 3.1, Eq. 2: L lower triangular, L[i][i] = exp(theta_ii),
 * L[i][j] = 2 sigmoid(theta_ij) - 1 for the strictly lower entries (the paper
 * writes "i<j"; for a lower-triangular factor this is row > column).
 * Output: full N x N row-major matrix with zeros above the diagonal. */
static void act_lower(int N, const double* th, double* L) {
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) {
      double v = 0.0;
      if (j == i) v = exp(th[PIDX(i, i)]);
      else if (j < i) v = 2.0 / (1.0 + exp(-th[PIDX(i, j)])) - 1.0;
      L[i * N + j] = v;
    }
}

/* Eq. 8 context (Section 4.1): brightness alpha = exp(a), colour
 * c = sigmoid(gamma), weight w = alpha * c per RGB channel. */
static void act_weight(double a, const double* gam, double* w) {
  double alpha = exp(a);
  for (int c = 0; c < 3; ++c) w[c] = alpha * sigm(gam[c]);
}

/* Raw parameters -> evaluated Gaussians (L, m, w) in FP64.
 * Section 3.1 (Eq. 1-2) for parents; Section 3.3 (Eq. 6-7) for children:
 * L_c = L_p U and m_c = L_p m_u + m_p, U activated like L. */
void oracle_activate(int N, int G, int has_children, const double* mean,
                     const double* theta, const double* alpha_raw,
                     const double* color_raw, const double* u_theta,
                     const double* m_u, const double* c_alpha_raw,
                     const double* c_color_raw, double* L, double* m,
                     double* w) {
  const int P = N * (N + 1) / 2;
  for (int g = 0; g < G; ++g) {
    double* Lp = L + (size_t)g * N * N;
    act_lower(N, theta + (size_t)g * P, Lp);
    for (int i = 0; i < N; ++i) m[(size_t)g * N + i] = mean[(size_t)g * N + i];
    act_weight(alpha_raw[g], color_raw + (size_t)g * 3, w + (size_t)g * 3);
    if (!has_children) continue;
    size_t e = (size_t)G + g;
    double U[OMAXN * OMAXN];
    act_lower(N, u_theta + (size_t)g * P, U);
    double* Lc = L + e * N * N;
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < N; ++j) {
        double s = 0.0;
        for (int k = 0; k < N; ++k) s += Lp[i * N + k] * U[k * N + j];
        Lc[i * N + j] = s;
      }
    for (int i = 0; i < N; ++i) {
      double s = 0.0;
      for (int k = 0; k < N; ++k) s += Lp[i * N + k] * m_u[(size_t)g * N + k];
      m[e * N + i] = s + mean[(size_t)g * N + i];
    }
    act_weight(c_alpha_raw[g], c_color_raw + (size_t)g * 3, w + e * 3);
  }
}

/* Eq. 1: s = (x-m)^T V^{-1} (x-m) with V = L L^T, computed by solving
 * L z = x - m by forward substitution; s = |z|^2.  Also returns z. */
static double mahalanobis(int N, const double* L, const double* m,
                          const double* x, double* z) {
  double s = 0.0;
  for (int i = 0; i < N; ++i) {
    double r = x[i] - m[i];
    for (int j = 0; j < i; ++j) r -= L[i * N + j] * z[j];
    z[i] = r / L[i * N + i];
    s += z[i] * z[i];
  }
  return s;
}

/* Candidate list of tile t: dense (all Ge) when offsets == NULL. */
static void tile_list(long long t, int Ge, const long long* offsets,
                      const int* ids, const int** lst, long long* n) {
  if (!offsets) { *lst = NULL; *n = Ge; return; }
  *lst = ids + offsets[t];
  *n = offsets[t + 1] - offsets[t];
}

/* Eq. 1 and Eq. 8: y_q = sum over the candidates g of tile(q) of
 * w_g exp(-s_g(x_q)/2).  offsets == NULL evaluates every Gaussian. */
void oracle_eval(int N, int Ge, const double* L, const double* m,
                 const double* w, long long Q, const double* x, int tile,
                 const long long* offsets, const int* ids, double* y) {
#pragma omp parallel for schedule(dynamic, 64)
  for (long long q = 0; q < Q; ++q) {
    const int* lst; long long n;
    tile_list(q / tile, Ge, offsets, ids, &lst, &n);
    double acc[3] = {0.0, 0.0, 0.0}, z[OMAXN];
    for (long long c = 0; c < n; ++c) {
      int g = lst ? lst[c] : (int)c;
      double s = mahalanobis(N, L + (size_t)g * N * N, m + (size_t)g * N,
                             x + q * N, z);
      double ex = exp(-0.5 * s);
      for (int k = 0; k < 3; ++k) acc[k] += w[(size_t)g * 3 + k] * ex;
    }
    for (int k = 0; k < 3; ++k) y[q * 3 + k] = acc[k];
  }
}

/* Per-Gaussian cull radius in units of sigma (Eq. 5 uses 3).  With a
 * contribution cutoff > 0 the radius is the one beyond which
 * w_max exp(-s/2) < cutoff, i.e. sqrt(2 ln(w_max / cutoff)); a Gaussian
 * whose largest weight is below the cutoff is culled everywhere (-1). */
static double cutoff_radius(const double* w, double cutoff, double k_sigma) {
  if (!(cutoff > 0.0)) return k_sigma;
  double wm = w[0];
  if (w[1] > wm) wm = w[1];
  if (w[2] > wm) wm = w[2];
  if (!(wm > cutoff)) return -1.0;
  return sqrt(2.0 * log(wm / cutoff));
}

/* The radius of evaluated Gaussian g.  Section 3.3: a child starts with a
 * negligible, randomised contribution spanning its parent and is optimised
 * with the mixture until it materialises.  Reading R7: a child (g >=
 * n_parents) keeps a radius of at least child_k_min (> 0, e.g. the 3 of
 * Eq. 5) even when its largest weight is below the cutoff, so it is still
 * evaluated, and receives a gradient, where it spans its parent; a larger
 * radius only keeps more pairs, so every dropped contribution stays below
 * the cutoff. */
static double cull_radius(const double* w, double cutoff, double k_sigma, int g, int n_parents,
                          double child_k_min) {
  double r = cutoff_radius(w, cutoff, k_sigma);
  if (g >= n_parents && child_k_min > 0.0 && child_k_min > r) r = child_k_min;
  return r;
}

/* Section 3.2, Eq. 3-5, exact real-valued test in FP64.  For each tile t of
 * `tile` consecutive queries and each projection r_j: the tile's query
 * projections span [lo, hi]; Gaussian g projects to m_r = m^T r_j with
 * sigma_r^2 = r^T V r = |L^T r|^2.  g is kept for t iff for every j the
 * interval [m_r - k sigma_r, m_r + k sigma_r] meets [lo, hi] (it is culled
 * iff the tile lies entirely outside the interval).  keep is [T][Ge]. */
void oracle_cull_exact(int N, int Ge, const double* L, const double* m,
                       const double* w, long long Q, const double* x, int tile,
                       int k, const double* proj, double cutoff,
                       double k_sigma, int n_parents, double child_k_min,
                       unsigned char* keep) {
  long long T = (Q + tile - 1) / tile;
#pragma omp parallel for schedule(dynamic, 4)
  for (long long t = 0; t < T; ++t) {
    long long q0 = t * tile, q1 = q0 + tile < Q ? q0 + tile : Q;
    for (int g = 0; g < Ge; ++g) {
      const double* Lg = L + (size_t)g * N * N;
      const double* mg = m + (size_t)g * N;
      double kg = cull_radius(w + (size_t)g * 3, cutoff, k_sigma, g, n_parents, child_k_min);
      int ok = kg >= 0.0;
      for (int j = 0; ok && j < k; ++j) {
        const double* r = proj + (size_t)j * N;
        double lo = INFINITY, hi = -INFINITY;
        for (long long q = q0; q < q1; ++q) {
          double v = 0.0;
          for (int d = 0; d < N; ++d) v += x[q * N + d] * r[d];
          if (v < lo) lo = v;
          if (v > hi) hi = v;
        }
        double mr = 0.0, s2 = 0.0;
        for (int d = 0; d < N; ++d) mr += mg[d] * r[d];
        for (int c = 0; c < N; ++c) {
          double tc = 0.0;
          for (int i = 0; i < N; ++i) tc += Lg[i * N + c] * r[i];
          s2 += tc * tc;
        }
        double sr = sqrt(s2);
        if (mr + kg * sr < lo || mr - kg * sr > hi) ok = 0;
      }
      keep[t * Ge + g] = (unsigned char)ok;
    }
  }
}

/* ---- FP32 bucket contract -------------------------------------------------
 * The exact test is real-valued; a CPU/GPU bit-exact candidate set needs an
 * integer contract computed from identical FP32 values with a fixed order of
 * correctly rounded operations (no contraction):
 *   - FP32 inputs: L, m, w rounded once from the FP64 activations above;
 *     queries and projections as given.
 *   - every dot product is an fmaf chain in ascending index order starting
 *     from 0; sigma_r = sqrtf(sum_c (sum_{i>=c} L[i][c] r_i)^2), the inner sum
 *     over ascending i, the outer over ascending c.
 *   - k_g = (float) of the FP64 cull radius computed from the FP32 weights.
 *   - per projection: lo_j / hi_j = min / max over all queries of q_r;
 *     inv_h_j = B / (hi_j - lo_j) in FP32, or 0 when the range is not wider
 *     than 1e-3 (1 + max(|lo_j|, |hi_j|)).
 *   - bucket(v) = floor((v - lo_j) * inv_h_j), saturated to [-2, B+1].
 *   - Gaussian: blo = bucket(m_r - k sigma_r) - 1, bhi = bucket(m_r + k sigma_r)
 *     + 1; if bhi < 0 or blo > B-1 the Gaussian misses every query and is
 *     culled everywhere; else both are clamped to [0, B-1].
 *   - tile: tlo = bucket(min q_r), thi = bucket(max q_r) clamped to [0, B-1].
 *   - g in cand(t) iff k_g >= 0 and blo <= thi and tlo <= bhi for every j.
 * The +-1 bucket of slack absorbs FP32 rounding against the real test. */

static float dotf(int N, const float* a, const float* b) {
  float acc = 0.0f;
  for (int d = 0; d < N; ++d) acc = fmaf(a[d], b[d], acc);
  return acc;
}

static int bucket_raw(float v, float lo, float inv_h, int B) {
  float t = (v - lo) * inv_h;
  if (t != t) return 0;
  if (t < -1.0f) return -2;
  if (t >= (float)(B + 1)) return B + 1;
  return (int)floorf(t);
}

/* Section 3.2: when every input beyond position is constant for an image,
 * x_c = (x_4, .., x_N), each Gaussian restricted to x_c is a 3-D Gaussian
 * over position.  With the precision A = V^-1 = M^T M (M = L^-1) split into
 * the position block p (dims 0-2) and the rest c, completing the square gives
 *   (x - m)^T A (x - m) = (x_p - mu)^T A_pp (x_p - mu) + q_c,
 *   b = A_pc d_c, d_c = x_c - m_c, mu = m_p - A_pp^-1 b,
 *   q_c = d_c^T A_cc d_c - b^T A_pp^-1 b,
 * so the restriction is w exp(-q_c / 2) times a 3-D Gaussian with mean mu
 * and covariance A_pp^-1 = T^T T, T = C^-1 for A_pp = C C^T (Cholesky).
 * Per Gaussian g (N >= 4): mu [3], T [9] (row-major, lower), and the
 * conditional weight wc [3] = w exp(-q_c / 2) with w the weights given. */
void oracle_condition(int N, int Ge, const double* L, const double* m,
                      const double* w, const double* xc, double* mu, double* T,
                      double* wc) {
#pragma omp parallel for schedule(static)
  for (int g = 0; g < Ge; ++g) {
    const double* Lg = L + (size_t)g * N * N;
    const double* mg = m + (size_t)g * N;
    double M[OMAXN * OMAXN], A[OMAXN * OMAXN];
    /* M = L^-1 by forward substitution, column by column */
    for (int j = 0; j < N; ++j) {
      for (int i = 0; i < N; ++i) M[i * N + j] = 0.0;
      M[j * N + j] = 1.0 / Lg[j * N + j];
      for (int i = j + 1; i < N; ++i) {
        double s = 0.0;
        for (int k = j; k < i; ++k) s += Lg[i * N + k] * M[k * N + j];
        M[i * N + j] = -s / Lg[i * N + i];
      }
    }
    /* A = M^T M */
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < N; ++j) {
        double s = 0.0;
        for (int k = 0; k < N; ++k) s += M[k * N + i] * M[k * N + j];
        A[i * N + j] = s;
      }
    double dc[OMAXN], b[3];
    for (int i = 3; i < N; ++i) dc[i] = xc[i - 3] - mg[i];
    for (int i = 0; i < 3; ++i) {
      double s = 0.0;
      for (int k = 3; k < N; ++k) s += A[i * N + k] * dc[k];
      b[i] = s;
    }
    /* Cholesky of A_pp (3 x 3): C lower with C C^T = A_pp */
    double C[9];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j <= i; ++j) {
        double s = A[i * N + j];
        for (int k = 0; k < j; ++k) s -= C[i * 3 + k] * C[j * 3 + k];
        C[i * 3 + j] = (i == j) ? sqrt(s) : s / C[j * 3 + j];
      }
    /* z = A_pp^-1 b: C y = b, C^T z = y */
    double y3[3], z[3];
    for (int i = 0; i < 3; ++i) {
      double s = b[i];
      for (int k = 0; k < i; ++k) s -= C[i * 3 + k] * y3[k];
      y3[i] = s / C[i * 3 + i];
    }
    for (int i = 2; i >= 0; --i) {
      double s = y3[i];
      for (int k = i + 1; k < 3; ++k) s -= C[k * 3 + i] * z[k];
      z[i] = s / C[i * 3 + i];
    }
    double qc = 0.0;
    for (int i = 3; i < N; ++i) {
      double s = 0.0;
      for (int k = 3; k < N; ++k) s += A[i * N + k] * dc[k];
      qc += dc[i] * s;
    }
    for (int i = 0; i < 3; ++i) qc -= b[i] * z[i];
    const double f = exp(-0.5 * qc);
    for (int i = 0; i < 3; ++i) {
      mu[(size_t)g * 3 + i] = mg[i] - z[i];
      wc[(size_t)g * 3 + i] = w[(size_t)g * 3 + i] * f;
    }
    /* T = C^-1 (lower) by forward substitution */
    double* Tg = T + (size_t)g * 9;
    for (int j = 0; j < 3; ++j) {
      for (int i = 0; i < 3; ++i) Tg[i * 3 + j] = 0.0;
      Tg[j * 3 + j] = 1.0 / C[j * 3 + j];
      for (int i = j + 1; i < 3; ++i) {
        double s = 0.0;
        for (int k = j; k < i; ++k) s += C[i * 3 + k] * Tg[k * 3 + j];
        Tg[i * 3 + j] = -s / C[i * 3 + i];
      }
    }
  }
}

/* Runs the contract; writes the candidate lists as CSR (ascending ids per
 * tile).  ids may be NULL to count only.  Returns E, the total entries.
 * sel == NULL: every tile, offsets [T+1].  Otherwise only the n_sel tiles
 * listed in sel (in that order), offsets [n_sel+1]; the global per-projection
 * ranges and the keys are the same as for the whole query set, so each
 * selected tile's list equals its list in the full run.
 * xc != NULL (N >= 4, the inputs beyond position constant, xc [N - 3]): the
 * same contract on the position dims only, for the Gaussians restricted to
 * xc (oracle_condition): a Gaussian's key uses mu, T and the conditional
 * weight, rounded to FP32 (sigma_r = |T r|), and every projection and query
 * enters with its first three components. */
long long oracle_cull_contract(int N, int Ge, const double* L, const double* m,
                               const double* w, long long Q, const double* x,
                               int tile, int k, const double* proj,
                               double cutoff, double k_sigma, int B,
                               int n_parents, double child_k_min,
                               long long n_sel, const long long* sel,
                               const double* xc, long long* offsets, int* ids) {
  long long T = (Q + tile - 1) / tile;
  float* xf = (float*)malloc(sizeof(float) * (size_t)(Q * N + 1));
  float* rf = (float*)malloc(sizeof(float) * (size_t)(k * N + 1));
  float* qv = (float*)malloc(sizeof(float) * (size_t)(Q * (k ? k : 1)));
  float* lo = (float*)malloc(sizeof(float) * (size_t)(k + 1));
  float* hi = (float*)malloc(sizeof(float) * (size_t)(k + 1));
  float* ih = (float*)malloc(sizeof(float) * (size_t)(k + 1));
  int* gk = (int*)malloc(sizeof(int) * (size_t)Ge * (2 * k + 1));
  int* tk = (int*)malloc(sizeof(int) * (size_t)T * (2 * k + 1));
  for (long long i = 0; i < Q * N; ++i) xf[i] = (float)x[i];
  for (long long i = 0; i < (long long)k * N; ++i) rf[i] = (float)proj[i];
  const int ND = xc ? 3 : N;  /* dims that enter the projections */
  double *cmu = NULL, *cT = NULL, *cw = NULL;
  if (xc) {
    double* wr = (double*)malloc(sizeof(double) * (size_t)Ge * 3 + 8);
    cmu = (double*)malloc(sizeof(double) * (size_t)Ge * 3 + 8);
    cT = (double*)malloc(sizeof(double) * (size_t)Ge * 9 + 8);
    cw = (double*)malloc(sizeof(double) * (size_t)Ge * 3 + 8);
    /* the conditional weight starts from the FP32 weights, as the key does */
    for (long long i = 0; i < (long long)Ge * 3; ++i) wr[i] = (double)(float)w[i];
    oracle_condition(N, Ge, L, m, wr, xc, cmu, cT, cw);
    free(wr);
  }
  for (int j = 0; j < k; ++j) {
    lo[j] = INFINITY;
    hi[j] = -INFINITY;
    for (long long q = 0; q < Q; ++q) {
      float v = dotf(ND, xf + q * N, rf + (size_t)j * N);
      qv[q * k + j] = v;
      if (v < lo[j]) lo[j] = v;
      if (v > hi[j]) hi[j] = v;
    }
    float range = hi[j] - lo[j];
    float mag = fabsf(lo[j]) > fabsf(hi[j]) ? fabsf(lo[j]) : fabsf(hi[j]);
    ih[j] = (Q > 0 && range > 1e-3f * (1.0f + mag)) ? (float)B / range : 0.0f;
  }
  /* Gaussian keys: gk[g][0] = live flag, then (blo, bhi) per projection. */
  for (int g = 0; g < Ge; ++g) {
    int* key = gk + (size_t)g * (2 * k + 1);
    float Lf[OMAXN * OMAXN], mf[OMAXN], wf[3];
    double wd[3];
    if (xc) {  /* the position-only Gaussian: mean mu, factor T^T, weight wc */
      for (int i = 0; i < 9; ++i) Lf[i] = (float)cT[(size_t)g * 9 + i];
      for (int i = 0; i < 3; ++i) mf[i] = (float)cmu[(size_t)g * 3 + i];
      for (int c = 0; c < 3; ++c) { wf[c] = (float)cw[(size_t)g * 3 + c]; wd[c] = wf[c]; }
    } else {
      for (int i = 0; i < N * N; ++i) Lf[i] = (float)L[(size_t)g * N * N + i];
      for (int i = 0; i < N; ++i) mf[i] = (float)m[(size_t)g * N + i];
      for (int c = 0; c < 3; ++c) { wf[c] = (float)w[(size_t)g * 3 + c]; wd[c] = wf[c]; }
    }
    double kgd = cull_radius(wd, (double)(float)cutoff, (double)(float)k_sigma, g, n_parents,
                             (double)(float)child_k_min);
    key[0] = kgd >= 0.0;
    float kg = (float)kgd;
    for (int j = 0; key[0] && j < k; ++j) {
      const float* r = rf + (size_t)j * N;
      float mr = dotf(ND, mf, r);
      float s2 = 0.0f;
      if (xc) {  /* sigma_r^2 = |T r|^2, T lower (row-major 3 x 3) */
        for (int i = 0; i < 3; ++i) {
          float tc = 0.0f;
          for (int c = 0; c <= i; ++c) tc = fmaf(Lf[i * 3 + c], r[c], tc);
          s2 = fmaf(tc, tc, s2);
        }
      } else {
        for (int c = 0; c < N; ++c) {
          float tc = 0.0f;
          for (int i = c; i < N; ++i) tc = fmaf(Lf[i * N + c], r[i], tc);
          s2 = fmaf(tc, tc, s2);
        }
      }
      float sr = sqrtf(s2);
      float ks = kg * sr;
      int blo = bucket_raw(mr - ks, lo[j], ih[j], B) - 1;
      int bhi = bucket_raw(mr + ks, lo[j], ih[j], B) + 1;
      if (bhi < 0 || blo > B - 1) { key[0] = 0; break; }
      key[1 + 2 * j] = blo < 0 ? 0 : blo;
      key[2 + 2 * j] = bhi > B - 1 ? B - 1 : bhi;
    }
  }
  for (long long t = 0; t < T; ++t) {
    long long q0 = t * tile, q1 = q0 + tile < Q ? q0 + tile : Q;
    int* key = tk + t * (2 * k + 1);
    for (int j = 0; j < k; ++j) {
      float a = INFINITY, b = -INFINITY;
      for (long long q = q0; q < q1; ++q) {
        float v = qv[q * k + j];
        if (v < a) a = v;
        if (v > b) b = v;
      }
      int tl = bucket_raw(a, lo[j], ih[j], B), th = bucket_raw(b, lo[j], ih[j], B);
      key[1 + 2 * j] = tl < 0 ? 0 : (tl > B - 1 ? B - 1 : tl);
      key[2 + 2 * j] = th < 0 ? 0 : (th > B - 1 ? B - 1 : th);
    }
  }
  /* Overlap test of every Gaussian against each (selected) tile: a count
   * pass, the list offsets, then a fill pass (tiles are independent). */
  const long long nt = sel ? n_sel : T;
  long long* cnt = (long long*)malloc(sizeof(long long) * (size_t)(nt + 1));
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 1 && !ids) break;
#pragma omp parallel for schedule(dynamic, 1)
    for (long long i = 0; i < nt; ++i) {
      const long long t = sel ? sel[i] : i;
      const int* tkey = tk + t * (2 * k + 1);
      long long e = pass ? cnt[i] : 0;
      for (int g = 0; g < Ge; ++g) {
        const int* key = gk + (size_t)g * (2 * k + 1);
        int ok = key[0];
        for (int j = 0; ok && j < k; ++j)
          if (key[1 + 2 * j] > tkey[2 + 2 * j] || tkey[1 + 2 * j] > key[2 + 2 * j]) ok = 0;
        if (ok) {
          if (pass) ids[e] = g;
          ++e;
        }
      }
      if (!pass) cnt[i] = e;
    }
    if (pass == 0) {  /* counts -> offsets */
      long long E = 0;
      for (long long i = 0; i < nt; ++i) {
        const long long c = cnt[i];
        cnt[i] = E;
        E += c;
      }
      cnt[nt] = E;
    }
  }
  const long long E = cnt[nt];
  if (offsets)
    for (long long i = 0; i <= nt; ++i) offsets[i] = cnt[i];
  free(cnt);
  free(cmu); free(cT); free(cw);
  free(xf); free(rf); free(qv); free(lo); free(hi); free(ih); free(gk); free(tk);
  return E;
}

/* Plain L2 loss (mean over Q x 3 outputs) and its gradient with respect to
 * the outputs: l = sum (y - t)^2 / (3Q), dl/dy = 2 (y - t) / (3Q). */
double oracle_loss_l2(long long Q, const double* y, const double* target,
                      double* gbar) {
  double acc = 0.0, n = 3.0 * (double)Q;
  for (long long i = 0; i < 3 * Q; ++i) {
    double d = y[i] - target[i];
    acc += d * d;
    if (gbar) gbar[i] = 2.0 * d / n;
  }
  return Q > 0 ? acc / n : 0.0;
}

/* Relative L2.  Section 4.1 trains with a relative L2 loss (after
 * Noise2Noise) without printing it; the reading taken here: each squared
 * error is divided by the square of the output itself plus eps, and the
 * denominator is held constant when differentiating:
 *   l = sum (y - t)^2 / (y^2 + eps) / (3Q),
 *   dl/dy = 2 (y - t) / (y^2 + eps) / (3Q). */
double oracle_loss_rel_l2(long long Q, const double* y, const double* target,
                          double eps, double* gbar) {
  double acc = 0.0, n = 3.0 * (double)Q;
  for (long long i = 0; i < 3 * Q; ++i) {
    double d = y[i] - target[i];
    double den = y[i] * y[i] + eps;
    acc += d * d / den;
    if (gbar) gbar[i] = 2.0 * d / den / n;
  }
  return Q > 0 ? acc / n : 0.0;
}

/* Is g in the sorted candidate list of tile t (dense when offsets == NULL)? */
static int in_tile(long long t, int g, const long long* offsets, const int* ids) {
  if (!offsets) return 1;
  long long a = offsets[t], b = offsets[t + 1];
  while (a < b) {
    long long c = (a + b) / 2;
    if (ids[c] == g) return 1;
    if (ids[c] < g) a = c + 1; else b = c;
  }
  return 0;
}

/* Gradient of the loss with respect to every raw parameter, given
 * gbar = dl/dy.  Derived independently of the GPU's matrix form:
 *   z = L^{-1} d, d = x - m, s = |z|^2, u = L^{-T} z.  Differentiating
 *   L z = d gives dz = L^{-1}(dd - dL z), so ds = 2 z^T dz yields
 *   ds/dL_ij = -2 u_i z_j (i >= j) and ds/dm = -2 u.
 *   dl/ds = -1/2 exp(-s/2) sum_c gbar_c w_c; dl/dw_c = gbar_c exp(-s/2).
 * Children (Eq. 6-7): L_c = L_p U, m_c = L_p m_u + m_p, chained by the
 * product rule entry by entry; activations (Eq. 2, Eq. 8) by their
 * derivatives written from theta: exp for the diagonal, 2 sig (1 - sig) for
 * the strictly lower entries and the colour, alpha for the brightness.
 * The candidate lists must be ascending per tile (or offsets == NULL). */
void oracle_grad(int N, int G, int has_children, const double* mean,
                 const double* theta, const double* alpha_raw,
                 const double* color_raw, const double* u_theta,
                 const double* m_u, const double* c_alpha_raw,
                 const double* c_color_raw, long long Q, const double* x,
                 int tile, const long long* offsets, const int* ids,
                 const double* gbar, double* g_mean, double* g_theta,
                 double* g_alpha, double* g_color, double* g_u_theta,
                 double* g_m_u, double* g_c_alpha, double* g_c_color) {
  const int P = N * (N + 1) / 2;
  const int Ge = has_children ? 2 * G : G;
  double* L = (double*)malloc(sizeof(double) * (size_t)Ge * N * N + 8);
  double* m = (double*)malloc(sizeof(double) * (size_t)Ge * N + 8);
  double* w = (double*)malloc(sizeof(double) * (size_t)Ge * 3 + 8);
  double* GL = (double*)calloc((size_t)Ge * N * N + 1, sizeof(double));
  double* Gm = (double*)calloc((size_t)Ge * N + 1, sizeof(double));
  double* Gw = (double*)calloc((size_t)Ge * 3 + 1, sizeof(double));
  oracle_activate(N, G, has_children, mean, theta, alpha_raw, color_raw,
                  u_theta, m_u, c_alpha_raw, c_color_raw, L, m, w);
  long long T = (Q + tile - 1) / tile;
#pragma omp parallel for schedule(dynamic, 1)
  for (int e = 0; e < Ge; ++e) {
    const double* Le = L + (size_t)e * N * N;
    const double* me = m + (size_t)e * N;
    const double* we = w + (size_t)e * 3;
    double* gL = GL + (size_t)e * N * N;
    double* gm = Gm + (size_t)e * N;
    double* gw = Gw + (size_t)e * 3;
    double z[OMAXN], u[OMAXN];
    for (long long t = 0; t < T; ++t) {
      if (!in_tile(t, e, offsets, ids)) continue;
      long long q1 = (t + 1) * tile < Q ? (t + 1) * tile : Q;
      for (long long q = t * tile; q < q1; ++q) {
        double s = mahalanobis(N, Le, me, x + q * N, z);
        double ex = exp(-0.5 * s);
        const double* gb = gbar + q * 3;
        double h = 0.0;
        for (int c = 0; c < 3; ++c) {
          gw[c] += gb[c] * ex;
          h += gb[c] * we[c];
        }
        h *= -0.5 * ex; /* dl/ds */
        for (int i = N - 1; i >= 0; --i) { /* L^T u = z, back substitution */
          double r = z[i];
          for (int j = i + 1; j < N; ++j) r -= Le[j * N + i] * u[j];
          u[i] = r / Le[i * N + i];
        }
        for (int i = 0; i < N; ++i) {
          gm[i] += h * (-2.0 * u[i]);
          for (int j = 0; j <= i; ++j) gL[i * N + j] += h * (-2.0 * u[i] * z[j]);
        }
      }
    }
  }
  /* Chain to the raw parameters. */
  for (int g = 0; g < G; ++g) {
    const double* Lp = L + (size_t)g * N * N;
    double gLp[OMAXN * OMAXN], gmp[OMAXN];
    for (int i = 0; i < N * N; ++i) gLp[i] = GL[(size_t)g * N * N + i];
    for (int i = 0; i < N; ++i) gmp[i] = Gm[(size_t)g * N + i];
    if (has_children) {
      size_t c = (size_t)G + g;
      const double* gLc = GL + c * N * N;
      const double* gmc = Gm + c * N;
      const double* mu = m_u + (size_t)g * N;
      double U[OMAXN * OMAXN];
      act_lower(N, u_theta + (size_t)g * P, U);
      /* L_c[i][k] = sum_j L_p[i][j] U[j][k]  =>  dLc_ik/dLp_ij = U_jk */
      for (int i = 0; i < N; ++i)
        for (int j = 0; j <= i; ++j) {
          double s = 0.0;
          for (int k = 0; k < N; ++k) s += gLc[i * N + k] * U[j * N + k];
          gLp[i * N + j] += s + gmc[i] * mu[j];
        }
      for (int i = 0; i < N; ++i) gmp[i] += gmc[i];
      /* dLc_ik/dU_jk = L_p[i][j] */
      for (int j = 0; j < N; ++j)
        for (int k = 0; k <= j; ++k) {
          double s = 0.0;
          for (int i = 0; i < N; ++i) s += Lp[i * N + j] * gLc[i * N + k];
          double th = u_theta[(size_t)g * P + PIDX(j, k)];
          double dact = (j == k) ? exp(th) : 2.0 * sigm(th) * (1.0 - sigm(th));
          g_u_theta[(size_t)g * P + PIDX(j, k)] = s * dact;
        }
      for (int j = 0; j < N; ++j) {
        double s = 0.0;
        for (int i = 0; i < N; ++i) s += Lp[i * N + j] * gmc[i];
        g_m_u[(size_t)g * N + j] = s;
      }
      double ac = exp(c_alpha_raw[g]), ga = 0.0;
      for (int k = 0; k < 3; ++k) {
        double sg = sigm(c_color_raw[(size_t)g * 3 + k]);
        ga += Gw[c * 3 + k] * ac * sg;
        g_c_color[(size_t)g * 3 + k] = Gw[c * 3 + k] * ac * sg * (1.0 - sg);
      }
      g_c_alpha[g] = ga;
    }
    for (int i = 0; i < N; ++i) {
      g_mean[(size_t)g * N + i] = gmp[i];
      for (int j = 0; j <= i; ++j) {
        double th = theta[(size_t)g * P + PIDX(i, j)];
        double dact = (j == i) ? exp(th) : 2.0 * sigm(th) * (1.0 - sigm(th));
        g_theta[(size_t)g * P + PIDX(i, j)] = gLp[i * N + j] * dact;
      }
    }
    double ap = exp(alpha_raw[g]), ga = 0.0;
    for (int k = 0; k < 3; ++k) {
      double sg = sigm(color_raw[(size_t)g * 3 + k]);
      ga += Gw[(size_t)g * 3 + k] * ap * sg;
      g_color[(size_t)g * 3 + k] = Gw[(size_t)g * 3 + k] * ap * sg * (1.0 - sg);
    }
    g_alpha[g] = ga;
  }
  free(L); free(m); free(w); free(GL); free(Gm); free(Gw);
}

/* Adam (Kingma & Ba 2015, Algorithm 1) on n scalars, step t >= 1; the paper
 * does not name its optimiser. */
void oracle_adam(long long n, double* p, const double* g, double* m1,
                 double* m2, int t, double lr, double b1, double b2,
                 double eps) {
  double c1 = 1.0 - pow(b1, t), c2 = 1.0 - pow(b2, t);
  for (long long i = 0; i < n; ++i) {
    m1[i] = b1 * m1[i] + (1.0 - b1) * g[i];
    m2[i] = b2 * m2[i] + (1.0 - b2) * g[i] * g[i];
    double mh = m1[i] / c1, vh = m2[i] / c2;
    p[i] -= lr * mh / (sqrt(vh) + eps);
  }
}

/* Section 3.3 refinement step (materialisation).  A child whose brightness
 * raw value exceeds a_thr (= ln t rounded to FP32 by the caller) becomes an
 * independent Gaussian appended at row G + rank: L = L_p U written back to
 * raw form (theta_ii = ln L_ii, theta_ij = ln((1+L)/(1-L)) after clamping
 * |L_ij| to 1 - 1e-6), m = L_p m_u + m_p, and the child's own brightness and
 * colour.  At most G_cap - G children materialise; when more qualify, the
 * largest raw brightness values win and ties at the boundary are all left
 * out.  Every materialised parent and every new row then receives a fresh
 * child drawn from its noise row (standard normals, one row per slot,
 * P + N + 4 values): u_theta = 0.05 xi, m_u = 0.1 xi, c_alpha = ln(t/10)
 * + 0.1 xi, c_color = own colour + 0.1 xi.  With has_children == 0 no child
 * exists yet: every parent receives a fresh child and nothing materialises.
 * Raw arrays have G_cap rows and are updated in place; mat_flag[G] records
 * which parents materialised.  Returns the new G. */
static int desc_double(const void* a, const void* b) {
  double x = *(const double*)a, y = *(const double*)b;
  return (x < y) - (x > y);
}

int oracle_densify(int N, int G, int G_cap, int has_children, double a_thr,
                   double a_child0, double* mean, double* theta,
                   double* alpha_raw, double* color_raw, double* u_theta,
                   double* m_u, double* c_alpha_raw, double* c_color_raw,
                   const double* noise, unsigned char* mat_flag) {
  const int P = N * (N + 1) / 2, NR = P + N + 4;
  int room = G_cap - G, nflag = 0;
  unsigned char* fresh = (unsigned char*)calloc((size_t)G_cap + 1, 1);
  for (int g = 0; g < G; ++g) {
    mat_flag[g] = has_children && c_alpha_raw[g] > a_thr;
    nflag += mat_flag[g];
  }
  if (nflag > room) {
    /* keep the `room` largest raw brightness values; when the room-th
     * largest value is tied with values beyond the room, all of that value
     * are left out */
    double* v = (double*)malloc(sizeof(double) * (size_t)(nflag + 1));
    int n = 0;
    for (int g = 0; g < G; ++g) if (mat_flag[g]) v[n++] = c_alpha_raw[g];
    qsort(v, (size_t)n, sizeof(double), desc_double);
    if (room > 0) {
      double thr = v[room - 1];
      int with_eq = 0;
      for (int i = 0; i < n; ++i) if (v[i] >= thr) ++with_eq;
      for (int g = 0; g < G; ++g) {
        if (!mat_flag[g]) continue;
        int keepit = with_eq > room ? c_alpha_raw[g] > thr : c_alpha_raw[g] >= thr;
        mat_flag[g] = (unsigned char)keepit;
      }
    } else {
      for (int g = 0; g < G; ++g) mat_flag[g] = 0;
    }
    free(v);
  }
  int Gn = G;
  for (int g = 0; g < G; ++g) {
    if (!mat_flag[g]) continue;
    int d = Gn++;
    double Lp[OMAXN * OMAXN], U[OMAXN * OMAXN];
    act_lower(N, theta + (size_t)g * P, Lp);
    act_lower(N, u_theta + (size_t)g * P, U);
    for (int i = 0; i < N; ++i) {
      double s = 0.0;
      for (int k = 0; k < N; ++k) s += Lp[i * N + k] * m_u[(size_t)g * N + k];
      mean[(size_t)d * N + i] = s + mean[(size_t)g * N + i];
      for (int j = 0; j <= i; ++j) {
        double lc = 0.0;
        for (int k = 0; k < N; ++k) lc += Lp[i * N + k] * U[k * N + j];
        double th;
        if (i == j) th = log(lc);
        else {
          double lim = 1.0 - 1e-6;
          if (lc > lim) lc = lim;
          if (lc < -lim) lc = -lim;
          th = log((1.0 + lc) / (1.0 - lc));
        }
        theta[(size_t)d * P + PIDX(i, j)] = th;
      }
    }
    alpha_raw[d] = c_alpha_raw[g];
    for (int k = 0; k < 3; ++k) color_raw[(size_t)d * 3 + k] = c_color_raw[(size_t)g * 3 + k];
    fresh[g] = 1;
    fresh[d] = 1;
  }
  for (int g = 0; g < Gn; ++g) {
    if (has_children && !fresh[g]) continue;
    const double* xi = noise + (size_t)g * NR;
    for (int i = 0; i < P; ++i) u_theta[(size_t)g * P + i] = 0.05 * xi[i];
    for (int i = 0; i < N; ++i) m_u[(size_t)g * N + i] = 0.1 * xi[P + i];
    c_alpha_raw[g] = a_child0 + 0.1 * xi[P + N];
    for (int k = 0; k < 3; ++k)
      c_color_raw[(size_t)g * 3 + k] = color_raw[(size_t)g * 3 + k] + 0.1 * xi[P + N + 1 + k];
  }
  free(fresh);
  return Gn;
}

/* Host threads the parallel loops above use (1 without OpenMP), and a way
 * to change that count (timing of the oracle on one core and on all). */
int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
