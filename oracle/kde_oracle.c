/*
 * kde_oracle.c -- FP64 CPU oracle for exact kernel-density bandwidth selection,
 * following Gramacki & Andrzejewski, "Density Estimations for Approximate Query
 * Processing on SIMD Architectures" (arXiv 1505.01998).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the plain, slow, obviously correct
 * statement of what the CUDA library computes.  Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header, constant table or helper with the CUDA path, and it never calls it.
 *
 * Conventions
 *  - Samples are a d x n matrix with one sample per column, stored row-major:
 *    x[k*n + i] is coordinate k of sample i (Sec. 4.4.2, Eq. LSCV-InputData).
 *  - All arithmetic is IEEE double, round to nearest.  Every sum over pairs is
 *    an explicit double loop over i<j.  Each row i keeps its own Neumaier-
 *    compensated sum over j>i; the row sums are then added in index order with
 *    the same compensation, so results do not depend on the thread count.
 *  - Readings of the paper where it is garbled or silent (numbered as in the
 *    design notes):
 *      R1  psi_r normalisation: the n K^(r)(0) diagonal term sits inside the
 *          n^-2 g^-(r+1) factor (Sec. 4.4.1, Eqs. PLUGIN-Psi6Estimate and
 *          PLUGIN-Psi4Estimate print it outside, which is dimensionally wrong).
 *      R2  LSCV uses n^-2 on the pair sum, as printed (Eq. LSCV-gh).
 *      R3  R(K) in g(h) is (4 pi)^(-d/2) |Sigma|^(-1/2) (Eqs. LSCV-Kx, LSCV-KKx,
 *          LSCV_MULTI-rk at H = h^2 Sigma).
 *      R4  h0 = (4/((d+2) n))^(1/(d+4)) (normal scale; equals Eq. LSCV-h0 at d=1).
 *      R7  variances and covariances are computed two-pass (mean first), which
 *          equals Eqs. PLUGIN-VarianceEstimator / LSCV-covariance exactly.
 *  - Parity pins: psi sums, plug-in chain, g(h), g(H): pinned by the tests
 *    (closed forms, brute force, quadrature, invariants).  Nothing here is
 *    "parity unpinned".
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define KDEO_OK 0
#define KDEO_EDEGENERATE 1
#define KDEO_EINVAL 2
#define KDEO_ENOMEM 3

static const double KDEO_PI = 3.14159265358979323846264338327950288;

/* ---------------------------------------------------------------- sums */

typedef struct {
  double s, c;
} nsum_t;

/* Neumaier's improvement of Kahan summation. */
static void nsum_add(nsum_t *a, double v) {
  double t = a->s + v;
  if (fabs(a->s) >= fabs(v))
    a->c += (a->s - t) + v;
  else
    a->c += (v - t) + a->s;
  a->s = t;
}

static double nsum_get(const nsum_t *a) { return a->s + a->c; }

static int pick_threads(int threads) {
#ifdef _OPENMP
  if (threads <= 0) return omp_get_max_threads();
  return threads;
#else
  (void)threads;
  return 1;
#endif
}

int kdeo_have_openmp(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 0;
#endif
}

/* --------------------------------------------------- sample statistics */

/* Mean vector and covariance matrix with the n-1 denominator
 * (Sec. 4.4.2, Eqs. LSCV-CovarianceMatrix, LSCV-variance, LSCV-covariance;
 * for d=1 this is Eq. PLUGIN-VarianceEstimator).  Two-pass form (R7). */
int kdeo_mean_cov(const double *x, long n, int d, double *mean, double *cov) {
  if (n < 2 || d < 1) return KDEO_EINVAL;
  for (int a = 0; a < d; ++a) {
    nsum_t s = {0, 0};
    for (long i = 0; i < n; ++i) nsum_add(&s, x[(long)a * n + i]);
    mean[a] = nsum_get(&s) / (double)n;
  }
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < d; ++b) {
      nsum_t s = {0, 0};
      for (long i = 0; i < n; ++i)
        nsum_add(&s, (x[(long)a * n + i] - mean[a]) * (x[(long)b * n + i] - mean[b]));
      cov[a * d + b] = nsum_get(&s) / (double)(n - 1);
    }
  return KDEO_OK;
}

/* Determinant and inverse of a small dense matrix by Gauss-Jordan elimination
 * with partial pivoting (Sec. 4.4.2, steps 2 and 3: det(Sigma), Sigma^-1). */
int kdeo_invert(const double *A, int d, double *Ainv, double *det) {
  double *m = (double *)malloc(sizeof(double) * (size_t)(d * 2 * d));
  if (!m) return KDEO_ENOMEM;
  for (int r = 0; r < d; ++r)
    for (int c = 0; c < 2 * d; ++c)
      m[r * 2 * d + c] = c < d ? A[r * d + c] : (c - d == r ? 1.0 : 0.0);
  double dt = 1.0;
  for (int col = 0; col < d; ++col) {
    int piv = col;
    for (int r = col + 1; r < d; ++r)
      if (fabs(m[r * 2 * d + col]) > fabs(m[piv * 2 * d + col])) piv = r;
    double p = m[piv * 2 * d + col];
    if (p == 0.0) {
      free(m);
      *det = 0.0;
      return KDEO_EDEGENERATE;
    }
    if (piv != col) {
      for (int c = 0; c < 2 * d; ++c) {
        double t = m[col * 2 * d + c];
        m[col * 2 * d + c] = m[piv * 2 * d + c];
        m[piv * 2 * d + c] = t;
      }
      dt = -dt;
    }
    dt *= p;
    for (int c = 0; c < 2 * d; ++c) m[col * 2 * d + c] /= p;
    for (int r = 0; r < d; ++r) {
      if (r == col) continue;
      double f = m[r * 2 * d + col];
      if (f == 0.0) continue;
      for (int c = 0; c < 2 * d; ++c) m[r * 2 * d + c] -= f * m[col * 2 * d + c];
    }
  }
  for (int r = 0; r < d; ++r)
    for (int c = 0; c < d; ++c) Ainv[r * d + c] = m[r * 2 * d + d + c];
  *det = dt;
  free(m);
  return KDEO_OK;
}

/* ----------------------------------------------- Gaussian derivatives */

/* Probabilists' Hermite polynomial He_r(x) by the three-term recurrence
 * He_0 = 1, He_1 = x, He_{k+1} = x He_k - k He_{k-1}. */
double kdeo_hermite(int r, double x) {
  if (r == 0) return 1.0;
  double hm1 = 1.0, h = x;
  for (int k = 1; k < r; ++k) {
    double hp = x * h - (double)k * hm1;
    hm1 = h;
    h = hp;
  }
  return h;
}

/* K^(r)(x): r-th derivative of the standard normal density phi
 * (Sec. 4.4.1: K^6 and K^4 under Eqs. PLUGIN-Psi6Estimate, PLUGIN-Psi4Estimate).
 * d^r/dx^r phi(x) = (-1)^r He_r(x) phi(x). */
double kdeo_gauss_deriv(int r, double x) {
  double phi = exp(-0.5 * x * x) / sqrt(2.0 * KDEO_PI);
  double sgn = (r % 2) ? -1.0 : 1.0;
  return sgn * kdeo_hermite(r, x) * phi;
}

/* ------------------------------------------------------ psi functionals */

/* Sum over pairs (i, j), i in [i0, i1), j in [j0, j1), i < j, of
 * K^(r)((x_i - x_j) / g): the double sum of Eqs. PLUGIN-Psi6Estimate /
 * PLUGIN-Psi4Estimate restricted to a block of the pair triangle. */
double kdeo_psi_pair_sum_block(const double *x, long n, int r, double g, long i0, long i1,
                               long j0, long j1, int threads) {
  if (i0 < 0) i0 = 0;
  if (i1 > n) i1 = n;
  if (j1 > n) j1 = n;
  long rows = i1 > i0 ? i1 - i0 : 0;
  if (rows == 0) return 0.0;
  double *row = (double *)calloc((size_t)rows, sizeof(double));
  if (!row) return NAN;
  int nt = pick_threads(threads);
#pragma omp parallel for schedule(dynamic, 8) num_threads(nt)
  for (long ii = 0; ii < rows; ++ii) {
    long i = i0 + ii;
    nsum_t s = {0, 0};
    long jb = j0 > i + 1 ? j0 : i + 1;
    for (long j = jb; j < j1; ++j) nsum_add(&s, kdeo_gauss_deriv(r, (x[i] - x[j]) / g));
    row[ii] = nsum_get(&s);
  }
  nsum_t tot = {0, 0};
  for (long ii = 0; ii < rows; ++ii) nsum_add(&tot, row[ii]);
  free(row);
  return nsum_get(&tot);
}

/* Magnitude scale of the same block: sum of |K^(r)((x_i - x_j)/g)|.  Used only
 * to state the error of a signed sum relative to the size of its terms. */
double kdeo_psi_abs_pair_sum_block(const double *x, long n, int r, double g, long i0, long i1,
                                   long j0, long j1, int threads) {
  if (i0 < 0) i0 = 0;
  if (i1 > n) i1 = n;
  if (j1 > n) j1 = n;
  long rows = i1 > i0 ? i1 - i0 : 0;
  if (rows == 0) return 0.0;
  double *row = (double *)calloc((size_t)rows, sizeof(double));
  if (!row) return NAN;
  int nt = pick_threads(threads);
#pragma omp parallel for schedule(dynamic, 8) num_threads(nt)
  for (long ii = 0; ii < rows; ++ii) {
    long i = i0 + ii;
    nsum_t s = {0, 0};
    long jb = j0 > i + 1 ? j0 : i + 1;
    for (long j = jb; j < j1; ++j) nsum_add(&s, fabs(kdeo_gauss_deriv(r, (x[i] - x[j]) / g)));
    row[ii] = nsum_get(&s);
  }
  nsum_t tot = {0, 0};
  for (long ii = 0; ii < rows; ++ii) nsum_add(&tot, row[ii]);
  free(row);
  return nsum_get(&tot);
}

double kdeo_psi_pair_sum(const double *x, long n, int r, double g, int threads) {
  return kdeo_psi_pair_sum_block(x, n, r, g, 0, n, 0, n, threads);
}

/* psi_r(g) = n^-2 g^-(r+1) [ 2 sum_{i<j} K^(r)((x_i-x_j)/g) + n K^(r)(0) ]
 * (Eqs. PLUGIN-Psi6Estimate, PLUGIN-Psi4Estimate under reading R1). */
double kdeo_psi(const double *x, long n, int r, double g, int threads) {
  double s = kdeo_psi_pair_sum(x, n, r, g, threads);
  double dn = (double)n;
  return (2.0 * s + dn * kdeo_gauss_deriv(r, 0.0)) / (dn * dn * pow(g, (double)(r + 1)));
}

/* ---------------------------------------------------------- plug-in */

typedef struct {
  double var, sigma, psi8_ns, g1, psi6, g2, psi4, h;
  int status;
} kdeo_plugin_t;

/* Step 3, Eq. PLUGIN-Psi8Estimate. */
double kdeo_psi8_ns(double sigma) { return 105.0 / (32.0 * sqrt(KDEO_PI) * pow(sigma, 9.0)); }

/* Step 4, Eq. PLUGIN-g1 with mu_2(K) = 1. */
double kdeo_plugin_g1(double psi8, long n) {
  return pow(-2.0 * kdeo_gauss_deriv(6, 0.0) / (psi8 * (double)n), 1.0 / 9.0);
}

/* Step 6, Eq. PLUGIN-g2 with mu_2(K) = 1. */
double kdeo_plugin_g2(double psi6, long n) {
  return pow(-2.0 * kdeo_gauss_deriv(4, 0.0) / (psi6 * (double)n), 1.0 / 7.0);
}

/* Step 8, Eq. PLUGIN-Final_h with R(K) = 1/(2 sqrt(pi)), mu_2(K) = 1. */
double kdeo_plugin_h(double psi4, long n) {
  double rk = 1.0 / (2.0 * sqrt(KDEO_PI));
  return pow(rk / (psi4 * (double)n), 0.2);
}

/* The PLUGIN method, Sec. 4.4.1 steps 1-8, for univariate x[0..n). */
int kdeo_plugin(const double *x, long n, int threads, kdeo_plugin_t *out) {
  memset(out, 0, sizeof(*out));
  if (n < 2) return out->status = KDEO_EINVAL;
  double mean, var;
  kdeo_mean_cov(x, n, 1, &mean, &var);
  out->var = var;
  out->sigma = sqrt(var);
  if (!(out->sigma > 0.0)) return out->status = KDEO_EDEGENERATE;
  out->psi8_ns = kdeo_psi8_ns(out->sigma);
  out->g1 = kdeo_plugin_g1(out->psi8_ns, n);
  out->psi6 = kdeo_psi(x, n, 6, out->g1, threads);
  if (!(out->psi6 < 0.0)) return out->status = KDEO_EDEGENERATE;
  out->g2 = kdeo_plugin_g2(out->psi6, n);
  out->psi4 = kdeo_psi(x, n, 4, out->g2, threads);
  if (!(out->psi4 > 0.0)) return out->status = KDEO_EDEGENERATE;
  out->h = kdeo_plugin_h(out->psi4, n);
  return out->status = KDEO_OK;
}

/* ------------------------------------------------------------- LSCV_h */

/* Rule-of-thumb starting bandwidth, Eq. LSCV-h0 under reading R4. */
double kdeo_h0(long n, int d) {
  return pow(4.0 / ((double)(d + 2) * (double)n), 1.0 / (double)(d + 4));
}

/* The default grid over Z(h0) = [h0/4, 4 h0) (Eq. LSCV-Zh0): n_h log-spaced
 * points h_k = (h0/4) 16^(k/n_h), k = 0 .. n_h-1 (reading R6: Sec. 7.1 gives
 * the number of points, not their spacing).  With n_h a multiple of 8 there
 * are n_h/8 points per octave of 1/h^2. */
void kdeo_grid_default(long n, int d, int n_h, double *h) {
  const double z = kdeo_h0(n, d);
  for (int k = 0; k < n_h; ++k) h[k] = 0.25 * z * pow(16.0, (double)k / (double)n_h);
}

/* n_h log-spaced points from hmin to hmax inclusive (the search range of
 * Eq. LSCV-Zh0 sampled at a fixed number of points, Sec. 7.1). */
void kdeo_grid_log(double hmin, double hmax, int n_h, double *h) {
  if (n_h == 1) {
    h[0] = hmin;
    return;
  }
  double lr = log(hmax / hmin);
  for (int k = 0; k < n_h; ++k) h[k] = hmin * exp(lr * (double)k / (double)(n_h - 1));
}

/* Pair sums for the LSCV_h objective over the block i in [i0,i1), j in [j0,j1),
 * i<j, for every bandwidth h[k] (Sec. 4.4.2, Eqs. LSCV-gh, LSCV-Tx, LSCV-Kx,
 * LSCV-KKx):
 *   s_kk[k] = sum exp(-S(v)/(4 h^2)),   s_k[k] = sum exp(-S(v)/(2 h^2)),
 *   s_t[k]  = sum T(v/h) = sum [(K*K)(v/h) - 2 K(v/h)],
 * with v = X_i - X_j and S(v) = v^T Sigma^-1 v evaluated directly from the
 * inverse covariance (Eq. LSCV_MOD-Pv), both exponentials evaluated separately.
 * Any of the three outputs may be NULL. */
int kdeo_lscv_sums_block(const double *x, long n, int d, const double *h, int n_h, long i0,
                         long i1, long j0, long j1, double *s_kk, double *s_k, double *s_t,
                         int threads) {
  if (n < 2 || d < 1 || n_h < 1) return KDEO_EINVAL;
  double *mean = (double *)malloc(sizeof(double) * (size_t)d);
  double *cov = (double *)malloc(sizeof(double) * (size_t)(d * d));
  double *icov = (double *)malloc(sizeof(double) * (size_t)(d * d));
  if (!mean || !cov || !icov) return KDEO_ENOMEM;
  kdeo_mean_cov(x, n, d, mean, cov);
  double det;
  int st = kdeo_invert(cov, d, icov, &det);
  if (st != KDEO_OK || !(det > 0.0)) {
    free(mean), free(cov), free(icov);
    return KDEO_EDEGENERATE;
  }
  double ckk = pow(4.0 * KDEO_PI, -0.5 * d) / sqrt(det); /* Eq. LSCV-KKx */
  double ck = pow(2.0 * KDEO_PI, -0.5 * d) / sqrt(det);  /* Eq. LSCV-Kx  */
  if (i0 < 0) i0 = 0;
  if (i1 > n) i1 = n;
  if (j1 > n) j1 = n;
  long rows = i1 > i0 ? i1 - i0 : 0;
  double *rkk = (double *)calloc((size_t)rows * n_h + 1, sizeof(double));
  double *rk = (double *)calloc((size_t)rows * n_h + 1, sizeof(double));
  double *rt = (double *)calloc((size_t)rows * n_h + 1, sizeof(double));
  if (!rkk || !rk || !rt) return KDEO_ENOMEM;
  int nt = pick_threads(threads);
#pragma omp parallel num_threads(nt)
  {
    double *v = (double *)malloc(sizeof(double) * (size_t)d);
    nsum_t *akk = (nsum_t *)malloc(sizeof(nsum_t) * (size_t)n_h);
    nsum_t *ak = (nsum_t *)malloc(sizeof(nsum_t) * (size_t)n_h);
    nsum_t *at = (nsum_t *)malloc(sizeof(nsum_t) * (size_t)n_h);
#pragma omp for schedule(dynamic, 4)
    for (long ii = 0; ii < rows; ++ii) {
      long i = i0 + ii;
      for (int k = 0; k < n_h; ++k) akk[k].s = akk[k].c = ak[k].s = ak[k].c = at[k].s = at[k].c = 0;
      long jb = j0 > i + 1 ? j0 : i + 1;
      for (long j = jb; j < j1; ++j) {
        for (int a = 0; a < d; ++a) v[a] = x[(long)a * n + i] - x[(long)a * n + j];
        /* S(v) = sum_a (sum_c v_c m_ca) v_a  (Eq. yrpFinal with M = Sigma^-1) */
        double q = 0.0;
        for (int a = 0; a < d; ++a) {
          double part = 0.0;
          for (int c = 0; c < d; ++c) part += v[c] * icov[c * d + a];
          q += part * v[a];
        }
        for (int k = 0; k < n_h; ++k) {
          double hh = h[k] * h[k];
          double ekk = exp(-0.25 * q / hh);
          double ek = exp(-0.5 * q / hh);
          nsum_add(&akk[k], ekk);
          nsum_add(&ak[k], ek);
          nsum_add(&at[k], ckk * ekk - 2.0 * ck * ek);
        }
      }
      for (int k = 0; k < n_h; ++k) {
        rkk[ii * n_h + k] = nsum_get(&akk[k]);
        rk[ii * n_h + k] = nsum_get(&ak[k]);
        rt[ii * n_h + k] = nsum_get(&at[k]);
      }
    }
    free(v), free(akk), free(ak), free(at);
  }
  for (int k = 0; k < n_h; ++k) {
    nsum_t tkk = {0, 0}, tk = {0, 0}, tt = {0, 0};
    for (long ii = 0; ii < rows; ++ii) {
      nsum_add(&tkk, rkk[ii * n_h + k]);
      nsum_add(&tk, rk[ii * n_h + k]);
      nsum_add(&tt, rt[ii * n_h + k]);
    }
    if (s_kk) s_kk[k] = nsum_get(&tkk);
    if (s_k) s_k[k] = nsum_get(&tk);
    if (s_t) s_t[k] = nsum_get(&tt);
  }
  free(rkk), free(rk), free(rt);
  free(mean), free(cov), free(icov);
  return KDEO_OK;
}

/* The LSCV_h objective g(h) at every grid point (Eq. LSCV-gh with
 * R(K) per reading R3) and the first index attaining the minimum
 * (Eq. LSCV-finalH on the grid).  Optional outputs: s_kk, s_k (see above). */
int kdeo_lscv_h(const double *x, long n, int d, const double *h, int n_h, double *g,
                int *argmin, double *s_kk, double *s_k, int threads) {
  double *st = (double *)malloc(sizeof(double) * (size_t)n_h);
  double *mean = (double *)malloc(sizeof(double) * (size_t)d);
  double *cov = (double *)malloc(sizeof(double) * (size_t)(d * d));
  double *icov = (double *)malloc(sizeof(double) * (size_t)(d * d));
  if (!st || !mean || !cov || !icov) return KDEO_ENOMEM;
  int rc = kdeo_lscv_sums_block(x, n, d, h, n_h, 0, n, 0, n, s_kk, s_k, st, threads);
  if (rc != KDEO_OK) {
    free(st), free(mean), free(cov), free(icov);
    return rc;
  }
  kdeo_mean_cov(x, n, d, mean, cov);
  double det;
  kdeo_invert(cov, d, icov, &det);
  double rk = pow(4.0 * KDEO_PI, -0.5 * d) / sqrt(det); /* reading R3 */
  double dn = (double)n;
  int best = 0;
  for (int k = 0; k < n_h; ++k) {
    g[k] = pow(h[k], -(double)d) * (2.0 / (dn * dn) * st[k] + rk / dn);
    if (g[k] < g[best]) best = k;
  }
  if (argmin) *argmin = best;
  free(st), free(mean), free(cov), free(icov);
  return KDEO_OK;
}

/* Exact leave-one-out variant of the objective (the paper's Eq. LSCV-gh uses
 * n^-2 on the pair sum, reading R2; exact leave-one-out cross-validation uses
 * 1/(n(n-1)) on the K term):
 *   g_loo(h) = int fhat^2 - (2/n) sum_i fhat_{-i}(X_i)
 *            = n^-2 [n (K*K)_H(0) + 2 sum_{i<j} (K*K)_H(v)] - 4/(n(n-1)) sum_{i<j} K_H(v)
 * with H = h^2 Sigma, (K*K)_H(v) = h^-d (K*K)(v/h) and K_H(v) = h^-d K(v/h). */
int kdeo_lscv_h_loo(const double *x, long n, int d, const double *h, int n_h, double *g,
                    int threads) {
  double *skk = (double *)malloc(sizeof(double) * (size_t)n_h);
  double *sk = (double *)malloc(sizeof(double) * (size_t)n_h);
  double *mean = (double *)malloc(sizeof(double) * (size_t)d);
  double *cov = (double *)malloc(sizeof(double) * (size_t)(d * d));
  double *icov = (double *)malloc(sizeof(double) * (size_t)(d * d));
  if (!skk || !sk || !mean || !cov || !icov) return KDEO_ENOMEM;
  int rc = kdeo_lscv_sums_block(x, n, d, h, n_h, 0, n, 0, n, skk, sk, NULL, threads);
  if (rc == KDEO_OK) {
    kdeo_mean_cov(x, n, d, mean, cov);
    double det;
    kdeo_invert(cov, d, icov, &det);
    double ckk = pow(4.0 * KDEO_PI, -0.5 * d) / sqrt(det);
    double ck = pow(2.0 * KDEO_PI, -0.5 * d) / sqrt(det);
    double dn = (double)n;
    for (int k = 0; k < n_h; ++k) {
      double hd = pow(h[k], -(double)d);
      double intf2 = (dn * hd * ckk + 2.0 * hd * ckk * skk[k]) / (dn * dn);
      double loo = 4.0 / (dn * (dn - 1.0)) * hd * ck * sk[k];
      g[k] = intf2 - loo;
    }
  }
  free(skk), free(sk), free(mean), free(cov), free(icov);
  return rc;
}

/* Bracketing search for the minimum of g(h) (the golden-section alternative
 * to the dense grid named in Sec. 4.4.2 and Sec. 6.2, evaluated P points at a
 * time): in round t the bracket [a, b] holds P interior points log-spaced at
 * a (b/a)^(k/(P+1)), k = 1..P; the bracket becomes the neighbours of the
 * first-index minimum among them (a and b stand for k = 0 and k = P+1).
 * Stops when log(b/a) <= 2 rel_tol or after max_rounds.  Returns the best
 * evaluated h (and g there); loo selects the exact leave-one-out objective. */
int kdeo_lscv_search(const double *x, long n, int d, double a, double b, int P, double rel_tol,
                     int max_rounds, int loo, double *h_best, double *g_best, int *rounds,
                     int threads) {
  double *u = (double *)malloc(sizeof(double) * (size_t)(P + 2));
  double *gu = (double *)malloc(sizeof(double) * (size_t)P);
  if (!u || !gu) return KDEO_ENOMEM;
  double hb = 0.0, gb = INFINITY;
  int t = 0;
  for (; t < max_rounds && log(b / a) > 2.0 * rel_tol; ++t) {
    for (int k = 0; k <= P + 1; ++k) u[k] = a * exp(log(b / a) * (double)k / (double)(P + 1));
    int rc = loo ? kdeo_lscv_h_loo(x, n, d, u + 1, P, gu, threads)
                 : kdeo_lscv_h(x, n, d, u + 1, P, gu, NULL, NULL, NULL, threads);
    if (rc != KDEO_OK) {
      free(u), free(gu);
      return rc;
    }
    int km = 0;
    for (int k = 1; k < P; ++k)
      if (gu[k] < gu[km]) km = k;
    if (gu[km] < gb) {
      gb = gu[km];
      hb = u[km + 1];
    }
    a = u[km];
    b = u[km + 2];
  }
  *h_best = hb;
  *g_best = gb;
  if (rounds) *rounds = t;
  free(u), free(gu);
  return KDEO_OK;
}

/* ------------------------------------------- consumers of the bandwidth */

/* Density estimate fhat(q) = n^-1 sum_i K_H(q - X_i) at m points q (d x m,
 * one point per column) with K_H(u) = (2 pi)^(-d/2) |H|^(-1/2)
 * exp(-u^T H^-1 u / 2) (Sec. 4.2, Eqs. kde-def-H, K_H, gaussian). */
int kdeo_kde_eval(const double *x, long n, int d, const double *H, const double *q, long m,
                  double *f, int threads) {
  double *Hi = (double *)malloc(sizeof(double) * (size_t)(d * d));
  if (!Hi) return KDEO_ENOMEM;
  double det;
  if (kdeo_invert(H, d, Hi, &det) != KDEO_OK || !(det > 0.0)) {
    free(Hi);
    return KDEO_EDEGENERATE;
  }
  double c = pow(2.0 * KDEO_PI, -0.5 * d) / sqrt(det) / (double)n;
  int nt = pick_threads(threads);
#pragma omp parallel num_threads(nt)
  {
    double *v = (double *)malloc(sizeof(double) * (size_t)d);
#pragma omp for schedule(dynamic, 4)
    for (long k = 0; k < m; ++k) {
      nsum_t s = {0, 0};
      for (long i = 0; i < n; ++i) {
        for (int a = 0; a < d; ++a) v[a] = q[(long)a * m + k] - x[(long)a * n + i];
        double qf = 0.0;
        for (int a = 0; a < d; ++a)
          for (int b = 0; b < d; ++b) qf += v[a] * Hi[a * d + b] * v[b];
        nsum_add(&s, exp(-0.5 * qf));
      }
      f[k] = c * nsum_get(&s);
    }
    free(v);
  }
  free(Hi);
  return KDEO_OK;
}

/* Approximate Count and Sum of a numeric column over ranges [lo_k, hi_k]
 * from its univariate estimate with bandwidth h (Sec. 4.3, Eqs. count, sum):
 *   count = n int_lo^hi fhat(x) dx = sum_i [Phi(b_i) - Phi(a_i)],
 *   sum   = n int_lo^hi x fhat(x) dx = sum_i [x_i (Phi(b_i) - Phi(a_i)) + h (phi(a_i) - phi(b_i))],
 * with a_i = (lo - x_i)/h, b_i = (hi - x_i)/h: the integrals of each Gaussian
 * term done exactly (Phi by the complementary error function). */
int kdeo_aqp(const double *x, long n, double h, const double *lo, const double *hi, long m,
             double *count, double *sum, int threads) {
  int nt = pick_threads(threads);
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
  for (long k = 0; k < m; ++k) {
    nsum_t sc = {0, 0}, ss = {0, 0};
    for (long i = 0; i < n; ++i) {
      double a = (lo[k] - x[i]) / h, b = (hi[k] - x[i]) / h;
      double Pa = 0.5 * erfc(-a / sqrt(2.0)), Pb = 0.5 * erfc(-b / sqrt(2.0));
      double pa = exp(-0.5 * a * a) / sqrt(2.0 * KDEO_PI), pb = exp(-0.5 * b * b) / sqrt(2.0 * KDEO_PI);
      nsum_add(&sc, Pb - Pa);
      nsum_add(&ss, x[i] * (Pb - Pa) + h * (pa - pb));
    }
    count[k] = nsum_get(&sc);
    sum[k] = nsum_get(&ss);
  }
  return KDEO_OK;
}

/* ------------------------------------------------------------- LSCV_H */

/* The LSCV_H objective g(H) for one symmetric positive-definite bandwidth
 * matrix H (Sec. 4.4.3, Eqs. LSCV_MULTI-gh, LSCV_MULTI-Tx, LSCV_MULTI-Kx,
 * LSCV_MULTI-KKx, LSCV_MULTI-rk).  Written independently of kdeo_lscv_h:
 * the quadratic form uses H^-1 and the constants use |H|. */
int kdeo_lscv_H(const double *x, long n, int d, const double *H, double *g, int threads) {
  if (n < 2 || d < 1) return KDEO_EINVAL;
  double *Hi = (double *)malloc(sizeof(double) * (size_t)(d * d));
  if (!Hi) return KDEO_ENOMEM;
  double detH;
  if (kdeo_invert(H, d, Hi, &detH) != KDEO_OK || !(detH > 0.0)) {
    free(Hi);
    return KDEO_EDEGENERATE;
  }
  double ck = pow(2.0 * KDEO_PI, -0.5 * d) / sqrt(detH);
  double ckk = pow(4.0 * KDEO_PI, -0.5 * d) / sqrt(detH);
  double rk = pow(2.0, -(double)d) * pow(KDEO_PI, -0.5 * d) / sqrt(detH);
  double *row = (double *)calloc((size_t)n, sizeof(double));
  if (!row) return KDEO_ENOMEM;
  int nt = pick_threads(threads);
#pragma omp parallel num_threads(nt)
  {
    double *v = (double *)malloc(sizeof(double) * (size_t)d);
#pragma omp for schedule(dynamic, 8)
    for (long i = 0; i < n; ++i) {
      nsum_t s = {0, 0};
      for (long j = i + 1; j < n; ++j) {
        for (int a = 0; a < d; ++a) v[a] = x[(long)a * n + i] - x[(long)a * n + j];
        double q = 0.0;
        for (int a = 0; a < d; ++a)
          for (int c = 0; c < d; ++c) q += v[a] * Hi[a * d + c] * v[c];
        nsum_add(&s, ckk * exp(-0.25 * q) - 2.0 * ck * exp(-0.5 * q));
      }
      row[i] = nsum_get(&s);
    }
    free(v);
  }
  nsum_t tot = {0, 0};
  for (long i = 0; i < n; ++i) nsum_add(&tot, row[i]);
  double dn = (double)n;
  *g = 2.0 / (dn * dn) * nsum_get(&tot) + rk / dn;
  free(row), free(Hi);
  return KDEO_OK;
}
