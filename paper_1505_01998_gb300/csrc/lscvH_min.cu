// LSCV_H minimisation (Sec. 4.4.3): Nelder-Mead (the method the paper names)
// over the bandwidth matrix H, from the normal-scale start.
//
// Parametrisation: H = L L^T with L lower triangular, theta = the d(d+1)/2
// entries of L column by column (vech order) with the diagonal entries stored
// as logarithms, so every simplex point is a positive-definite H (the
// requirement stated in Sec. 4.4.3).  Start: H_start = (4/(d+2))^(2/(d+4))
// n^(-2/(d+4)) S (the normal-scale rule of Eq. LSCV-H-start, read as a matrix
// of squared bandwidths; reading R5).  Each iteration evaluates the
// reflection, expansion and both contractions of the worst point together in
// one batched g(H) pass (kde_lscv_H), then applies the standard Nelder-Mead
// rules (alpha 1, gamma 2, rho 1/2, sigma 1/2); a shrink evaluates its d(d+1)/2
// new points in one more pass.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "host.hpp"
#include "internal.cuh"

using namespace gbkde;

namespace {

int vdim(int d) { return d * (d + 1) / 2; }

// theta -> H (row-major d x d)
void theta_to_H(const std::vector<double>& th, int d, double* H) {
  double L[KDE_MAX_D][KDE_MAX_D] = {};
  int k = 0;
  for (int j = 0; j < d; ++j)
    for (int i = j; i < d; ++i) L[i][j] = (i == j) ? std::exp(th[k++]) : th[k++];
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < d; ++b) {
      double s = 0;
      for (int c = 0; c < d; ++c) s += L[a][c] * L[b][c];
      H[a * d + b] = s;
    }
}

bool H_to_theta(const double* H, int d, std::vector<double>* th) {
  double L[KDE_MAX_D][KDE_MAX_D] = {};
  for (int j = 0; j < d; ++j) {
    double s = H[j * d + j];
    for (int k = 0; k < j; ++k) s -= L[j][k] * L[j][k];
    if (!(s > 0)) return false;
    L[j][j] = std::sqrt(s);
    for (int i = j + 1; i < d; ++i) {
      double t = H[i * d + j];
      for (int k = 0; k < j; ++k) t -= L[i][k] * L[j][k];
      L[i][j] = t / L[j][j];
    }
  }
  th->clear();
  for (int j = 0; j < d; ++j)
    for (int i = j; i < d; ++i) th->push_back(i == j ? std::log(L[i][j]) : L[i][j]);
  return true;
}

}  // namespace

extern "C" int kde_lscv_H_minimize(const void* x_dev, int dtype, int64_t n, int d, const double* H_start,
                                   int max_iter, double ftol, const kde_opts* opts, void* ws,
                                   size_t ws_bytes, void* stream, double* H_out, double* g_out,
                                   int* evals_out) {
  if (!H_out || !g_out) return fail(KDE_EINVAL, "H_out or g_out is NULL");
  if (max_iter < 1 || !(ftol >= 0)) return fail(KDE_EINVAL, "max_iter / ftol");
  int rc = check_common(x_dev, dtype, n, d, ws);
  if (rc) return rc;
  const int p = vdim(d);
  std::vector<double> H0(d * d);
  if (H_start) {
    for (int k = 0; k < d * d; ++k) H0[k] = H_start[k];
  } else {
    // sample covariance from the prologue: logdet only is exported, so form S
    // through the batch machinery with H = I (whitening by I keeps x - mean)
    double S[KDE_MAX_D * KDE_MAX_D];
    rc = kde_sample_covariance(x_dev, dtype, n, d, ws, ws_bytes, stream, S);
    if (rc) return rc;
    const double c = std::pow(4.0 / (d + 2), 2.0 / (d + 4)) * std::pow((double)n, -2.0 / (d + 4));
    for (int k = 0; k < d * d; ++k) H0[k] = c * S[k];
  }
  std::vector<double> th0;
  if (!H_to_theta(H0.data(), d, &th0)) return fail(KDE_EDEGENERATE, "H_start not positive definite");
  // initial simplex: theta0 and p points moved by 0.15 in one coordinate
  // (15 % in a log-diagonal entry, 0.15 * the diagonal scale off the diagonal)
  std::vector<std::vector<double>> X(p + 1, th0);
  {
    int k = 0;
    for (int j = 0; j < d; ++j)
      for (int i = j; i < d; ++i, ++k) {
        const double scale = (i == j) ? 1.0 : std::exp(th0[0]);
        X[k + 1][k] += 0.15 * scale;
      }
  }
  cudaStream_t st = (cudaStream_t)stream;
  int evals = 0;
  // one batch plan per pass size (the first simplex, the four candidates of
  // an iteration, a shrink), built once and reused with new matrices: a pass
  // then costs its launches and one synchronisation, not a plan (geometry,
  // pinned staging) built and freed every time
  struct Plans {
    kde_batch_plan* by_m[3] = {nullptr, nullptr, nullptr};
    ~Plans() {
      for (kde_batch_plan* q : by_m) batch_free(q);
    }
  } plans;
  auto eval = [&](const std::vector<std::vector<double>>& pts, std::vector<double>* f) -> int {
    const int m = (int)pts.size();
    std::vector<double> Hs((size_t)m * d * d);
    for (int k = 0; k < m; ++k) theta_to_H(pts[k], d, Hs.data() + (size_t)k * d * d);
    f->assign(m, 0.0);
    evals += m;
    const int slot = (m == 4) ? 0 : (m == p ? 1 : 2);
    return lscv_H_eval(&plans.by_m[slot], true, x_dev, dtype, n, d, Hs.data(), m, opts, ws, ws_bytes, st,
                       f->data());
  };
  std::vector<double> F;
  rc = eval(X, &F);
  if (rc) return rc;
  int it = 0;
  for (; it < max_iter; ++it) {
    std::vector<int> idx(p + 1);
    for (int k = 0; k <= p; ++k) idx[k] = k;
    std::sort(idx.begin(), idx.end(), [&](int a, int b) { return F[a] < F[b]; });
    const int best = idx[0], worst = idx[p], second = idx[p - 1];
    if (std::fabs(F[worst] - F[best]) <= ftol * std::max(std::fabs(F[best]), 1e-300)) break;
    std::vector<double> c(p, 0.0);
    for (int k = 0; k <= p; ++k)
      if (k != worst)
        for (int q = 0; q < p; ++q) c[q] += X[k][q] / p;
    auto along = [&](double t) {
      std::vector<double> v(p);
      for (int q = 0; q < p; ++q) v[q] = c[q] + t * (X[worst][q] - c[q]);
      return v;
    };
    // reflection (t = -1), expansion (-2), outside (-1/2) and inside (+1/2) contraction
    std::vector<std::vector<double>> cand = {along(-1.0), along(-2.0), along(-0.5), along(0.5)};
    std::vector<double> fc;
    rc = eval(cand, &fc);
    if (rc) return rc;
    const double fr = fc[0], fe = fc[1], foc = fc[2], fic = fc[3];
    if (fr < F[best]) {
      if (fe < fr) {
        X[worst] = cand[1];
        F[worst] = fe;
      } else {
        X[worst] = cand[0];
        F[worst] = fr;
      }
    } else if (fr < F[second]) {
      X[worst] = cand[0];
      F[worst] = fr;
    } else if (fr < F[worst] && foc <= fr) {
      X[worst] = cand[2];
      F[worst] = foc;
    } else if (fr >= F[worst] && fic < F[worst]) {
      X[worst] = cand[3];
      F[worst] = fic;
    } else {  // shrink towards the best point
      std::vector<std::vector<double>> sh;
      std::vector<int> who;
      for (int k = 0; k <= p; ++k) {
        if (k == best) continue;
        std::vector<double> v(p);
        for (int q = 0; q < p; ++q) v[q] = X[best][q] + 0.5 * (X[k][q] - X[best][q]);
        sh.push_back(v);
        who.push_back(k);
      }
      std::vector<double> fs;
      rc = eval(sh, &fs);
      if (rc) return rc;
      for (size_t k = 0; k < who.size(); ++k) {
        X[who[k]] = sh[k];
        F[who[k]] = fs[k];
      }
    }
  }
  int bi = 0;
  for (int k = 1; k <= p; ++k)
    if (F[k] < F[bi]) bi = k;
  theta_to_H(X[bi], d, H_out);
  *g_out = F[bi];
  if (evals_out) *evals_out = evals;
  return KDE_OK;
}
