// Host pieces of sharded selections: the prologue statistic a shard merge
// needs (log det S), the FP64 finish of g(h) from summed exponential sums,
// the scalar steps of the PLUGIN chain from summed psi pair sums, and the
// item geometry that keeps shard boundaries on item boundaries.
//
// A selection sharded over G GPUs gives every GPU all samples and a
// contiguous range of the pair-triangle tiles (kde_lscv_tile_sums /
// kde_psi_tile_sums); the FP64 sums are added across GPUs (one all-reduce per
// all-pairs pass: 2 n_h values for LSCV_h, one value each for psi_6 and
// psi_4), then kde_lscv_merge / kde_plugin_merge finish on every rank.
#include <cmath>
#include <cstddef>
#include <vector>

#include "host.hpp"
#include "internal.cuh"

using namespace gbkde;

extern "C" {

int kde_lscv_logdet(const void* x_dev, int dtype, int64_t n, int d, void* ws, size_t ws_bytes,
                    void* stream, double* logdet_S) {
  if (!logdet_S) return fail(KDE_EINVAL, "logdet_S is NULL");
  int rc = check_common(x_dev, dtype, n, d, ws);
  if (rc) return rc;
  Geometry g;
  rc = make_geometry(n, d, 1, nullptr, device_sms(), &g);
  if (rc) return rc;
  if (ws_bytes < g.total) return fail(KDE_ENOMEM, "workspace %zu bytes < %zu needed", ws_bytes, g.total);
  cudaStream_t st = (cudaStream_t)stream;
  unsigned char* w = static_cast<unsigned char*>(ws);
  DsDev init = make_desc(g, x_dev, dtype, KDE_METHOD_LSCV, w);
  DsDev* ds = reinterpret_cast<DsDev*>(w + g.off_ds);
  int64_t* off = reinterpret_cast<int64_t*>(w + g.off_off);
  const double one = 1.0;
  const int64_t offs[4] = {0, 0, 0, 0};
  cudaError_t e = launch_setup(ds, init, &one, 1, off, offs, 4, st);
  if (e == cudaSuccess) e = launch_prep(ds, 1, nullptr, g.prep_parts, st);
  kde_result r;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&r, w + g.off_ds + offsetof(DsDev, res), sizeof(r), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "kde_lscv_logdet");
  if (r.status != KDE_OK) return fail(r.status, "prologue failed: %s", kde_status_string(r.status));
  *logdet_S = r.logdet_S;
  return KDE_OK;
}

int kde_sample_covariance(const void* x_dev, int dtype, int64_t n, int d, void* ws, size_t ws_bytes,
                          void* stream, double* cov) {
  if (!cov) return fail(KDE_EINVAL, "cov is NULL");
  double logdet = 0;
  int rc = kde_lscv_logdet(x_dev, dtype, n, d, ws, ws_bytes, stream, &logdet);
  if (rc) return rc;
  Geometry g;
  rc = make_geometry(n, d, 1, nullptr, device_sms(), &g);
  if (rc) return rc;
  double c[KDE_MAX_D * KDE_MAX_D];
  cudaError_t e = cudaMemcpy(c, static_cast<unsigned char*>(ws) + g.off_ds + offsetof(DsDev, cov),
                             sizeof(c), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy");
  for (int k = 0; k < d * d; ++k) cov[k] = c[k];
  return KDE_OK;
}

int kde_lscv_merge(int64_t n, int d, double logdet_S, const double* h, int n_h, const double* s1,
                   const double* s2, double* g_out, kde_result* out) {
  if (!h || !s1 || !s2 || !out || n < 2 || d < 1 || d > KDE_MAX_D || n_h < 1 || n_h > KDE_MAX_NH ||
      !std::isfinite(logdet_S))
    return fail(KDE_EINVAL, "kde_lscv_merge: bad arguments");
  const double pi = 3.14159265358979323846;
  const double A = std::pow(4.0 * pi, -0.5 * d) * std::exp(-0.5 * logdet_S);
  const double c2 = std::exp2(1.0 + 0.5 * d);
  const double dn = (double)n;
  std::vector<double> g(n_h);
  int best = 0;
  for (int k = 0; k < n_h; ++k) {
    g[k] = std::pow(h[k], -(double)d) * A * (2.0 / (dn * dn) * (s1[k] - c2 * s2[k]) + 1.0 / dn);
    if (g[k] < g[best]) best = k;
  }
  if (g_out)
    for (int k = 0; k < n_h; ++k) g_out[k] = g[k];
  kde_result r{};
  r.status = KDE_OK;
  r.method = KDE_METHOD_LSCV;
  r.argmin = best;
  r.n_h = n_h;
  r.d = d;
  r.h = h[best];
  r.g_min = g[best];
  r.logdet_S = logdet_S;
  r.flags = (best == 0 ? KDE_FLAG_MIN_AT_LOWER_EDGE : 0) | (best == n_h - 1 ? KDE_FLAG_MIN_AT_UPPER_EDGE : 0);
  *out = r;
  return KDE_OK;
}

int kde_item_tiles(int64_t n, int d, const double* h, int n_h, const kde_opts* opts, int* lscv_tile,
                   int* lscv_K, int* psi_tile, int* psi_K) {
  if (n < 2 || d < 1 || d > KDE_MAX_D || n_h < 0 || n_h > KDE_MAX_NH)
    return fail(KDE_EINVAL, "kde_item_tiles: bad sizes");
  int rc = check_opts(opts);
  if (rc) return rc;
  Geometry g;
  rc = make_geometry(n, d, n_h, opts, device_sms(), &g);
  if (rc) return rc;
  if (n_h > 0) {  // the grid decides between the octave and the direct kernel
    std::vector<double> grid(n_h);
    if (h) {
      for (int k = 0; k < n_h; ++k) grid[k] = h[k];
    } else {
      kde_default_grid(n, d, n_h, grid.data());
    }
    apply_octave(&g, grid);
  }
  if (lscv_tile) *lscv_tile = g.T;
  if (lscv_K) *lscv_K = g.K;
  if (psi_tile) *psi_tile = g.Tp;
  if (psi_K) *psi_K = g.Kp;
  return KDE_OK;
}

int kde_plugin_merge(int64_t n, int stage, double value, kde_result* res) {
  if (!res || n < 2 || !std::isfinite(value)) return fail(KDE_EINVAL, "kde_plugin_merge: bad arguments");
  const double pi = 3.14159265358979323846;
  const double inv_sqrt_2pi = 1.0 / std::sqrt(2.0 * pi);
  const double k6_0 = -15.0 * inv_sqrt_2pi;  // K^(6)(0)
  const double k4_0 = 3.0 * inv_sqrt_2pi;    // K^(4)(0)
  const double dn = (double)n;
  kde_result& r = *res;
  switch (stage) {
    case 8: {  // value = sigma: Eqs. PLUGIN-Psi8Estimate, PLUGIN-g1
      if (!(value > 0)) return fail(KDE_EDEGENERATE, "sigma = %g", value);
      r = kde_result{};
      r.status = KDE_OK;
      r.method = KDE_METHOD_PLUGIN;
      r.d = 1;
      r.sigma = value;
      r.psi8_ns = 105.0 / (32.0 * std::sqrt(pi) * std::pow(value, 9.0));
      r.g1 = std::pow(-2.0 * k6_0 / (r.psi8_ns * dn), 1.0 / 9.0);
      return KDE_OK;
    }
    case 6: {  // value = sum_{i<j} K^(6)((x_i - x_j)/g1): Eqs. PLUGIN-Psi6Estimate, PLUGIN-g2
      if (!(r.g1 > 0)) return fail(KDE_EINVAL, "kde_plugin_merge: stage 6 needs g1 (stage 8 first)");
      r.psi6 = (2.0 * value + dn * k6_0) / (dn * dn * std::pow(r.g1, 7.0));
      if (!(r.psi6 < 0.0)) {
        r.status = KDE_EDEGENERATE;
        return fail(KDE_EDEGENERATE, "psi_6 = %g is not negative", r.psi6);
      }
      r.g2 = std::pow(-2.0 * k4_0 / (r.psi6 * dn), 1.0 / 7.0);
      return KDE_OK;
    }
    case 4: {  // value = sum_{i<j} K^(4)((x_i - x_j)/g2): Eqs. PLUGIN-Psi4Estimate, PLUGIN-Final_h
      if (!(r.g2 > 0)) return fail(KDE_EINVAL, "kde_plugin_merge: stage 4 needs g2 (stage 6 first)");
      r.psi4 = (2.0 * value + dn * k4_0) / (dn * dn * std::pow(r.g2, 5.0));
      if (!(r.psi4 > 0.0)) {
        r.status = KDE_EDEGENERATE;
        return fail(KDE_EDEGENERATE, "psi_4 = %g is not positive", r.psi4);
      }
      const double rk = 1.0 / (2.0 * std::sqrt(pi));  // R(K)
      r.h_plugin = std::pow(rk / (r.psi4 * dn), 0.2);
      r.h = r.h_plugin;
      r.h_data = r.h_plugin;
      return KDE_OK;
    }
    default:
      return fail(KDE_EINVAL, "kde_plugin_merge: stage %d (8, 6 or 4)", stage);
  }
}

}  // extern "C"
