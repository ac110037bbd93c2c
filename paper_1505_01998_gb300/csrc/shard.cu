// Host pieces of sharded LSCV_h: the prologue statistic a shard merge needs
// (log det S) and the FP64 finish of g(h) from summed exponential sums.
//
// A selection sharded over G GPUs gives every GPU all samples and a
// contiguous range of the pair-triangle tiles (kde_lscv_tile_sums); the 2 n_h
// FP64 sums are added across GPUs (one all-reduce), then kde_lscv_merge
// finishes g(h) and the argmin on any rank.
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

}  // extern "C"
