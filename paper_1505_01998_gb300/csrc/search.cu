// Bracketing search for the LSCV_h minimum: the alternative to the dense
// grid that Sec. 4.4.2 and Sec. 6.2 name (golden-section search), generalised
// to P = 8 interior points per round so that each round is one batched pass
// of the all-pairs kernel (8 bandwidths fill one chunk of a warp, costing the
// same as one).  Each round keeps the neighbours of the best interior point
// as the new bracket: the log-width shrinks by 2/9 per round.  Like any
// bracketing search it finds a local minimum when g(h) is not unimodal.
#include <cmath>
#include <vector>

#include "host.hpp"
#include "internal.cuh"

using namespace gbkde;

extern "C" int kde_lscv_search(const void* x_dev, int dtype, int64_t n, int d, double h_lo,
                               double h_hi, double rel_tol, int max_rounds, const kde_opts* opts,
                               void* ws, size_t ws_bytes, void* stream, kde_result* out,
                               int* rounds_out) {
  constexpr int P = 8;
  if (!out) return fail(KDE_EINVAL, "out is NULL");
  if (!(rel_tol > 0) || max_rounds < 1) return fail(KDE_EINVAL, "rel_tol / max_rounds");
  int rc = check_common(x_dev, dtype, n, d, ws);
  if (rc) return rc;
  double a = h_lo, b = h_hi;
  if (!(a > 0) || !(b > 0)) {  // Z(h0), Eq. LSCV-Zh0
    const double h0 = std::pow(4.0 / ((double)(d + 2) * (double)n), 1.0 / (double)(d + 4));
    a = h0 / 4.0;
    b = h0 * 4.0;
  }
  if (!(b > a) || !std::isfinite(b)) return fail(KDE_EINVAL, "bracket [%g, %g] invalid", a, b);
  const double a0 = a, b0 = b;
  double hb = 0.0, gb = INFINITY;
  kde_result best{};
  int t = 0;
  std::vector<double> u(P + 2), g(P);
  for (; t < max_rounds && std::log(b / a) > 2.0 * rel_tol; ++t) {
    for (int k = 0; k <= P + 1; ++k) u[k] = a * std::exp(std::log(b / a) * (double)k / (double)(P + 1));
    kde_grid grid{KDE_GRID_EXPLICIT, P, u.data() + 1, 0, 0};
    kde_result r;
    rc = kde_lscv(x_dev, dtype, n, d, &grid, opts, ws, ws_bytes, stream, g.data(), nullptr, &r);
    if (rc) return rc;
    const int km = r.argmin;  // first index attaining the minimum
    if (g[km] < gb) {
      gb = g[km];
      hb = u[km + 1];
      best = r;
    }
    a = u[km];
    b = u[km + 2];
  }
  best.h = hb;
  best.g_min = gb;
  best.h_data = (d == 1) ? hb * best.sigma : 0.0;
  best.argmin = 0;
  best.n_h = 0;
  // the bracket never left an end of the range: the minimum is at (or beyond) it
  best.flags = (a == a0 ? KDE_FLAG_MIN_AT_LOWER_EDGE : 0) | (b == b0 ? KDE_FLAG_MIN_AT_UPPER_EDGE : 0);
  *out = best;
  if (rounds_out) *rounds_out = t;
  return KDE_OK;
}
