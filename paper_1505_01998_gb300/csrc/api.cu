// Host side of the C ABI declared in include/gbkde.h: argument checks, work
// plans, workspace layout and the launch sequences of the single-dataset
// entry points.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "internal.cuh"
#include "host.hpp"

namespace gbkde {

thread_local bool t_dependent_launch = false;

namespace {
thread_local int t_err_status = KDE_OK;
thread_local char t_err_msg[512] = "";
thread_local cudaEvent_t t_ev[4] = {nullptr, nullptr, nullptr, nullptr};
}  // namespace

static cudaError_t mark(int k, cudaStream_t st) {
  return t_ev[k] ? cudaEventRecord(t_ev[k], st) : cudaSuccess;
}

cudaError_t mark_event(int k, cudaStream_t st) { return mark(k, st); }

int fail(int status, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(t_err_msg, sizeof(t_err_msg), fmt, ap);
  va_end(ap);
  t_err_status = status;
  return status;
}

int cuda_fail(cudaError_t e, const char* where) {
  return fail(KDE_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

int device_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return sms;
}

static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int check_opts(const kde_opts* o) {
  if (!o) return KDE_OK;
  if (o->precision != KDE_FP32_KAHAN && o->precision != KDE_FP32_PLAIN)
    return fail(KDE_EINVAL, "opts.precision %d invalid", o->precision);
  if (o->tile != 0 && o->tile != 32 && o->tile != 128)
    return fail(KDE_EINVAL, "opts.tile %d invalid (0, 32 or 128)", o->tile);
  if (o->bw_per_thread != 0 && o->bw_per_thread != 2 && o->bw_per_thread != 8 && o->bw_per_thread != 16)
    return fail(KDE_EINVAL, "opts.bw_per_thread %d invalid (0, 2, 8 or 16)", o->bw_per_thread);
  if (o->tiles_per_item < 0 || o->tiles_per_item > 4096)
    return fail(KDE_EINVAL, "opts.tiles_per_item %d invalid", o->tiles_per_item);
  if (o->ctas_per_sm < 0 || o->ctas_per_sm > 8)
    return fail(KDE_EINVAL, "opts.ctas_per_sm %d invalid", o->ctas_per_sm);
  if (o->cv != KDE_CV_PAPER && o->cv != KDE_CV_LOO) return fail(KDE_EINVAL, "opts.cv %d invalid", o->cv);
  return KDE_OK;
}

// Host check of the LSCV kernel's warp roles for every group size cg that
// the geometry can produce: each chunk is walked by exactly S warps whose
// column slices tile [0, T) in 16-byte steps, and every shared-memory slot the
// item-end combine reads (slice * cg + chunk) is a real warp.
int check_warp_roles(int T) {
  for (int cg = 1; cg <= kWarps; ++cg) {
    std::vector<int> cover(cg, 0);
    for (int w = 0; w < kWarps; ++w) {
      const WarpRole r = warp_role(w, cg);
      if (r.S < 1 || r.S * cg > kWarps || T % r.S || (T / r.S) % 4) return KDE_EINTERNAL;
      if (r.active) {
        if (r.slice * cg + r.chunk != w) return KDE_EINTERNAL;
        cover[r.chunk] += 1;
      }
    }
    for (int c = 0; c < cg; ++c)
      if (cover[c] != warp_role(0, cg).S) return KDE_EINTERNAL;
  }
  return KDE_OK;
}

// Geometry of one selection.  Deterministic in (n, d, n_h, opts, SM count).
int make_geometry(int64_t n, int d, int n_h, const kde_opts* o, int sms, Geometry* g,
                  double max_item_evals) {
  // Options left at 0 take the autotuner's cached choice for this device,
  // dimension and size bucket (throughput tuning first), else the fixed rules.
  kde_opts eff{};
  if (o) eff = *o;
  const int B_given = eff.bw_per_thread;
  int kscale = 1;
  kde_opts t;
  if (n_h > 0 && (!eff.tile || !eff.bw_per_thread || !eff.ctas_per_sm || !eff.tiles_per_item) &&
      (tuned_lookup(1, d, n_h, n, &t) || tuned_lookup(0, d, n_h, n, &t))) {
    if (!eff.tile) eff.tile = t.tile;
    if (!eff.bw_per_thread) eff.bw_per_thread = t.bw_per_thread;
    if (!eff.ctas_per_sm) eff.ctas_per_sm = t.ctas_per_sm;
    if (!eff.tiles_per_item) kscale = -t.tiles_per_item;
  }
  o = &eff;
  memset(g, 0, sizeof(*g));
  g->n = n;
  g->d = d;
  g->dk = d <= 4 ? d : (d + 3) / 4 * 4;
  g->n_h = n_h;
  g->n_pad = (int64_t)align_up((size_t)n, kPadTo);
  g->kahan = !(o && o->precision == KDE_FP32_PLAIN);
  g->cv_loo = (o && o->cv == KDE_CV_LOO) ? 1 : 0;
  const bool cps_given = o && o->ctas_per_sm;
  const int cps = cps_given ? o->ctas_per_sm : 2;
  g->ctas = std::max(1, sms) * cps;
  g->oct_P = 0;
  // LSCV
  g->T = (o && o->tile) ? o->tile : (n <= 2048 ? 32 : 128);
  if (g->dk > 4) g->T = 32;  // one row per lane keeps the d > 4 coordinates in registers
  g->R = g->T / 32;
  g->ctas_oct = g->ctas;
  // items: with the default CTA counts about 12 per SM (6 per CTA at 2 CTAs
  // per SM, 4 at 3), with an explicit count, or for the server's capped
  // items (a step spans many requests), about 4 per CTA
  const bool balanced = !cps_given && !(max_item_evals > 0);
  g->item_target = balanced ? 12 * (int64_t)std::max(1, sms) : 4 * (int64_t)g->ctas;
  // a one- or two-point grid (one g(H) of LSCV_H is a one-point grid) takes 2
  // bandwidths per thread unless the caller asked otherwise, whatever the
  // tuner chose for its size bucket: 8 would evaluate 6 padding bandwidths
  if (B_given)
    g->B = B_given;
  else if (n_h <= 2)
    g->B = 2;
  else
    g->B = o->bw_per_thread ? o->bw_per_thread : (n_h <= 64 ? 8 : 16);
  const int nh = std::max(n_h, 1);
  g->n_h_pad = (nh + g->B - 1) / g->B * g->B;
  g->n_chunks = g->n_h_pad / g->B;
  g->G = (g->n_chunks + kWarps - 1) / kWarps;
  if (check_warp_roles(g->T) != KDE_OK) return fail(KDE_EINTERNAL, "warp roles inconsistent for T = %d", g->T);
  g->tiles = tri_tiles(n, g->T);
  const int64_t kcap = (max_item_evals > 0 && !(o && o->tiles_per_item))
                           ? std::max<int64_t>(1, (int64_t)(max_item_evals / ((double)g->T * g->T *
                                                                            std::min(g->n_h_pad, kWarps * g->B))))
                           : 4096;
  if (o && o->tiles_per_item) {
    g->K = o->tiles_per_item;
  } else {
    // block items: item_target; warp items (equal tile counts, one per
    // warp) keep the partial rows, and so the reduction, short
    const int64_t target = lscv_warp_items(g->dk, g->B) ? (int64_t)g->ctas * kWarps : g->item_target;
    g->K = (int)std::min<int64_t>(4096, kscale * std::max<int64_t>(1, (g->tiles * g->G + target - 1) / target));
  }
  g->K = (int)std::min<int64_t>(g->K, kcap);
  g->K_oct = g->K;
  if (balanced && !(o && o->tiles_per_item) && !lscv_warp_items(g->dk, g->B)) {
    // Items are walked in grid-stride order by persistent CTAs, so the last
    // wave is full only when the item count is (nearly) a multiple of the
    // CTA count.  Tiles per item are chosen within a factor 2 of the rule
    // above for the best balance, separately for the direct kernel (2 CTAs
    // per SM) and the octave kernel, which takes 3 CTAs per SM (d <= 4)
    // when that balances at least as well as 2.
    const int64_t work = g->tiles;
    auto balance = [&](int64_t K, int64_t C) {
      const int64_t items = (work + K - 1) / K * g->G;
      return (double)items / ((double)C * (double)((items + C - 1) / C));
    };
    auto best_k = [&](int64_t C, double* eff) {
      const int64_t k0 = g->K;
      int64_t best = k0;
      double be = balance(k0, C);
      for (int64_t K = std::max<int64_t>(1, k0 / 2); K <= std::min<int64_t>(kcap, 2 * k0); ++K) {
        const double e = balance(K, C);
        if (e > be + 1e-12 || (e > be - 1e-12 && K > best)) {
          best = K;
          be = e;
        }
      }
      *eff = be;
      return (int)best;
    };
    const int64_t S = std::max(1, sms);
    double e2 = 0, e3 = 0;
    const int k2 = best_k(2 * S, &e2);
    g->K = k2;
    g->K_oct = k2;
    if (oct_ctas_per_sm(g->dk) == 3) {
      const int k3 = best_k(3 * S, &e3);
      if (e3 >= e2) {
        g->K_oct = k3;
        g->ctas_oct = (int)(3 * S);
      }
    }
  }
  g->rows = (g->tiles + g->K - 1) / g->K;
  g->rows_oct = (g->tiles + g->K_oct - 1) / g->K_oct;
  g->items = g->rows * g->G;
  // psi: tiles of 512 (two row groups per CTA) from n = 65,536, where the
  // per-tile work is the larger share of a 256-tile; about 4 items per CTA,
  // and with the default CTA count the tiles per item, between half that
  // rule's and the rule's, that fill the last wave best.  The server's item
  // cap applies after that choice and is above the rule's count at the
  // sizes it serves, so a served request has the items, and so the bits, of
  // the same single call.
  g->Tp = n >= 65536 ? 512 : (n >= 16384 ? 256 : 64);
  g->Rp = g->Tp / 32;
  g->ptiles = tri_tiles(n, g->Tp);
  {
    const int64_t target = 4 * (int64_t)g->ctas;
    g->Kp = (int)std::min<int64_t>(4096, std::max<int64_t>(1, (g->ptiles + target - 1) / target));
    if (!cps_given) {
      const int64_t C = g->ctas, k0 = g->Kp;
      auto balance = [&](int64_t K) {
        const int64_t items = (g->ptiles + K - 1) / K;
        return (double)items / ((double)C * (double)((items + C - 1) / C));
      };
      double be = balance(k0);
      for (int64_t K = std::max<int64_t>(1, k0 / 2); K <= k0; ++K) {
        const double e = balance(K);
        if (e > be + 1e-12 || (e > be - 1e-12 && K > g->Kp)) {
          g->Kp = (int)K;
          be = e;
        }
      }
    }
    if (max_item_evals > 0)
      g->Kp = (int)std::max<int64_t>(1, std::min<int64_t>(g->Kp, (int64_t)(max_item_evals / ((double)g->Tp * g->Tp))));
  }
  g->prows = (g->ptiles + g->Kp - 1) / g->Kp;
  // workspace layout
  size_t o0 = 0;
  g->off_ds = o0;
  o0 = align_up(o0 + sizeof(DsDev), 256);
  g->off_g = o0;  // right after the descriptor: the result and g[] come back in one short copy
  o0 = align_up(o0 + KDE_MAX_NH * sizeof(double), 256);
  g->off_off = o0;
  o0 = align_up(o0 + 8 * sizeof(int64_t), 256);
  g->off_h = o0;
  o0 = align_up(o0 + KDE_MAX_NH * sizeof(double), 256);
  g->off_nc = o0;
  o0 = align_up(o0 + KDE_MAX_NH * sizeof(float), 256);
  g->off_sum = o0;
  o0 = align_up(o0 + 2 * KDE_MAX_NH * sizeof(double), 256);
  g->off_x = o0;
  o0 = align_up(o0 + (size_t)d * n * sizeof(double), 256);
  g->off_y = o0;
  o0 = align_up(o0 + (size_t)g->dk * g->n_pad * sizeof(float), 256);
  g->off_xc = o0;
  o0 = align_up(o0 + (size_t)g->n_pad * sizeof(float), 256);
  g->off_lpart = o0;
  o0 = align_up(o0 + (n_h > 0 ? (size_t)std::max(g->rows, g->rows_oct) * 2 * g->n_h_pad * sizeof(double) : 0), 256);
  g->off_ppart = o0;
  o0 = align_up(o0 + (size_t)g->prows * sizeof(double), 256);
  g->prep_parts = prep_parts_for(n);
  g->off_prep = o0;
  o0 = align_up(o0 + (size_t)g->prep_parts * kPrepRecord * sizeof(double), 256);
  g->total = o0;
  return KDE_OK;
}

int check_common(const void* x, int dtype, int64_t n, int d, void* ws) {
  if (!x) return fail(KDE_EINVAL, "x is NULL");
  if (dtype != KDE_F32 && dtype != KDE_F64) return fail(KDE_EINVAL, "dtype %d invalid", dtype);
  if (n < 2) return fail(KDE_EINVAL, "n = %lld: need at least 2 samples", (long long)n);
  if (n > ((int64_t)1 << 31)) return fail(KDE_EINVAL, "n = %lld too large", (long long)n);
  if (d < 1 || d > KDE_MAX_D) return fail(KDE_EINVAL, "d = %d outside [1, %d]", d, KDE_MAX_D);
  if (!ws) return fail(KDE_EINVAL, "workspace is NULL");
  if (reinterpret_cast<uintptr_t>(ws) % 256) return fail(KDE_EINVAL, "workspace not 256-byte aligned");
  return KDE_OK;
}

int build_grid(const kde_grid* grid, int64_t n, int d, std::vector<double>* h) {
  if (!grid) return fail(KDE_EINVAL, "grid is NULL");
  if (grid->n_h < 1 || grid->n_h > KDE_MAX_NH)
    return fail(KDE_EINVAL, "grid n_h = %d outside [1, %d]", grid->n_h, KDE_MAX_NH);
  h->resize(grid->n_h);
  double lo = 0, hi = 0;
  switch (grid->kind) {
    case KDE_GRID_EXPLICIT:
      if (!grid->h) return fail(KDE_EINVAL, "explicit grid with NULL h");
      for (int k = 0; k < grid->n_h; ++k) (*h)[k] = grid->h[k];
      break;
    case KDE_GRID_DEFAULT_Z: {
      // h0 = (4 / ((d+2) n))^(1/(d+4)) (Eq. LSCV-h0, normal scale); n_h points
      // h_k = (h0/4) 16^(k/n_h) over Z = [h0/4, 4 h0): log-spaced, and with n_h
      // a multiple of 8, n_h/8 points per octave of 1/h^2
      const double h0 = std::pow(4.0 / ((double)(d + 2) * (double)n), 1.0 / (double)(d + 4));
      for (int k = 0; k < grid->n_h; ++k) (*h)[k] = 0.25 * h0 * std::pow(16.0, (double)k / (double)grid->n_h);
      break;
    }
    case KDE_GRID_LOG:
      lo = grid->h_min;
      hi = grid->h_max;
      if (!(lo > 0) || !(hi >= lo) || !std::isfinite(hi))
        return fail(KDE_EINVAL, "grid range [%g, %g] invalid", lo, hi);
      for (int k = 0; k < grid->n_h; ++k)
        (*h)[k] = grid->n_h == 1 ? lo
                                 : lo * std::exp(std::log(hi / lo) * (double)k / (double)(grid->n_h - 1));
      break;
    default:
      return fail(KDE_EINVAL, "grid kind %d invalid", grid->kind);
  }
  for (double v : *h)
    if (!(v > 0) || !std::isfinite(v)) return fail(KDE_EINVAL, "grid value %g invalid", v);
  return KDE_OK;
}

void apply_octave(Geometry* g, const std::vector<double>& h) {
  g->oct_P = 0;
  const int nh = (int)h.size();
  if (g->B != 16 || nh < 16 || nh % 16 != 0 || g->n_h_pad != nh) return;
  const int P = nh / 8;
  // the kernel forms octave arguments by exponent adds, exact while
  // |1/h^2| <= 2^40, and masks pairs with a finite squared distance that
  // zeroes every term while |1/h^2| >= 2^-40: outside, the direct kernel
  for (int k = 0; k < nh; ++k)
    if (!(h[k] >= 0x1p-20 && h[k] <= 0x1p20)) return;
  for (int k = P; k < nh; ++k) {
    // c_(k-P) = 2 c_k with c = 1/h^2, i.e. h_k^2 = 2 h_(k-P)^2
    const double r = (h[k] * h[k]) / (h[k - P] * h[k - P]);
    if (!(std::fabs(r - 2.0) <= 1e-12)) return;
  }
  g->oct_P = P;
  g->K = g->K_oct;  // the octave kernel's item size and rows (the workspace holds either)
  g->rows = g->rows_oct;
  g->items = g->rows * g->G;
}

// Descriptor for one selection on workspace `ws` laid out by `g`.
DsDev make_desc(const Geometry& g, const void* x, int dtype, int methods, unsigned char* ws) {
  DsDev s;
  memset(&s, 0, sizeof(s));
  s.x = x;
  s.n = g.n;
  s.d = g.d;
  s.dk = g.dk;
  s.cv_loo = g.cv_loo;
  s.dtype = dtype;
  s.n_pad = g.n_pad;
  s.methods = methods;
  s.y = reinterpret_cast<float*>(ws + g.off_y);
  s.xc = g.d == 1 ? reinterpret_cast<float*>(ws + g.off_xc) : nullptr;
  s.prep_parts = g.prep_parts;
  s.oct_P = g.oct_P;
  s.prep_part = reinterpret_cast<double*>(ws + g.off_prep);
  s.prep_count = 0;
  s.n_h = g.n_h;
  s.n_h_pad = g.n_h > 0 ? g.n_h_pad : 0;
  s.n_chunks = g.n_chunks;
  s.n_groups = g.G;
  s.lscv_tile = g.T;
  s.lscv_K = g.K;
  s.lscv_tiles = g.tiles;
  s.lscv_rows = g.rows;
  s.lscv_t0 = 0;
  s.h = reinterpret_cast<double*>(ws + g.off_h);
  s.nc = reinterpret_cast<float*>(ws + g.off_nc);
  s.lscv_part = reinterpret_cast<double*>(ws + g.off_lpart);
  s.lscv_sum = reinterpret_cast<double*>(ws + g.off_sum);
  s.g = reinterpret_cast<double*>(ws + g.off_g);
  s.psi_tile = g.Tp;
  s.psi_K = g.Kp;
  s.psi_tiles = g.ptiles;
  s.psi_rows = g.prows;
  s.psi_t0 = 0;
  s.psi_part = reinterpret_cast<double*>(ws + g.off_ppart);
  // the constant factors of A (Eqs. LSCV-Kx, LSCV-KKx) and of the pilot g1 (Eqs.
  // PLUGIN-Psi8Estimate, PLUGIN-g1) in FP64 on the host
  const double pi = 3.14159265358979323846;
  const double k6_0 = -15.0 / std::sqrt(2.0 * pi);
  s.c_A = std::pow(4.0 * pi, -0.5 * g.d);
  s.c_g1 = std::pow(-2.0 * k6_0 * 32.0 * std::sqrt(pi) / (105.0 * (double)g.n), 1.0 / 9.0);
  s.res.status = KDE_OK;
  return s;
}

// Monic polynomial p_r(y) with He_r(u) = kappa^(r/2) p_r(y), u^2 = kappa y,
// kappa = 2 ln 2 (see psi.cu), in Horner order.  He_r from its recurrence.
PsiCoef psi_coef(int r) {
  std::vector<double> hm1(r + 2, 0.0), h(r + 2, 0.0), hp(r + 2, 0.0);
  hm1[0] = 1.0;  // He_0
  h[1] = 1.0;    // He_1
  for (int k = 1; k < r; ++k) {
    std::fill(hp.begin(), hp.end(), 0.0);
    for (int j = 0; j <= r; ++j) {
      if (j + 1 <= r + 1) hp[j + 1] += h[j];
      hp[j] -= (double)k * hm1[j];
    }
    hm1 = h;
    h = hp;
  }
  const double kappa = 2.0 * std::log(2.0);
  const int M = r / 2;
  // b[m]: coefficient of y^m in the monic p_r(y) = He_r(sqrt(kappa y)) / kappa^M
  std::vector<double> b(M + 1);
  for (int m = 0; m <= M; ++m) b[m] = h[2 * m] * std::pow(kappa, (double)(m - M));
  // y = w - s with s = b[M-1] / M: q(w) = sum_k b[k] (w - s)^k, whose w^(M-1) term vanishes
  const double sh = b[M - 1] / (double)M;
  std::vector<double> dq(M + 1, 0.0);
  for (int k = 0; k <= M; ++k) {
    double binom = 1.0;  // C(k, m)
    for (int m = 0; m <= k; ++m) {
      dq[m] += b[k] * binom * std::pow(-sh, (double)(k - m));
      binom = binom * (double)(k - m) / (double)(m + 1);
    }
  }
  PsiCoef cf;
  memset(&cf, 0, sizeof(cf));
  for (int i = 0; i + 2 <= M; ++i) cf.c[i] = (float)dq[M - 2 - i];  // Horner: w^(M-2), ..., w^0
  cf.shift = (float)sh;
  cf.post = std::exp2(sh);
  return cf;
}

}  // namespace gbkde

using namespace gbkde;

#define CK(call)                                            \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);     \
  } while (0)

extern "C" {

const char* kde_version(void) { return "gbkde 0.1 (sm_103a)"; }

int kde_last_error(char* buf, size_t len) {
  if (buf && len) {
    strncpy(buf, t_err_msg, len - 1);
    buf[len - 1] = 0;
  }
  return t_err_status;
}

const char* kde_status_string(int s) {
  switch (s) {
    case KDE_OK: return "ok";
    case KDE_EINVAL: return "invalid argument";
    case KDE_ENOMEM: return "workspace or arena too small";
    case KDE_ECUDA: return "CUDA error";
    case KDE_EDEGENERATE: return "method undefined for these data";
    case KDE_EBUSY: return "server busy";
    case KDE_EAGAIN: return "not ready";
    case KDE_ETIMEDOUT: return "timed out";
    case KDE_ECANCELLED: return "cancelled";
    case KDE_ENOTFOUND: return "unknown ticket";
    case KDE_EINTERNAL: return "internal error";
    default: return "unknown status";
  }
}

int kde_tile_count(int64_t n, int tile, int64_t* tiles) {
  if (!tiles || n < 0 || tile <= 0) return fail(KDE_EINVAL, "kde_tile_count: bad arguments");
  *tiles = tri_tiles(n, tile);
  return KDE_OK;
}

int kde_tile_coords(int64_t bx, int64_t* l, int64_t* q) {
  if (!l || !q || bx < 0) return fail(KDE_EINVAL, "kde_tile_coords: bad arguments");
  tile_coords(bx, *l, *q);
  return KDE_OK;
}

int kde_default_grid(int64_t n, int d, int n_h, double* h_out) {
  if (!h_out || n < 2 || d < 1 || d > KDE_MAX_D) return fail(KDE_EINVAL, "kde_default_grid: bad arguments");
  kde_grid gr{KDE_GRID_DEFAULT_Z, n_h, nullptr, 0, 0};
  std::vector<double> h;
  int rc = build_grid(&gr, n, d, &h);
  if (rc) return rc;
  for (int k = 0; k < n_h; ++k) h_out[k] = h[k];
  return KDE_OK;
}

int kde_workspace_size(int64_t n, int d, int n_h, const kde_opts* opts, size_t* bytes) {
  if (!bytes) return fail(KDE_EINVAL, "bytes is NULL");
  if (n < 2 || d < 1 || d > KDE_MAX_D || n_h < 0 || n_h > KDE_MAX_NH)
    return fail(KDE_EINVAL, "kde_workspace_size: bad sizes");
  int rc = check_opts(opts);
  if (rc) return rc;
  Geometry g;
  { const int grc = make_geometry(n, d, n_h, opts, device_sms(), &g); if (grc) return grc; }
  *bytes = g.total;
  return KDE_OK;
}

int kde_ws_result_offset(size_t* result_offset, size_t* g_offset) {
  Geometry g;
  make_geometry(2, 1, 1, nullptr, 1, &g);
  if (result_offset) *result_offset = g.off_ds + offsetof(DsDev, res);
  if (g_offset) *g_offset = g.off_g;
  return KDE_OK;
}

int kde_psi_tile_edge(int64_t n, const kde_opts* opts, int* tile) {
  if (!tile || n < 2) return fail(KDE_EINVAL, "kde_psi_tile_edge: bad arguments");
  Geometry g;
  { const int grc = make_geometry(n, 1, 0, opts, device_sms(), &g); if (grc) return grc; }
  *tile = g.Tp;
  return KDE_OK;
}

// -------------------------------------------------------------- LSCV_h

// Partial tables that the last CTA of a single-selection pair kernel reduces
// itself: at most one chunk of rows per column strip (the reduction's chunk
// size, 64 rows) and at most 8 strips (n_h_pad <= 128), so its loads are a
// single L2 round trip per strip.  Larger tables go to the many-CTA
// reduction kernel: one CTA walking chunk after chunk measured slower than
// that kernel's launch (n = 1,000, 32 bandwidths: 19 against 15 us).
constexpr int64_t kFuseMaxRows = 64;
constexpr int kFuseMaxStrips = 8;

static int lscv_queue(const void* x_dev, int dtype, int64_t n, int d, const std::vector<double>& h,
                      const kde_opts* opts, void* ws, size_t ws_bytes, cudaStream_t st,
                      int64_t tile_begin, int64_t tile_end, Geometry* gout) {
  int rc = check_opts(opts);
  if (rc) return rc;
  Geometry g;
  { const int grc = make_geometry(n, d, (int)h.size(), opts, device_sms(), &g); if (grc) return grc; }
  apply_octave(&g, h);
  if (ws_bytes < g.total)
    return fail(KDE_ENOMEM, "workspace %zu bytes < %zu needed", ws_bytes, g.total);
  unsigned char* w = static_cast<unsigned char*>(ws);
  DsDev init = make_desc(g, x_dev, dtype, KDE_METHOD_LSCV, w);
  if (tile_begin >= 0) {
    init.lscv_t0 = tile_begin;
    init.lscv_tiles = tile_end;
    init.lscv_rows = (tile_end - tile_begin + g.K - 1) / g.K;
    g.rows = init.lscv_rows;
    g.items = g.rows * g.G;
  }
  DsDev* ds = reinterpret_cast<DsDev*>(w + g.off_ds);
  int64_t* off = reinterpret_cast<int64_t*>(w + g.off_off);
  const int64_t offs[4] = {0, g.items, 0, 0};
  DependentLaunchScope pdl;
  CK(launch_setup_prep(ds, init, h.data(), (int)h.size(), off, offs, 4, st));
  Phase ph{ds, off, nullptr, 1, 0, g.items};
  // small partial tables: the pair kernel's last CTA reduces and finishes
  // (saves two launches); large ones keep the many-CTA reduction
  const bool fuse = !lscv_warp_items(g.dk, g.B) && g.rows <= kFuseMaxRows &&
                    (2 * g.n_h_pad + 31) / 32 <= kFuseMaxStrips;
  ph.fuse = fuse ? 1 : 0;
  const int grid = (int)std::min<int64_t>(g.items, g.oct_P > 0 ? g.ctas_oct : g.ctas);
  CK(mark(0, st));
  CK(launch_lscv(ph, g.dk, g.B, g.R, g.kahan, g.oct_P > 0, std::max(grid, 1), st));
  CK(mark(1, st));
  if (!fuse) CK(launch_lscv_reduce(ds, 1, nullptr, g.n_h_pad, g.rows, st));
  if (gout) *gout = g;
  return KDE_OK;
}

int kde_lscv_async(const void* x_dev, int dtype, int64_t n, int d, const kde_grid* grid,
                   const kde_opts* opts, void* ws, size_t ws_bytes, void* stream) {
  int rc = check_common(x_dev, dtype, n, d, ws);
  if (rc) return rc;
  std::vector<double> h;
  rc = build_grid(grid, n, d, &h);
  if (rc) return rc;
  return lscv_queue(x_dev, dtype, n, d, h, opts, ws, ws_bytes, (cudaStream_t)stream, -1, -1, nullptr);
}

// Result (and g[], h[]) of a queued selection.  The result and g[] come
// back in one copy of the workspace span between them (tens of KB: one copy
// costs less than two); h[] is the grid the host built and uploaded.
static int fetch_result(const Geometry& g, void* ws, cudaStream_t st, double* g_host,
                        const std::vector<double>* h, double* h_host, kde_result* out) {
  unsigned char* w = static_cast<unsigned char*>(ws);
  kde_result r;
  const size_t off_r = g.off_ds + offsetof(DsDev, res);
  if (g_host && g.n_h > 0 && g.off_g > off_r) {
    thread_local std::vector<unsigned char> span;
    const size_t bytes = g.off_g + sizeof(double) * g.n_h - off_r;
    span.resize(bytes);
    CK(cudaMemcpyAsync(span.data(), w + off_r, bytes, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    memcpy(&r, span.data(), sizeof(r));
    memcpy(g_host, span.data() + (g.off_g - off_r), sizeof(double) * g.n_h);
  } else {
    CK(cudaMemcpyAsync(&r, w + off_r, sizeof(r), cudaMemcpyDeviceToHost, st));
    if (g_host && g.n_h > 0)
      CK(cudaMemcpyAsync(g_host, w + g.off_g, sizeof(double) * g.n_h, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  }
  if (h_host && g.n_h > 0) {
    if (h && (int)h->size() == g.n_h) {
      memcpy(h_host, h->data(), sizeof(double) * g.n_h);
    } else {
      CK(cudaMemcpy(h_host, w + g.off_h, sizeof(double) * g.n_h, cudaMemcpyDeviceToHost));
    }
  }
  if (out) *out = r;
  if (r.status != KDE_OK) return fail(r.status, "selection failed on the device: %s", kde_status_string(r.status));
  return KDE_OK;
}

int kde_lscv(const void* x_dev, int dtype, int64_t n, int d, const kde_grid* grid,
             const kde_opts* opts, void* ws, size_t ws_bytes, void* stream, double* g_host,
             double* h_host, kde_result* out) {
  if (!out) return fail(KDE_EINVAL, "out is NULL");
  int rc = check_common(x_dev, dtype, n, d, ws);
  if (rc) return rc;
  std::vector<double> h;
  rc = build_grid(grid, n, d, &h);
  if (rc) return rc;
  Geometry g;
  cudaStream_t st = (cudaStream_t)stream;
  rc = lscv_queue(x_dev, dtype, n, d, h, opts, ws, ws_bytes, st, -1, -1, &g);
  if (rc) return rc;
  return fetch_result(g, ws, st, g_host, &h, h_host, out);
}

int kde_lscv_host(const void* x_host, int dtype, int64_t n, int d, const kde_grid* grid,
                  const kde_opts* opts, void* ws, size_t ws_bytes, void* stream, double* g_host,
                  kde_result* out) {
  if (!out) return fail(KDE_EINVAL, "out is NULL");
  int rc = check_common(x_host, dtype, n, d, ws);
  if (rc) return rc;
  std::vector<double> h;
  rc = build_grid(grid, n, d, &h);
  if (rc) return rc;
  rc = check_opts(opts);
  if (rc) return rc;
  Geometry g;
  { const int grc = make_geometry(n, d, (int)h.size(), opts, device_sms(), &g); if (grc) return grc; }
  if (ws_bytes < g.total) return fail(KDE_ENOMEM, "workspace %zu bytes < %zu needed", ws_bytes, g.total);
  cudaStream_t st = (cudaStream_t)stream;
  void* xd = static_cast<unsigned char*>(ws) + g.off_x;
  const size_t bytes = (size_t)d * n * (dtype == KDE_F64 ? 8 : 4);
  CK(cudaMemcpyAsync(xd, x_host, bytes, cudaMemcpyHostToDevice, st));
  rc = lscv_queue(xd, dtype, n, d, h, opts, ws, ws_bytes, st, -1, -1, &g);
  if (rc) return rc;
  return fetch_result(g, ws, st, g_host, &h, nullptr, out);
}

int kde_lscv_tile_sums(const void* x_dev, int dtype, int64_t n, int d, const double* h_host,
                       int n_h, int64_t tile_begin, int64_t tile_end, const kde_opts* opts,
                       void* ws, size_t ws_bytes, void* stream, double* s1_host,
                       double* s2_host) {
  int rc = check_common(x_dev, dtype, n, d, ws);
  if (rc) return rc;
  if (!h_host || n_h < 1 || n_h > KDE_MAX_NH) return fail(KDE_EINVAL, "bad h / n_h");
  kde_grid gr{KDE_GRID_EXPLICIT, n_h, h_host, 0, 0};
  std::vector<double> h;
  rc = build_grid(&gr, n, d, &h);
  if (rc) return rc;
  rc = check_opts(opts);
  if (rc) return rc;
  Geometry g;
  { const int grc = make_geometry(n, d, n_h, opts, device_sms(), &g); if (grc) return grc; }
  if (tile_begin < 0 || tile_end < tile_begin || tile_end > g.tiles)
    return fail(KDE_EINVAL, "tile range [%lld, %lld) outside [0, %lld)", (long long)tile_begin,
                (long long)tile_end, (long long)g.tiles);
  if (tile_end == tile_begin) {
    for (int k = 0; k < n_h; ++k) {
      if (s1_host) s1_host[k] = 0;
      if (s2_host) s2_host[k] = 0;
    }
    return KDE_OK;
  }
  cudaStream_t st = (cudaStream_t)stream;
  rc = lscv_queue(x_dev, dtype, n, d, h, opts, ws, ws_bytes, st, tile_begin, tile_end, &g);
  if (rc) return rc;
  std::vector<double> sums(2 * g.n_h_pad);
  unsigned char* w = static_cast<unsigned char*>(ws);
  kde_result r;
  CK(cudaMemcpyAsync(sums.data(), w + g.off_sum, sizeof(double) * 2 * g.n_h_pad, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&r, w + g.off_ds + offsetof(DsDev, res), sizeof(r), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (r.status != KDE_OK) return fail(r.status, "tile sums failed on the device: %s", kde_status_string(r.status));
  for (int k = 0; k < n_h; ++k) {
    if (s1_host) s1_host[k] = sums[2 * k];
    if (s2_host) s2_host[k] = sums[2 * k + 1];
  }
  return KDE_OK;
}

// -------------------------------------------------------------- PLUGIN

static int plugin_queue(const void* x_dev, int dtype, int64_t n, const kde_opts* opts, void* ws,
                        size_t ws_bytes, cudaStream_t st, Geometry* gout) {
  int rc = check_opts(opts);
  if (rc) return rc;
  Geometry g;
  { const int grc = make_geometry(n, 1, 0, opts, device_sms(), &g); if (grc) return grc; }
  if (ws_bytes < g.total) return fail(KDE_ENOMEM, "workspace %zu bytes < %zu needed", ws_bytes, g.total);
  unsigned char* w = static_cast<unsigned char*>(ws);
  DsDev init = make_desc(g, x_dev, dtype, KDE_METHOD_PLUGIN, w);
  init.y = nullptr;  // plug-in needs only the centred samples
  DsDev* ds = reinterpret_cast<DsDev*>(w + g.off_ds);
  int64_t* off = reinterpret_cast<int64_t*>(w + g.off_off);
  const int64_t offs[4] = {0, 0, 0, g.prows};
  DependentLaunchScope pdl;
  CK(launch_setup_prep(ds, init, nullptr, 0, off, offs, 4, st));
  Phase ph{ds, off + 2, nullptr, 1, 0, g.prows};
  const int grid = std::max(1, (int)std::min<int64_t>(g.prows, g.ctas));
  // the last CTA of each psi launch reduces its item partials and advances
  // the chain (the partials are one value per item)
  ph.fuse = 6;
  CK(mark(2, st));
  CK(launch_psi(ph, 6, g.Rp, g.kahan, psi_coef(6), grid, st));
  CK(mark(3, st));
  ph.fuse = 4;
  CK(launch_psi(ph, 4, g.Rp, g.kahan, psi_coef(4), grid, st));
  if (gout) *gout = g;
  return KDE_OK;
}

int kde_plugin_async(const void* x_dev, int dtype, int64_t n, const kde_opts* opts, void* ws,
                     size_t ws_bytes, void* stream) {
  int rc = check_common(x_dev, dtype, n, 1, ws);
  if (rc) return rc;
  return plugin_queue(x_dev, dtype, n, opts, ws, ws_bytes, (cudaStream_t)stream, nullptr);
}

int kde_plugin(const void* x_dev, int dtype, int64_t n, const kde_opts* opts, void* ws,
               size_t ws_bytes, void* stream, kde_result* out) {
  if (!out) return fail(KDE_EINVAL, "out is NULL");
  int rc = check_common(x_dev, dtype, n, 1, ws);
  if (rc) return rc;
  Geometry g;
  cudaStream_t st = (cudaStream_t)stream;
  rc = plugin_queue(x_dev, dtype, n, opts, ws, ws_bytes, st, &g);
  if (rc) return rc;
  return fetch_result(g, ws, st, nullptr, nullptr, nullptr, out);
}

int kde_plugin_host(const void* x_host, int dtype, int64_t n, const kde_opts* opts, void* ws,
                    size_t ws_bytes, void* stream, kde_result* out) {
  if (!out) return fail(KDE_EINVAL, "out is NULL");
  int rc = check_common(x_host, dtype, n, 1, ws);
  if (rc) return rc;
  rc = check_opts(opts);
  if (rc) return rc;
  Geometry g;
  { const int grc = make_geometry(n, 1, 0, opts, device_sms(), &g); if (grc) return grc; }
  if (ws_bytes < g.total) return fail(KDE_ENOMEM, "workspace %zu bytes < %zu needed", ws_bytes, g.total);
  cudaStream_t st = (cudaStream_t)stream;
  void* xd = static_cast<unsigned char*>(ws) + g.off_x;
  CK(cudaMemcpyAsync(xd, x_host, (size_t)n * (dtype == KDE_F64 ? 8 : 4), cudaMemcpyHostToDevice, st));
  rc = plugin_queue(xd, dtype, n, opts, ws, ws_bytes, st, &g);
  if (rc) return rc;
  return fetch_result(g, ws, st, nullptr, nullptr, nullptr, out);
}

int kde_set_kernel_events(void* lscv_begin, void* lscv_end, void* psi_begin, void* psi_end) {
  t_ev[0] = (cudaEvent_t)lscv_begin;
  t_ev[1] = (cudaEvent_t)lscv_end;
  t_ev[2] = (cudaEvent_t)psi_begin;
  t_ev[3] = (cudaEvent_t)psi_end;
  return KDE_OK;
}

int kde_psi_tile_sums(const void* x_dev, int dtype, int64_t n, int r, double gpil,
                      int64_t tile_begin, int64_t tile_end, const kde_opts* opts, void* ws,
                      size_t ws_bytes, void* stream, double* sum_host) {
  int rc = check_common(x_dev, dtype, n, 1, ws);
  if (rc) return rc;
  if (r != 4 && r != 6 && r != 8) return fail(KDE_EINVAL, "r = %d: only 4, 6, 8", r);
  if (!(gpil > 0) || !std::isfinite(gpil)) return fail(KDE_EINVAL, "g = %g invalid", gpil);
  rc = check_opts(opts);
  if (rc) return rc;
  Geometry g;
  { const int grc = make_geometry(n, 1, 0, opts, device_sms(), &g); if (grc) return grc; }
  if (ws_bytes < g.total) return fail(KDE_ENOMEM, "workspace %zu bytes < %zu needed", ws_bytes, g.total);
  if (tile_begin < 0 || tile_end < tile_begin || tile_end > g.ptiles)
    return fail(KDE_EINVAL, "tile range outside [0, %lld)", (long long)g.ptiles);
  if (tile_end == tile_begin) {
    if (sum_host) *sum_host = 0;
    return KDE_OK;
  }
  cudaStream_t st = (cudaStream_t)stream;
  unsigned char* w = static_cast<unsigned char*>(ws);
  DsDev init = make_desc(g, x_dev, dtype, 0, w);
  init.y = nullptr;
  init.psi_t0 = tile_begin;
  init.psi_tiles = tile_end;
  init.psi_rows = (tile_end - tile_begin + g.Kp - 1) / g.Kp;
  init.psi_scale = (float)(std::sqrt(0.5 / std::log(2.0)) / gpil);
  DsDev* ds = reinterpret_cast<DsDev*>(w + g.off_ds);
  int64_t* off = reinterpret_cast<int64_t*>(w + g.off_off);
  const int64_t offs[4] = {0, 0, 0, init.psi_rows};
  CK(launch_setup_prep(ds, init, nullptr, 0, off, offs, 4, st));
  Phase ph{ds, off + 2, nullptr, 1, 0, init.psi_rows};
  const int grid = std::max(1, (int)std::min<int64_t>(init.psi_rows, g.ctas));
  CK(launch_psi(ph, r, g.Rp, g.kahan, psi_coef(r), grid, st));
  CK(launch_psi_finish(ds, 1, nullptr, 0, r, st));
  kde_result res;
  CK(cudaMemcpyAsync(&res, w + g.off_ds + offsetof(DsDev, res), sizeof(res), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (res.status != KDE_OK) return fail(res.status, "psi tile sums failed on the device: %s", kde_status_string(res.status));
  if (sum_host) *sum_host = res.g_min;
  return KDE_OK;
}

// ------------------------------------------------------------- probe

int kde_probe_alu(void* ws, size_t ws_bytes, void* stream, double* mufu, double* ffma,
                  double* ffma2, double* fmul2_fadd2, int* sm_count, double* sm_mhz) {
  const int sms = device_sms();
  if (sms <= 0) return fail(KDE_ECUDA, "no CUDA device");
  const int grid = sms;  // one 1024-thread CTA per SM (the probe's shared memory forces it)
  if (!ws || ws_bytes < sizeof(double) * 2 * grid) return fail(KDE_ENOMEM, "probe needs %zu bytes", sizeof(double) * 2 * grid);
  cudaStream_t st = (cudaStream_t)stream;
  double* dout = static_cast<double*>(ws);
  const int iters[4] = {1000, 4000, 4000, 4000};
  const double lanes_per_op[4] = {1.0, 1.0, 2.0, 2.0};  // modes 2, 3: packed FP32x2 instructions
  double rate[4] = {0, 0, 0, 0}, mhz = 0;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  std::vector<double> cyc(grid);
  for (int mode = 0; mode < 4; ++mode) {
    CK(launch_probe_mode(mode, dout, iters[mode] / 4, grid, st));  // warm-up
    CK(cudaEventRecord(e0, st));
    CK(launch_probe_mode(mode, dout, iters[mode], grid, st));
    CK(cudaEventRecord(e1, st));
    CK(cudaMemcpyAsync(cyc.data(), dout, sizeof(double) * grid, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    std::vector<double> s = cyc;
    std::sort(s.begin(), s.end());
    const double med = s[grid / 2];
    const double ops_per_sm = 1024.0 * iters[mode] * 32.0 * lanes_per_op[mode];
    rate[mode] = ops_per_sm / med;
    if (mode == 0) mhz = s[grid - 1] / (ms * 1e3);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (mufu) *mufu = rate[0];
  if (ffma) *ffma = rate[1];
  if (ffma2) *ffma2 = rate[2];
  if (fmul2_fadd2) *fmul2_fadd2 = rate[3];
  if (sm_count) *sm_count = sms;
  if (sm_mhz) *sm_mhz = mhz;
  return KDE_OK;
}

}  // extern "C"
