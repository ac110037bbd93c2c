// Autotuner of the LSCV pair-kernel geometry.
//
// Candidates: tile edge T in {32, 128}, bandwidths per thread B in {8, 16},
// resident CTAs per SM in {1, 2}, tiles per item K at 1x or 2x the default
// rule.  Each candidate is timed on the caller's samples with CUDA events
// around the pair kernel (best of two), either alone (latency: one dataset
// on an otherwise idle GPU) or replicated until the launch fills the GPU
// (throughput: the situation inside a batch or a serving step).  The winner
// is cached per (device, d, n_h bucket, n bucket); the geometry of every
// entry point then uses the cached values for options the caller leaves at 0.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "host.hpp"
#include "internal.cuh"

using namespace gbkde;

namespace gbkde {

namespace {

struct Tuned {
  int tile, bw, cps, kscale;
  double rate;
};

std::mutex g_mu;
std::map<std::tuple<std::string, int, int, int, int>, Tuned> g_cache;  // (device, mode, d, nhb, nb)

std::string device_key() {
  int dev = 0;
  cudaDeviceProp p;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "none";
  char buf[300];
  snprintf(buf, sizeof(buf), "%s/%d", p.name, p.multiProcessorCount);
  for (char* c = buf; *c; ++c)
    if (*c == ' ') *c = '_';
  return buf;
}

int bucket(int64_t v) {  // ceil(log2 v)
  int b = 0;
  while (((int64_t)1 << b) < v) ++b;
  return b;
}

// Exact number of pairs i < j < n in tiles [tb, te) of edge T.
double pairs_in_tiles(int64_t n, int T, int64_t tb, int64_t te) {
  double p = 0;
  for (int64_t t = tb; t < te; ++t) {
    int64_t l, q;
    tile_coords(t, l, q);
    const int64_t rv = std::max<int64_t>(0, std::min<int64_t>(T, n - q * T));
    const int64_t cv = std::max<int64_t>(0, std::min<int64_t>(T, n - l * T));
    p += (q == l) ? 0.5 * (double)cv * (double)(cv - 1) : (double)rv * (double)cv;
  }
  return p;
}

// The default tiles-per-item rule (make_geometry's item target).
int64_t base_k(const Geometry& g) {
  const int64_t target = g.item_target;
  return std::max<int64_t>(1, (g.tiles * g.G + target - 1) / target);
}

}  // namespace

// Cached tuning for the current device (mode 0 = latency, 1 = throughput).
bool tuned_lookup(int mode, int d, int n_h, int64_t n, kde_opts* out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_cache.empty()) return false;
  auto it = g_cache.find(std::make_tuple(device_key(), mode, d, bucket(std::max(n_h, 1)), bucket(n)));
  if (it == g_cache.end()) return false;
  memset(out, 0, sizeof(*out));
  out->tile = it->second.tile;
  out->bw_per_thread = it->second.bw;
  out->ctas_per_sm = it->second.cps;
  out->tiles_per_item = -it->second.kscale;  // negative: a multiple of the default rule
  return true;
}

}  // namespace gbkde

extern "C" {

int kde_autotune(const void* x_dev, int dtype, int64_t n, int d, int n_h, int mode, void* ws,
                 size_t ws_bytes, void* stream, kde_opts* best, double* best_evals_per_s) {
  if (!best) return fail(KDE_EINVAL, "best is NULL");
  if (mode != KDE_TUNE_LATENCY && mode != KDE_TUNE_THROUGHPUT) return fail(KDE_EINVAL, "mode %d", mode);
  if (n_h < 1 || n_h > KDE_MAX_NH) return fail(KDE_EINVAL, "n_h = %d", n_h);
  int rc = check_common(x_dev, dtype, n, d, ws);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int sms = device_sms();
  kde_grid gr{KDE_GRID_DEFAULT_Z, n_h, nullptr, 0, 0};
  std::vector<double> h;
  rc = build_grid(&gr, n, d, &h);
  if (rc) return rc;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(KDE_ECUDA, "events");
  Tuned win{0, 0, 0, 0, 0.0};
  for (int T : {32, 128})
    for (int B : {8, 16})
      for (int cps : {1, 2})
        for (int ks : {1, 2}) {
          kde_opts o{KDE_FP32_KAHAN, T, B, 0, cps};
          Geometry g;
          if (make_geometry(n, d, n_h, &o, sms, &g)) continue;
          o.tiles_per_item = (int)std::min<int64_t>(4096, base_k(g) * ks);
          // copies of the dataset so that one launch fills the GPU (throughput mode)
          int copies = 1;
          if (mode == KDE_TUNE_THROUGHPUT) {
            make_geometry(n, d, n_h, &o, sms, &g);
            copies = (int)std::min<int64_t>(64, std::max<int64_t>(1, (4 * (int64_t)g.ctas + g.items - 1) / g.items));
          }
          std::vector<kde_request> reqs(copies, kde_request{x_dev, dtype, d, n, KDE_METHOD_LSCV,
                                                            kde_grid{KDE_GRID_EXPLICIT, n_h, h.data(), 0, 0}});
          kde_batch_plan* p = nullptr;
          if (kde_batch_plan_create(reqs.data(), copies, &o, &p, nullptr) != KDE_OK) continue;
          double ms_best = 1e30;
          size_t need = 0;
          kde_batch_workspace_size(reqs.data(), copies, &o, &need);
          bool ok = need <= ws_bytes;
          for (int rep = 0; rep < 3 && ok; ++rep) {
            kde_set_kernel_events(e0, e1, nullptr, nullptr);
            ok = batch_run(p, ws, ws_bytes, st, false) == KDE_OK;
            kde_set_kernel_events(nullptr, nullptr, nullptr, nullptr);
            ok = ok && cudaStreamSynchronize(st) == cudaSuccess;
            float ms = 0;
            ok = ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
            if (ok && rep > 0) ms_best = std::min(ms_best, (double)ms);
          }
          batch_free(p);
          if (!ok || !(ms_best < 1e29)) continue;
          const double evals = (double)copies * pairs_in_tiles(n, T, 0, g.tiles) * n_h;
          const double rate = evals / (ms_best * 1e-3);
          if (rate > win.rate) win = Tuned{T, B, cps, ks, rate};
        }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (win.rate <= 0) return fail(KDE_ENOMEM, "autotune: no candidate fits the %zu-byte workspace", ws_bytes);
  {
    std::lock_guard<std::mutex> lk(g_mu);
    g_cache[std::make_tuple(device_key(), mode, d, bucket(n_h), bucket(n))] = win;
  }
  memset(best, 0, sizeof(*best));
  best->tile = win.tile;
  best->bw_per_thread = win.bw;
  best->ctas_per_sm = win.cps;
  Geometry g;
  kde_opts o{KDE_FP32_KAHAN, win.tile, win.bw, 0, win.cps};
  make_geometry(n, d, n_h, &o, sms, &g);
  best->tiles_per_item = (int)std::min<int64_t>(4096, base_k(g) * win.kscale);
  if (best_evals_per_s) *best_evals_per_s = win.rate;
  return KDE_OK;
}

int kde_autotune_clear(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_cache.clear();
  return KDE_OK;
}

int kde_autotune_save(const char* path) {
  if (!path) return fail(KDE_EINVAL, "path is NULL");
  std::lock_guard<std::mutex> lk(g_mu);
  FILE* f = fopen(path, "w");
  if (!f) return fail(KDE_EINVAL, "cannot write %s", path);
  fprintf(f, "# gbkde autotune cache: device mode d nh_bucket n_bucket tile bw ctas_per_sm k_scale evals_per_s\n");
  for (auto& kv : g_cache)
    fprintf(f, "%s %d %d %d %d %d %d %d %d %.6e\n", std::get<0>(kv.first).c_str(), std::get<1>(kv.first),
            std::get<2>(kv.first), std::get<3>(kv.first), std::get<4>(kv.first), kv.second.tile,
            kv.second.bw, kv.second.cps, kv.second.kscale, kv.second.rate);
  fclose(f);
  return KDE_OK;
}

int kde_autotune_load(const char* path) {
  if (!path) return fail(KDE_EINVAL, "path is NULL");
  FILE* f = fopen(path, "r");
  if (!f) return fail(KDE_EINVAL, "cannot read %s", path);
  char line[512], dev[300];
  int loaded = 0;
  std::lock_guard<std::mutex> lk(g_mu);
  while (fgets(line, sizeof(line), f)) {
    if (line[0] == '#') continue;
    int mode, d, nhb, nb, T, B, cps, ks;
    double rate;
    if (sscanf(line, "%299s %d %d %d %d %d %d %d %d %lf", dev, &mode, &d, &nhb, &nb, &T, &B, &cps, &ks, &rate) != 10)
      continue;
    if ((T != 32 && T != 128) || (B != 8 && B != 16) || cps < 1 || cps > 8 || ks < 1 || ks > 64) continue;
    g_cache[std::make_tuple(std::string(dev), mode, d, nhb, nb)] = Tuned{T, B, cps, ks, rate};
    ++loaded;
  }
  fclose(f);
  return loaded > 0 ? KDE_OK : fail(KDE_EINVAL, "no valid entries in %s", path);
}

}  // extern "C"
