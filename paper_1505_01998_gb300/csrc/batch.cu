// Batched selection: many datasets of different sizes, methods and grids in
// one persistent launch per kernel variant, the whole sequence captured once
// in a CUDA graph and replayed.
//
// Every dataset keeps the geometry a single-dataset call would give it (tile,
// bandwidths per thread, tiles per item), and every item writes its own FP64
// partial row, so each result is bitwise the same alone and inside a batch.
// Datasets are not reordered: each launch walks all datasets through an
// item-offset table in which datasets outside its kernel variant own no items.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <tuple>
#include <vector>

#include "host.hpp"
#include "internal.cuh"

using namespace gbkde;

struct kde_batch_plan {
  int n_req = 0;
  bool has_opts = false;
  kde_opts opts{};
  int sms = 0;
  std::vector<Geometry> geo;
  std::vector<DsDev> desc;  // host image of the descriptor table (pointers filled at bind time)
  std::vector<std::vector<double>> grids;
  std::vector<int> lscv_group, psi_group;  // per request: group index or -1
  struct Group {
    int d, B, R, Rp;
    bool kahan;
    bool oct;  // octave-grid LSCV variant
    int64_t total;
    std::vector<int64_t> off;  // [n_req + 1]
  };
  std::vector<Group> lscv_groups, psi_groups;
  int n_h_pad_max = 0;
  int64_t lscv_rows_max = 0;
  // workspace layout (bytes from the base)
  size_t off_desc = 0, off_offs = 0, off_tables = 0, staged = 0, total = 0;
  std::vector<size_t> off_h, off_nc, off_y, off_xc, off_lpart, off_lsum, off_g, off_ppart, off_prep;
  int prep_parts_max = 1;
  // host staging and graph
  unsigned char* pin_in = nullptr;   // image of ws[0, staged)
  unsigned char* pin_out = nullptr;  // copy of the descriptor table after a run
  // one-shot plans (built, run once and freed inside one call) stage through
  // pageable memory: a pinned allocation and its release cost far more than
  // the copies of a few kilobytes they would speed up (kde_lscv_H at
  // n = 16,384, d = 2: 436 -> 123 us per call with one matrix, 597 -> 271 us
  // with four); plans that are kept and replayed stay pinned
  bool pageable = false;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t exec = nullptr;
  void* bound_ws = nullptr;
};

namespace gbkde {

static size_t align256(size_t v) { return (v + 255) / 256 * 256; }

// Builds geometry, groups and layout for the requests; `H` (optional,
// m x d x d) turns each request into an LSCV_H evaluation whitened by H.
int batch_plan_build(const kde_request* reqs, int n_req, const kde_opts* opts, const double* H,
                     kde_batch_plan* p) {
  if (!reqs || n_req < 1) return fail(KDE_EINVAL, "batch: no requests");
  int rc = check_opts(opts);
  if (rc) return rc;
  p->n_req = n_req;
  p->has_opts = opts != nullptr;
  if (opts) p->opts = *opts;
  p->sms = device_sms();
  p->geo.resize(n_req);
  p->desc.resize(n_req);
  p->grids.resize(n_req);
  p->lscv_group.assign(n_req, -1);
  p->psi_group.assign(n_req, -1);
  std::map<std::tuple<int, int, int, bool, bool>, int> lkey;
  std::map<std::tuple<int, bool>, int> pkey;
  for (int r = 0; r < n_req; ++r) {
    const kde_request& q = reqs[r];
    if (!q.x) return fail(KDE_EINVAL, "request %d: x is NULL", r);
    if (q.dtype != KDE_F32 && q.dtype != KDE_F64) return fail(KDE_EINVAL, "request %d: bad dtype", r);
    if (q.n < 2 || q.n > ((int64_t)1 << 31)) return fail(KDE_EINVAL, "request %d: n = %lld", r, (long long)q.n);
    if (q.d < 1 || q.d > KDE_MAX_D) return fail(KDE_EINVAL, "request %d: d = %d", r, q.d);
    if (!(q.methods & (KDE_METHOD_LSCV | KDE_METHOD_PLUGIN)) || (q.methods & ~3))
      return fail(KDE_EINVAL, "request %d: methods = %d", r, q.methods);
    if ((q.methods & KDE_METHOD_PLUGIN) && q.d != 1)
      return fail(KDE_EINVAL, "request %d: PLUGIN needs d = 1", r);
    int n_h = 0;
    if (q.methods & KDE_METHOD_LSCV) {
      rc = build_grid(&q.grid, q.n, q.d, &p->grids[r]);
      if (rc) return rc;
      n_h = (int)p->grids[r].size();
    }
    Geometry& g = p->geo[r];
    rc = make_geometry(q.n, q.d, n_h, opts, p->sms, &g);
    if (rc) return rc;
    if (q.methods & KDE_METHOD_LSCV) {
      apply_octave(&g, p->grids[r]);
      auto k = std::make_tuple(g.dk, g.B, g.R, g.kahan, g.oct_P > 0);
      auto it = lkey.find(k);
      if (it == lkey.end()) {
        it = lkey.emplace(k, (int)p->lscv_groups.size()).first;
        p->lscv_groups.push_back({g.dk, g.B, g.R, 0, g.kahan, g.oct_P > 0, 0, {}});
      }
      p->lscv_group[r] = it->second;
      p->n_h_pad_max = std::max(p->n_h_pad_max, g.n_h_pad);
      p->lscv_rows_max = std::max(p->lscv_rows_max, g.rows);
    }
    if (q.methods & KDE_METHOD_PLUGIN) {
      auto k = std::make_tuple(g.Rp, g.kahan);
      auto it = pkey.find(k);
      if (it == pkey.end()) {
        it = pkey.emplace(k, (int)p->psi_groups.size()).first;
        p->psi_groups.push_back({1, 0, 0, g.Rp, g.kahan, false, 0, {}});
      }
      p->psi_group[r] = it->second;
    }
  }
  for (size_t gi = 0; gi < p->lscv_groups.size(); ++gi) {
    auto& G = p->lscv_groups[gi];
    G.off.assign(n_req + 1, 0);
    for (int r = 0; r < n_req; ++r)
      G.off[r + 1] = G.off[r] + (p->lscv_group[r] == (int)gi ? p->geo[r].items : 0);
    G.total = G.off[n_req];
  }
  for (size_t gi = 0; gi < p->psi_groups.size(); ++gi) {
    auto& G = p->psi_groups[gi];
    G.off.assign(n_req + 1, 0);
    for (int r = 0; r < n_req; ++r)
      G.off[r + 1] = G.off[r] + (p->psi_group[r] == (int)gi ? p->geo[r].prows : 0);
    G.total = G.off[n_req];
  }
  // ---- layout: [descriptors][item offsets][h, -1/h^2 tables] = staged image; then data
  size_t o = 0;
  p->off_desc = o;
  o = align256(o + sizeof(DsDev) * n_req);
  p->off_offs = o;
  o = align256(o + sizeof(int64_t) * (n_req + 1) * (p->lscv_groups.size() + p->psi_groups.size()));
  p->off_tables = o;
  p->off_h.assign(n_req, 0);
  p->off_nc.assign(n_req, 0);
  for (int r = 0; r < n_req; ++r) {
    if (!(reqs[r].methods & KDE_METHOD_LSCV)) continue;
    p->off_h[r] = o;
    o = align256(o + sizeof(double) * p->grids[r].size());
    p->off_nc[r] = o;
    o = align256(o + sizeof(float) * p->geo[r].n_h_pad);
  }
  p->staged = o;
  p->off_y.assign(n_req, 0);
  p->off_xc.assign(n_req, 0);
  p->off_lpart.assign(n_req, 0);
  p->off_lsum.assign(n_req, 0);
  p->off_g.assign(n_req, 0);
  p->off_ppart.assign(n_req, 0);
  p->off_prep.assign(n_req, 0);
  for (int r = 0; r < n_req; ++r) {
    const Geometry& g = p->geo[r];
    const int m = reqs[r].methods;
    if (m & KDE_METHOD_LSCV) {
      p->off_y[r] = o;
      o = align256(o + sizeof(float) * g.dk * g.n_pad);
      p->off_lpart[r] = o;
      o = align256(o + sizeof(double) * g.rows * 2 * g.n_h_pad);
      p->off_lsum[r] = o;
      o = align256(o + sizeof(double) * 2 * g.n_h_pad);
      p->off_g[r] = o;
      o = align256(o + sizeof(double) * g.n_h);
    }
    if (m & KDE_METHOD_PLUGIN) {
      p->off_xc[r] = o;
      o = align256(o + sizeof(float) * g.n_pad);
      p->off_ppart[r] = o;
      o = align256(o + sizeof(double) * g.prows);
    }
  }
  p->prep_parts_max = 1;
  for (int r = 0; r < n_req; ++r) {
    p->off_prep[r] = o;
    o = align256(o + sizeof(double) * kPrepRecord * p->geo[r].prep_parts);
    p->prep_parts_max = std::max(p->prep_parts_max, p->geo[r].prep_parts);
  }
  p->total = o;
  // ---- host descriptor images (pointers are relative until bound to a workspace)
  for (int r = 0; r < n_req; ++r) {
    const Geometry& g = p->geo[r];
    DsDev s = make_desc(g, reqs[r].x, reqs[r].dtype, reqs[r].methods, nullptr);
    if (H) {
      s.given_H = 1;
      const int d = reqs[r].d;
      for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) s.cov[a * d + b] = H[(size_t)r * d * d + a * d + b];
    }
    p->desc[r] = s;
  }
  return KDE_OK;
}

static int batch_bind(kde_batch_plan* p, unsigned char* ws) {
  if (!p->pin_in) {
    if (p->pageable) {
      p->pin_in = new (std::nothrow) unsigned char[std::max<size_t>(p->staged, 256)];
      p->pin_out = new (std::nothrow) unsigned char[sizeof(DsDev) * p->n_req];
      if (!p->pin_in || !p->pin_out) return fail(KDE_ENOMEM, "batch: host staging");
    } else if (cudaMallocHost(&p->pin_in, std::max<size_t>(p->staged, 256)) != cudaSuccess ||
               cudaMallocHost(&p->pin_out, sizeof(DsDev) * p->n_req) != cudaSuccess) {
      return fail(KDE_ENOMEM, "batch: pinned host staging");
    }
  }
  unsigned char* img = p->pin_in;
  memset(img, 0, p->staged);
  DsDev* d = reinterpret_cast<DsDev*>(img + p->off_desc);
  for (int r = 0; r < p->n_req; ++r) {
    DsDev s = p->desc[r];
    const int m = s.methods;
    auto at = [&](size_t off) { return ws + off; };
    s.y = (m & KDE_METHOD_LSCV) ? reinterpret_cast<float*>(at(p->off_y[r])) : nullptr;
    s.xc = (m & KDE_METHOD_PLUGIN) ? reinterpret_cast<float*>(at(p->off_xc[r])) : nullptr;
    s.h = (m & KDE_METHOD_LSCV) ? reinterpret_cast<double*>(at(p->off_h[r])) : nullptr;
    s.nc = (m & KDE_METHOD_LSCV) ? reinterpret_cast<float*>(at(p->off_nc[r])) : nullptr;
    s.lscv_part = (m & KDE_METHOD_LSCV) ? reinterpret_cast<double*>(at(p->off_lpart[r])) : nullptr;
    s.lscv_sum = (m & KDE_METHOD_LSCV) ? reinterpret_cast<double*>(at(p->off_lsum[r])) : nullptr;
    s.g = (m & KDE_METHOD_LSCV) ? reinterpret_cast<double*>(at(p->off_g[r])) : nullptr;
    s.psi_part = (m & KDE_METHOD_PLUGIN) ? reinterpret_cast<double*>(at(p->off_ppart[r])) : nullptr;
    s.prep_part = reinterpret_cast<double*>(at(p->off_prep[r]));
    s.prep_count = 0;
    d[r] = s;
    if (m & KDE_METHOD_LSCV) {
      double* h = reinterpret_cast<double*>(img + p->off_h[r]);
      float* nc = reinterpret_cast<float*>(img + p->off_nc[r]);
      const auto& gr = p->grids[r];
      for (size_t k = 0; k < gr.size(); ++k) {
        h[k] = gr[k];
        nc[k] = (float)(-1.0 / (gr[k] * gr[k]));  // as the single-dataset setup kernel computes it
      }
      for (int k = (int)gr.size(); k < p->geo[r].n_h_pad; ++k) nc[k] = -1.0f;
    }
  }
  int64_t* offs = reinterpret_cast<int64_t*>(img + p->off_offs);
  size_t k = 0;
  for (auto& G : p->lscv_groups) {
    memcpy(offs + k * (p->n_req + 1), G.off.data(), sizeof(int64_t) * (p->n_req + 1));
    ++k;
  }
  for (auto& G : p->psi_groups) {
    memcpy(offs + k * (p->n_req + 1), G.off.data(), sizeof(int64_t) * (p->n_req + 1));
    ++k;
  }
  return KDE_OK;
}

static int batch_enqueue(kde_batch_plan* p, unsigned char* ws, cudaStream_t st) {
#define BK(call)                                            \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);     \
  } while (0)
  DsDev* ds = reinterpret_cast<DsDev*>(ws + p->off_desc);
  const int64_t* offs = reinterpret_cast<const int64_t*>(ws + p->off_offs);
  const int n = p->n_req;
  const int ctas = std::max(1, p->sms) * ((p->has_opts && p->opts.ctas_per_sm) ? p->opts.ctas_per_sm : 2);
  BK(cudaMemcpyAsync(ws, p->pin_in, p->staged, cudaMemcpyHostToDevice, st));
  BK(launch_prep(ds, n, nullptr, p->prep_parts_max, st));
  size_t k = 0;
  BK(mark_event(0, st));
  for (auto& G : p->lscv_groups) {
    Phase ph{ds, offs + k * (n + 1), nullptr, n, 0, G.total};
    const bool cps_given = p->has_opts && p->opts.ctas_per_sm;
    const int gctas = (G.oct && !cps_given) ? std::max(1, p->sms) * oct_ctas_per_sm(G.d) : ctas;
    BK(launch_lscv(ph, G.d, G.B, G.R, G.kahan, G.oct, (int)std::max<int64_t>(1, std::min<int64_t>(G.total, gctas)), st));
    ++k;
  }
  BK(mark_event(1, st));
  const size_t k_psi = k;
  const PsiCoef c6 = psi_coef(6), c4 = psi_coef(4);
  for (size_t i = 0; i < p->psi_groups.size(); ++i) {
    auto& G = p->psi_groups[i];
    Phase ph{ds, offs + (k_psi + i) * (n + 1), nullptr, n, 0, G.total};
    BK(launch_psi(ph, 6, G.Rp, G.kahan, c6, (int)std::max<int64_t>(1, std::min<int64_t>(G.total, ctas)), st));
  }
  if (!p->lscv_groups.empty()) {
    BK(launch_lscv_reduce(ds, n, nullptr, p->n_h_pad_max, p->lscv_rows_max, st));
  }
  if (!p->psi_groups.empty()) {
    BK(launch_psi_finish(ds, n, nullptr, 6, 6, st));
    for (size_t i = 0; i < p->psi_groups.size(); ++i) {
      auto& G = p->psi_groups[i];
      Phase ph{ds, offs + (k_psi + i) * (n + 1), nullptr, n, 0, G.total};
      BK(launch_psi(ph, 4, G.Rp, G.kahan, c4, (int)std::max<int64_t>(1, std::min<int64_t>(G.total, ctas)), st));
    }
    BK(launch_psi_finish(ds, n, nullptr, 4, 4, st));
  }
  BK(cudaMemcpyAsync(p->pin_out, ws + p->off_desc, sizeof(DsDev) * n, cudaMemcpyDeviceToHost, st));
  return KDE_OK;
#undef BK
}

int batch_prepare_kernels(kde_batch_plan* p) {
  for (auto& G : p->lscv_groups) {
    cudaError_t e = prepare_lscv(G.d, G.B, G.R, G.kahan, G.oct);
    if (e != cudaSuccess) return cuda_fail(e, "prepare_lscv");
  }
  return KDE_OK;
}

int batch_run(kde_batch_plan* p, void* ws, size_t ws_bytes, cudaStream_t st, bool use_graph) {
  if (!ws || reinterpret_cast<uintptr_t>(ws) % 256) return fail(KDE_EINVAL, "batch: workspace NULL or misaligned");
  if (ws_bytes < p->total) return fail(KDE_ENOMEM, "batch: workspace %zu < %zu bytes", ws_bytes, p->total);
  unsigned char* w = static_cast<unsigned char*>(ws);
  if (!use_graph) {
    int rc = batch_bind(p, w);
    if (rc) return rc;
    rc = batch_prepare_kernels(p);
    if (rc) return rc;
    return batch_enqueue(p, w, st);
  }
  if (!p->exec || p->bound_ws != ws) {
    if (p->exec) {
      cudaGraphExecDestroy(p->exec);
      p->exec = nullptr;
    }
    int rc = batch_bind(p, w);
    if (rc) return rc;
    rc = batch_prepare_kernels(p);
    if (rc) return rc;
    if (!p->cap && cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking) != cudaSuccess)
      return fail(KDE_ECUDA, "batch: capture stream");
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
    rc = batch_enqueue(p, w, p->cap);
    e = cudaStreamEndCapture(p->cap, &graph);
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&p->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    p->bound_ws = ws;
  }
  cudaError_t e = cudaGraphLaunch(p->exec, st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
  return KDE_OK;
}

void batch_collect(const kde_batch_plan* p, kde_result* outs) {
  const DsDev* d = reinterpret_cast<const DsDev*>(p->pin_out);
  for (int r = 0; r < p->n_req; ++r) outs[r] = d[r].res;
}

void batch_free(kde_batch_plan* p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->cap) cudaStreamDestroy(p->cap);
  if (p->pageable) {
    delete[] p->pin_in;
    delete[] p->pin_out;
  } else {
    if (p->pin_in) cudaFreeHost(p->pin_in);
    if (p->pin_out) cudaFreeHost(p->pin_out);
  }
  delete p;
}

// g(H) of m bandwidth matrices (H: m x d x d) as one batch of one-point
// grids at h = 1, through *plan: built on the first call or when m changes,
// and afterwards reused with only the descriptors' matrices replaced (the
// geometry and the staging do not depend on H, so the results are those of
// a freshly built plan).  keep: the plan will be reused (pinned staging);
// otherwise it stages through pageable memory.  Synchronises `st`.  The
// caller frees *plan with batch_free.
int lscv_H_eval(kde_batch_plan** plan, bool keep, const void* x_dev, int dtype, int64_t n, int d,
                const double* H, int m, const kde_opts* opts, void* ws, size_t ws_bytes, cudaStream_t st,
                double* g_host) {
  if (!plan || !H || !g_host) return fail(KDE_EINVAL, "H or g is NULL");
  if (m < 1 || m > KDE_MAX_NH) return fail(KDE_EINVAL, "m = %d outside [1, %d]", m, KDE_MAX_NH);
  int rc = check_common(x_dev, dtype, n, d, ws);
  if (rc) return rc;
  for (int k = 0; k < m; ++k)
    for (int a = 0; a < d; ++a)
      for (int b = 0; b < d; ++b) {
        const double v = H[(size_t)k * d * d + a * d + b];
        if (!std::isfinite(v) || v != H[(size_t)k * d * d + b * d + a])
          return fail(KDE_EINVAL, "H[%d] not finite and symmetric", k);
      }
  kde_batch_plan* p = *plan;
  if (p && (p->n_req != m || p->desc[0].x != x_dev || p->desc[0].n != n || p->desc[0].d != d ||
            p->desc[0].dtype != dtype)) {
    batch_free(p);
    p = *plan = nullptr;
  }
  if (!p) {
    std::vector<kde_request> reqs(m);
    const double one = 1.0;
    for (int k = 0; k < m; ++k)
      reqs[k] = kde_request{x_dev, dtype, d, n, KDE_METHOD_LSCV, kde_grid{KDE_GRID_EXPLICIT, 1, &one, 0, 0}};
    p = new (std::nothrow) kde_batch_plan();
    if (!p) return fail(KDE_ENOMEM, "plan");
    p->pageable = !keep;
    rc = batch_plan_build(reqs.data(), m, opts, H, p);
    if (rc) {
      batch_free(p);
      return rc;
    }
    *plan = p;
  } else {
    for (int k = 0; k < m; ++k)
      for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) p->desc[k].cov[a * d + b] = H[(size_t)k * d * d + a * d + b];
  }
  rc = batch_run(p, ws, ws_bytes, st, false);
  if (rc) return rc;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  std::vector<kde_result> res(m);
  batch_collect(p, res.data());
  for (int k = 0; k < m; ++k) {
    if (res[k].status != KDE_OK) return fail(res[k].status, "H[%d]: %s", k, kde_status_string(res[k].status));
    g_host[k] = res[k].g_min;  // one grid point h = 1: g(H) itself
  }
  return KDE_OK;
}

}  // namespace gbkde

extern "C" {

int kde_batch_plan_create(const kde_request* reqs, int n_req, const kde_opts* opts,
                          kde_batch_plan** plan, size_t* ws_bytes) {
  if (!plan) return fail(KDE_EINVAL, "plan is NULL");
  *plan = nullptr;
  kde_batch_plan* p = new (std::nothrow) kde_batch_plan();
  if (!p) return fail(KDE_ENOMEM, "batch plan");
  int rc = batch_plan_build(reqs, n_req, opts, nullptr, p);
  if (rc) {
    batch_free(p);
    return rc;
  }
  if (ws_bytes) *ws_bytes = p->total;
  *plan = p;
  return KDE_OK;
}

int kde_batch_run_async(kde_batch_plan* plan, void* ws, size_t ws_bytes, void* stream) {
  if (!plan) return fail(KDE_EINVAL, "plan is NULL");
  return batch_run(plan, ws, ws_bytes, (cudaStream_t)stream, true);
}

int kde_batch_results(const kde_batch_plan* plan, kde_result* outs) {
  if (!plan || !outs) return fail(KDE_EINVAL, "plan or outs is NULL");
  batch_collect(plan, outs);
  return KDE_OK;
}

int kde_batch_run(kde_batch_plan* plan, void* ws, size_t ws_bytes, void* stream, kde_result* outs) {
  int rc = kde_batch_run_async(plan, ws, ws_bytes, stream);
  if (rc) return rc;
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  if (outs) batch_collect(plan, outs);
  return KDE_OK;
}

int kde_batch_g(const kde_batch_plan* plan, const void* ws, int req, double* g_host) {
  if (!plan || !ws || !g_host || req < 0 || req >= plan->n_req) return fail(KDE_EINVAL, "kde_batch_g: bad arguments");
  if (!(plan->desc[req].methods & KDE_METHOD_LSCV)) return fail(KDE_EINVAL, "request %d has no LSCV grid", req);
  cudaError_t e = cudaMemcpy(g_host, static_cast<const unsigned char*>(ws) + plan->off_g[req],
                             sizeof(double) * plan->geo[req].n_h, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy");
  return KDE_OK;
}

int kde_batch_plan_destroy(kde_batch_plan* plan) {
  batch_free(plan);
  return KDE_OK;
}

int kde_batch_workspace_size(const kde_request* reqs, int n_req, const kde_opts* opts, size_t* bytes) {
  if (!bytes) return fail(KDE_EINVAL, "bytes is NULL");
  kde_batch_plan p;
  int rc = batch_plan_build(reqs, n_req, opts, nullptr, &p);
  if (rc) return rc;
  *bytes = p.total;
  return KDE_OK;
}

int kde_select_batch(const kde_request* reqs, int n_req, const kde_opts* opts, void* ws,
                     size_t ws_bytes, void* stream, kde_result* outs) {
  if (!outs) return fail(KDE_EINVAL, "outs is NULL");
  kde_batch_plan* p = nullptr;
  int rc = kde_batch_plan_create(reqs, n_req, opts, &p, nullptr);
  if (rc) return rc;
  p->pageable = true;  // built, run once and freed here
  rc = batch_run(p, ws, ws_bytes, (cudaStream_t)stream, false);
  if (!rc) {
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaStreamSynchronize");
  }
  if (!rc) batch_collect(p, outs);
  batch_free(p);
  return rc;
}

int kde_lscv_H_workspace_size(int64_t n, int d, int m, const kde_opts* opts, size_t* bytes) {
  if (!bytes || m < 1 || m > KDE_MAX_NH || n < 2 || d < 1 || d > KDE_MAX_D)
    return fail(KDE_EINVAL, "kde_lscv_H_workspace_size: bad arguments");
  std::vector<kde_request> reqs(m);
  const double one = 1.0;
  for (int k = 0; k < m; ++k)
    reqs[k] = kde_request{reinterpret_cast<const void*>(256), KDE_F32, d, n, KDE_METHOD_LSCV,
                          kde_grid{KDE_GRID_EXPLICIT, 1, &one, 0, 0}};
  kde_batch_plan p;
  int rc = batch_plan_build(reqs.data(), m, opts, nullptr, &p);
  if (rc) return rc;
  *bytes = p.total;
  return KDE_OK;
}

int kde_lscv_H(const void* x_dev, int dtype, int64_t n, int d, const double* H_host, int m,
               const kde_opts* opts, void* ws, size_t ws_bytes, void* stream, double* g_host) {
  kde_batch_plan* plan = nullptr;
  const int rc = lscv_H_eval(&plan, false, x_dev, dtype, n, d, H_host, m, opts, ws, ws_bytes,
                             (cudaStream_t)stream, g_host);
  batch_free(plan);
  return rc;
}

}  // extern "C"
