// Serving: a scheduler thread that admits bandwidth-selection requests of
// different sizes under an HBM budget, keeps their samples and partial sums
// resident, and advances all of them together in scheduling steps
// (continuous batching).
//
// * Admission: FIFO; a request is admitted when a slot is free and its
//   workspace region (the layout a single call would use) fits in the
//   caller's arena (first-fit allocator, 256-byte aligned, coalescing).
//   Its host samples are copied on a copy stream that overlaps compute.
// * Step: prologue for newly admitted requests; then, for the active
//   requests in service order (a request waiting longer than 32 times its
//   standalone kernel time, at least 0.5 s, first; then shortest remaining
//   work first), the next slice of each one's items in its current phase
//   (LSCV items, psi_6 items, psi_4 items) until the step's evaluation
//   budget is spent, one persistent
//   launch per kernel variant over a slot table; then the finishing kernels of
//   requests whose phase completed.  Up to two steps are in flight; the host
//   builds the next step while the device runs the current one.
// * A request's items depend only on the request and the server
//   configuration, and items only ever write their own rows: results are
//   bitwise the same alone or in the mix.  Items are capped at a twelfth of a
//   CTA's share of a step (finer than a single call's), so results equal the
//   single-request entry points' within the FP32 tolerance, not bitwise.
//   The variant launches of a step run on side streams, so their tails overlap.
// * Failure handling on the host: a step that misses its deadline fails its
//   requests (KDE_ETIMEDOUT) without touching the device; their regions are
//   released once the device work that references them has completed.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "host.hpp"
#include "internal.cuh"

using namespace gbkde;
using Clock = std::chrono::steady_clock;

namespace gbkde {

// First-fit allocator over [0, size) with coalescing.
class Arena {
 public:
  void init(size_t size) {
    free_.clear();
    if (size) free_[0] = size;
    used_ = peak_ = 0;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = (bytes + 255) / 256 * 256;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes, start = it->first + bytes;
        free_.erase(it);
        if (rest) free_[start] = rest;
        used_ += bytes;
        peak_ = std::max(peak_, used_);
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) / 256 * 256;
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t used() const { return used_; }
  size_t peak() const { return peak_; }

 private:
  std::map<size_t, size_t> free_;
  size_t used_ = 0, peak_ = 0;
};

}  // namespace gbkde

namespace {

enum Phase_ { P_QUEUED, P_LSCV, P_PSI6, P_PSI4, P_DONE };

struct Req {
  uint64_t ticket = 0;
  int methods = 0, dtype = 0, d = 1;
  int64_t n = 0;
  std::vector<unsigned char> samples;
  std::vector<double> grid;
  std::vector<float> nc;  // -1/h^2, padded to the chunk size with -1
  Geometry geo{};
  int slot = -1;
  size_t region = 0, region_bytes = 0;
  bool prepped = false;           // prologue issued
  bool copy_issued = false;
  cudaEvent_t copied = nullptr;   // samples resident
  int phase = P_QUEUED;
  int64_t cursor = 0;             // next item of the current phase
  int pending_finish = 0;         // finish kernel of the phase issued
  uint64_t finish_step = 0;       // sequence number of the step that holds it
  int in_flight = 0;              // launched steps that reference this request
  bool cancel = false, failed = false, finished = false;
  int fail_status = 0;
  kde_result result{};
  Clock::time_point t_submit, t_admit, t_done;
  double evals = 0;
  double work_total = 0;  // cost of all its phases (direct-kernel evaluations), set at admission
};

constexpr int kMaxSlots = 1024;
constexpr int kSideStreams = 4;  // concurrent variant launches within a step

struct Step {
  cudaEvent_t done = nullptr;
  Clock::time_point launched;
  std::vector<uint64_t> refs;      // requests referenced
  std::vector<uint64_t> complete;  // requests whose last kernel is in this step
  int buf = 0;
  uint64_t seq = 0;  // launch order (1, 2, ...)
  double evals = 0;
};

}  // namespace

struct kde_server {
  kde_serve_config cfg{};
  kde_opts opts{};
  bool has_opts = false;
  int sms = 0;
  unsigned char* arena = nullptr;
  size_t table_off = 0, params_off[2] = {0, 0}, params_bytes = 0, heap_off = 0;
  Arena heap;
  // Steps alternate between two stream sets (by parameter buffer), so the
  // pair kernels of a step start while the previous step's launches drain.
  cudaStream_t comp[2] = {}, copy = nullptr;
  cudaStream_t side[2][kSideStreams] = {};
  cudaEvent_t ev_fork[2] = {}, ev_join[2][kSideStreams] = {};
  cudaEvent_t ev_kdone[2] = {};  // a step's pair kernels (and all earlier steps') finished
  bool have_kdone = false;
  unsigned char* pin_params[2] = {nullptr, nullptr};
  unsigned char* pin_table[2] = {nullptr, nullptr};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread worker;
  bool stop = false;
  uint64_t next_ticket = 1;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, Req*> reqs;
  std::vector<uint64_t> slot_owner;
  std::deque<Step> inflight;
  int next_buf = 0;
  // stats
  uint64_t submitted = 0, completed = 0, failed = 0, cancelled = 0, rejected = 0;
  int64_t steps = 0;
  int queue_max = 0, active_max = 0;
  std::vector<double> lat_ms, wait_ms;
  double evals_done = 0;
  Clock::time_point t_first_submit, t_last_done;
  bool any_submit = false;
  int worker_error = 0;
};

namespace {

// Work per scheduling step, in evaluations of the direct LSCV kernel
// (default 1.3e11: about 14 ms of the all-pairs kernels on a GB300, long
// against the ~0.1 ms launch overhead and the item tails of a step, short
// against the latency of a large request).
double step_budget(const kde_server* s) {
  return s->cfg.quantum_evals > 0 ? s->cfg.quantum_evals : 1.3e11;
}

// Cost of one evaluation relative to one of the direct LSCV kernel, from the
// kernels' measured rates on a GB300 (direct LSCV 9.3e12 evaluations/s,
// octave-grid LSCV 17.1e12, psi_6 5.6e12, psi_4 6.9e12), so that a step
// takes about the same time whatever mix of kernels it runs.
double cost_of(const Req* r, int phase) {
  if (phase == P_LSCV) return r->geo.oct_P > 0 ? 0.55 : 1.0;
  return phase == P_PSI6 ? 1.65 : 1.35;
}

double eval_cost(const Req* r) { return cost_of(r, r->phase); }

int64_t items_of(const Req* r, int phase) {
  return phase == P_LSCV ? r->geo.items : r->geo.prows;
}

double evals_per_item(const Req* r, int phase) {
  if (phase == P_LSCV)
    return (double)r->geo.K * r->geo.T * r->geo.T * std::min(r->geo.n_h_pad, kWarps * r->geo.B);
  return (double)r->geo.Kp * r->geo.Tp * r->geo.Tp;
}

int64_t phase_items(const Req* r) { return items_of(r, r->phase); }
double item_evals(const Req* r) { return evals_per_item(r, r->phase); }

// Work a request still needs, in direct-kernel evaluations: the rest of its
// current phase and all of its later phases.
double work_left(const Req* r) {
  double w = 0.0;
  for (int ph = std::max(r->phase, (int)P_LSCV); ph <= P_PSI4; ++ph) {
    if (ph == P_LSCV ? !(r->methods & KDE_METHOD_LSCV) : !(r->methods & KDE_METHOD_PLUGIN)) continue;
    const double items = (double)items_of(r, ph) - (ph == r->phase ? (double)r->cursor : 0.0);
    w += items * evals_per_item(r, ph) * cost_of(r, ph);
  }
  return w;
}

// Order of service: shortest remaining work first, except that a request
// waiting longer than max(kAgeFloorS, kAgeFactor x its work at the kernels'
// rate) goes before all others (oldest first), so that a large request
// cannot be starved by a stream of smaller ones.
constexpr double kDirectEvalsPerS = 9.3e12;  // direct LSCV kernel on a GB300
constexpr double kAgeFactor = 32.0;
constexpr double kAgeFloorS = 0.5;

bool overdue(const Req* r, Clock::time_point now) {
  const double age = std::chrono::duration<double>(now - r->t_submit).count();
  return age > std::max(kAgeFloorS, kAgeFactor * r->work_total / kDirectEvalsPerS);
}

void finish_req(kde_server* s, Req* r, int status) {
  r->finished = true;
  r->t_done = Clock::now();
  if (status != KDE_OK) {
    r->result.status = status;
    if (status == KDE_ECANCELLED)
      s->cancelled++;
    else
      s->failed++;
  } else {
    s->completed++;
    s->lat_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
    s->wait_ms.push_back(std::chrono::duration<double, std::milli>(r->t_admit - r->t_submit).count());
    s->evals_done += r->evals;
    s->t_last_done = r->t_done;
  }
}

void release_req(kde_server* s, Req* r) {
  if (r->slot >= 0) {
    s->heap.release(r->region - s->heap_off, r->region_bytes);  // heap offsets are heap-relative
    s->slot_owner[r->slot] = 0;
    r->slot = -1;
  }
  if (r->copied) {
    cudaEventDestroy(r->copied);
    r->copied = nullptr;
  }
  r->samples.clear();
  r->samples.shrink_to_fit();
}

// Bytes of the step parameter block: ids lists + per-group (off, base) arrays.
size_t params_block_bytes(int slots) {
  const size_t groups = 64;  // LSCV variants (d x B x R x precision) + psi variants, bounded
  return (size_t)(4 + 2 * groups) * (slots + 1) * sizeof(int64_t) + 4 * slots * sizeof(int) + 4096;
}

// Issue admissions: returns requests admitted now.
void admit(kde_server* s) {
  while (!s->queue.empty()) {
    Req* r = s->reqs[s->queue.front()];
    if (r->cancel) {
      s->queue.pop_front();
      finish_req(s, r, KDE_ECANCELLED);
      release_req(s, r);
      continue;
    }
    int slot = -1;
    for (int k = 0; k < s->cfg.max_slots; ++k)
      if (!s->slot_owner[k]) {
        slot = k;
        break;
      }
    if (slot < 0) break;
    size_t off = 0;
    if (!s->heap.alloc(r->region_bytes, &off)) break;  // wait for memory to free up
    s->queue.pop_front();
    r->slot = slot;
    r->region = s->heap_off + off;
    s->slot_owner[slot] = r->ticket;
    r->t_admit = Clock::now();
    r->phase = (r->methods & KDE_METHOD_LSCV) ? P_LSCV : P_PSI6;
    r->cursor = 0;
    r->work_total = work_left(r);
    // samples -> region (copy stream, overlaps running steps)
    unsigned char* base = s->arena + r->region;
    cudaMemcpyAsync(base + r->geo.off_x, r->samples.data(), r->samples.size(), cudaMemcpyHostToDevice, s->copy);
    cudaEventCreateWithFlags(&r->copied, cudaEventDisableTiming);
    cudaEventRecord(r->copied, s->copy);
    r->copy_issued = true;
  }
}


// Build and launch one step.  Returns false if there was nothing to do.
bool launch_step(kde_server* s, int* err) {
  const int S = s->cfg.max_slots;
  const double budget = step_budget(s);
  const int buf = s->next_buf;
  unsigned char* pin = s->pin_params[buf];
  unsigned char* dparams = s->arena + s->params_off[buf];
  DsDev* table = reinterpret_cast<DsDev*>(s->arena + s->table_off);
  memset(pin, 0, s->params_bytes);
  // layout of the parameter block
  int* prep_ids = reinterpret_cast<int*>(pin);
  int* lfin_ids = prep_ids + S;
  int* p6_ids = lfin_ids + S;
  int* p4_ids = p6_ids + S;
  int64_t* arrays = reinterpret_cast<int64_t*>(pin + (size_t)4 * S * sizeof(int) + 256 - ((size_t)4 * S * sizeof(int)) % 256);
  int n_prep = 0, n_lfin = 0, n_p6 = 0, n_p4 = 0, prep_parts_max = 1;
  struct G {
    int kind, d, B, R, Rp, r;
    bool kahan, oct;
    std::vector<int64_t> take, base;
    int64_t total = 0;
  };
  std::vector<G> groups;
  auto group_of = [&](int kind, const Req* r) -> G& {
    const Geometry& g = r->geo;
    const int rr = kind == P_LSCV ? 0 : (kind == P_PSI6 ? 6 : 4);
    for (auto& x : groups)
      if (x.kind == kind && x.kahan == g.kahan &&
          (kind == P_LSCV ? (x.d == g.dk && x.B == g.B && x.R == g.R && x.oct == (g.oct_P > 0))
                          : (x.Rp == g.Rp && x.r == rr)))
        return x;
    groups.push_back({kind, g.dk, g.B, g.R, g.Rp, rr, g.kahan, kind == P_LSCV && g.oct_P > 0,
                      std::vector<int64_t>(S, 0), std::vector<int64_t>(S, 0), 0});
    return groups.back();
  };
  Step st;
  st.buf = buf;
  st.seq = s->steps + 1;
  double used = 0, step_evals = 0;  // work in direct-kernel evaluations; evaluations run
  std::vector<Req*> new_descs;
  std::vector<Req*> active;
  for (int k = 0; k < S; ++k)
    if (s->slot_owner[k]) active.push_back(s->reqs[s->slot_owner[k]]);
  // Budget policy: the step's budget goes down the service order (overdue
  // requests oldest first, then shortest remaining work first), each request
  // taking what it can use.  Short requests finish within a few steps even
  // while long ones run; the age bound keeps long ones from starving.
  {
    const Clock::time_point now = Clock::now();
    struct Key {
      bool late;
      double left;
      Req* r;
    };
    std::vector<Key> keys;
    keys.reserve(active.size());
    for (Req* r : active) keys.push_back({overdue(r, now), work_left(r), r});
    std::sort(keys.begin(), keys.end(), [](const Key& a, const Key& b) {
      if (a.late != b.late) return a.late;
      if (a.late) return a.r->t_submit < b.r->t_submit;
      if (a.left != b.left) return a.left < b.left;
      return a.r->t_submit < b.r->t_submit;
    });
    for (size_t k = 0; k < keys.size(); ++k) active[k] = keys[k].r;
  }
  const std::vector<Req*>& order = active;
  std::vector<char> seen(S, 0);
  for (size_t oi = 0; oi < order.size(); ++oi) {
    Req* r = order[oi];
    if (r->failed || r->phase == P_DONE) continue;
    if (r->cancel) continue;
    bool referenced = false;
    if (!r->prepped) {
      prep_ids[n_prep++] = r->slot;
      prep_parts_max = std::max(prep_parts_max, r->geo.prep_parts);
      new_descs.push_back(r);
      r->prepped = true;
      referenced = true;
    }
    if (r->pending_finish) {  // waits for its phase finish to land before the next phase
      if (referenced && !seen[r->slot]) {
        seen[r->slot] = 1;
        st.refs.push_back(r->ticket);
        r->in_flight++;
      }
      continue;
    }
    const int64_t total = phase_items(r);
    const int64_t left = total - r->cursor;
    const double cap = budget;
    if (left > 0 && (used < cap || st.refs.empty())) {
      const double per = item_evals(r), cost = per * eval_cost(r);
      int64_t take = (int64_t)std::max(1.0, std::floor((cap - used) / cost));
      take = std::min(take, left);
      G& g = group_of(r->phase, r);
      if (g.take[r->slot] == 0) g.base[r->slot] = r->cursor;  // a second pass extends the range
      g.take[r->slot] += take;
      g.total += take;
      r->cursor += take;
      used += take * cost;
      step_evals += take * per;
      r->evals += take * per;
      referenced = true;
      if (r->cursor == total) {
        if (r->phase == P_LSCV) lfin_ids[n_lfin++] = r->slot;
        if (r->phase == P_PSI6) p6_ids[n_p6++] = r->slot;
        if (r->phase == P_PSI4) p4_ids[n_p4++] = r->slot;
        r->pending_finish = 1;
        r->finish_step = st.seq;
        const bool last = (r->phase == P_PSI4) || (r->phase == P_LSCV && !(r->methods & KDE_METHOD_PLUGIN));
        if (last) st.complete.push_back(r->ticket);
      }
    }
    if (referenced && !seen[r->slot]) {
      seen[r->slot] = 1;
      st.refs.push_back(r->ticket);
      r->in_flight++;
    }
  }
  if (st.refs.empty()) return false;
  // ---- parameter arrays: per group (off[S+1], base[S])
  std::vector<std::pair<size_t, size_t>> goff;  // byte offsets of off/base within the block
  int64_t* a = arrays;
  for (auto& g : groups) {
    int64_t* off = a;
    a += S + 1;
    int64_t* base = a;
    a += S;
    off[0] = 0;
    for (int k = 0; k < S; ++k) {
      off[k + 1] = off[k] + g.take[k];
      base[k] = g.base[k];
    }
    goff.emplace_back((unsigned char*)off - pin, (unsigned char*)base - pin);
  }
  const size_t used_bytes = (unsigned char*)a - pin;
  if (used_bytes > s->params_bytes) {
    *err = fail(KDE_EINTERNAL, "serve: parameter block overflow");
    return false;
  }
  cudaStream_t cs = s->comp[buf];
  auto ck = [&](cudaError_t e, const char* w) {
    if (e != cudaSuccess && !*err) *err = cuda_fail(e, w);
  };
  // descriptors of newly admitted requests (the table copy in pin_table is the host image)
  for (Req* r : new_descs) {
    unsigned char* base = s->arena + r->region;
    DsDev dsc = make_desc(r->geo, base + r->geo.off_x, r->dtype, r->methods, base);
    if (!(r->methods & KDE_METHOD_LSCV)) dsc.y = nullptr;
    if (!(r->methods & KDE_METHOD_PLUGIN)) dsc.xc = nullptr;
    // h and -1/h^2 go into the region's tables through the parameter block
    memcpy(s->pin_table[buf] + (size_t)r->slot * sizeof(DsDev), &dsc, sizeof(DsDev));
  }
  // upload: descriptors of new requests, their grids, then the parameter block
  for (Req* r : new_descs) {
    ck(cudaStreamWaitEvent(cs, r->copied, 0), "cudaStreamWaitEvent");
    ck(cudaMemcpyAsync(table + r->slot, s->pin_table[buf] + (size_t)r->slot * sizeof(DsDev), sizeof(DsDev),
                       cudaMemcpyHostToDevice, cs), "desc upload");
    if (r->methods & KDE_METHOD_LSCV) {
      unsigned char* base = s->arena + r->region;
      // grid tables from the request's host vectors (pageable copies are
      // staged before the call returns)
      ck(cudaMemcpyAsync(base + r->geo.off_h, r->grid.data(), sizeof(double) * r->grid.size(),
                         cudaMemcpyHostToDevice, cs), "grid upload");
      ck(cudaMemcpyAsync(base + r->geo.off_nc, r->nc.data(), sizeof(float) * r->nc.size(),
                         cudaMemcpyHostToDevice, cs), "nc upload");
    }
  }
  ck(cudaMemcpyAsync(dparams, pin, used_bytes, cudaMemcpyHostToDevice, cs), "params upload");
  const int* d_prep = reinterpret_cast<const int*>(dparams);
  const int* d_lfin = d_prep + S;
  const int* d_p6 = d_lfin + S;
  const int* d_p4 = d_p6 + S;
  ck(launch_prep(table, n_prep, d_prep, prep_parts_max, cs), "prep");
  const int ctas = std::max(1, s->sms) * ((s->has_opts && s->opts.ctas_per_sm) ? s->opts.ctas_per_sm : 2);
  const PsiCoef c6 = psi_coef(6), c4 = psi_coef(4);
  // One persistent launch per kernel variant, forked over side streams so
  // that the tail of one launch overlaps the work of the others; joined back
  // before the finishing kernels.  Nothing orders these launches after the
  // previous step's: their items are other tile ranges with their own
  // partial rows, and requests whose phase finished there have no items here.
  // A request's later items (any step) need its prologue, which ran in the
  // step that admitted it: every step's fork follows the previous step's fork
  // (the previous step's uploads and prologues), not its pair kernels.
  if (s->have_kdone) ck(cudaStreamWaitEvent(cs, s->ev_fork[buf ^ 1], 0), "previous fork wait");
  ck(cudaEventRecord(s->ev_fork[buf], cs), "fork");
  bool forked[kSideStreams] = {};
  for (size_t i = 0; i < groups.size(); ++i) {
    const G& g = groups[i];
    if (!g.total) continue;
    const int k = (int)(i % kSideStreams);
    cudaStream_t ss = s->side[buf][k];
    if (!forked[k]) ck(cudaStreamWaitEvent(ss, s->ev_fork[buf], 0), "fork wait");
    forked[k] = true;
    Phase ph{table, reinterpret_cast<const int64_t*>(dparams + goff[i].first),
             reinterpret_cast<const int64_t*>(dparams + goff[i].second), S, 0, g.total};
    const bool cps_given = s->has_opts && s->opts.ctas_per_sm;
    const int gctas = (g.kind == P_LSCV && g.oct && !cps_given) ? std::max(1, s->sms) * oct_ctas_per_sm(g.d) : ctas;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(g.total, gctas));
    if (g.kind == P_LSCV)
      ck(launch_lscv(ph, g.d, g.B, g.R, g.kahan, g.oct, grid, ss), "lscv");
    else
      ck(launch_psi(ph, g.r, g.Rp, g.kahan, g.r == 6 ? c6 : c4, grid, ss), "psi");
  }
  for (int k = 0; k < kSideStreams; ++k)
    if (forked[k]) {
      ck(cudaEventRecord(s->ev_join[buf][k], s->side[buf][k]), "join");
      ck(cudaStreamWaitEvent(cs, s->ev_join[buf][k], 0), "join wait");
    }
  // The finishing kernels reduce every item of a request, some launched by
  // earlier steps: wait for the previous step's pair kernels (whose own
  // marker covers the steps before it).
  if (s->have_kdone) ck(cudaStreamWaitEvent(cs, s->ev_kdone[buf ^ 1], 0), "previous step wait");
  ck(cudaEventRecord(s->ev_kdone[buf], cs), "kernels done");
  s->have_kdone = true;
  int nh_max = 0;
  int64_t rows_max = 0;
  for (int k = 0; k < n_lfin; ++k) {
    const Geometry& gk = s->reqs[s->slot_owner[lfin_ids[k]]]->geo;
    nh_max = std::max(nh_max, gk.n_h_pad);
    rows_max = std::max(rows_max, gk.rows);
  }
  ck(launch_lscv_reduce(table, n_lfin, d_lfin, nh_max, rows_max, cs), "lscv reduce");
  ck(launch_psi_finish(table, n_p6, d_p6, 6, 6, cs), "psi6 finish");
  ck(launch_psi_finish(table, n_p4, d_p4, 4, 4, cs), "psi4 finish");
  ck(cudaMemcpyAsync(s->pin_table[buf], table, sizeof(DsDev) * S, cudaMemcpyDeviceToHost, cs), "table download");
  if (!st.done) ck(cudaEventCreateWithFlags(&st.done, cudaEventDisableTiming), "event");
  ck(cudaEventRecord(st.done, cs), "event record");
  st.launched = Clock::now();
  st.evals = step_evals;
  s->inflight.push_back(st);
  s->next_buf ^= 1;
  s->steps++;
  return true;
}

// Process the oldest in-flight step if it has completed (or missed its deadline).
bool reap_step(kde_server* s, bool block) {
  if (s->inflight.empty()) return false;
  Step& st = s->inflight.front();
  cudaError_t q = cudaEventQuery(st.done);
  const bool late = s->cfg.step_deadline_ms > 0 &&
                    Clock::now() - st.launched > std::chrono::milliseconds(s->cfg.step_deadline_ms);
  if (q == cudaErrorNotReady) {
    if (late) {
      // host-side failure detection: fail the requests of a late step (their
      // regions are released only once the device work has completed)
      for (uint64_t t : st.refs) {
        Req* r = s->reqs[t];
        if (!r->finished && !r->failed) {
          r->failed = true;
          r->fail_status = KDE_ETIMEDOUT;
          finish_req(s, r, KDE_ETIMEDOUT);
        }
      }
      s->cv_done.notify_all();
    }
    if (!block) return false;
    cudaEventSynchronize(st.done);
  } else if (q != cudaSuccess) {
    s->worker_error = cuda_fail(q, "step");
  }
  const DsDev* tab = reinterpret_cast<const DsDev*>(s->pin_table[st.buf]);
  // phase transitions and completions observed by this step
  for (uint64_t t : st.refs) {
    Req* r = s->reqs[t];
    r->in_flight--;
    if (r->failed || r->finished) continue;
    // Only the step that ran the phase's finishing kernels carries its
    // result: with two steps in flight, the earlier one is reaped after the
    // later one (holding the finish) was built.
    if (r->pending_finish && r->finish_step == st.seq) {
      const kde_result& res = tab[r->slot].res;
      r->pending_finish = 0;
      const bool last = (r->phase == P_PSI4) || (r->phase == P_LSCV && !(r->methods & KDE_METHOD_PLUGIN));
      if (res.status != KDE_OK || last) {
        r->result = res;
        r->phase = P_DONE;
        finish_req(s, r, res.status);
      } else {
        r->phase = (r->phase == P_LSCV) ? P_PSI6 : P_PSI4;
        r->cursor = 0;
      }
    }
  }
  for (uint64_t t : st.refs) {
    Req* r = s->reqs[t];
    if ((r->finished || r->cancel) && r->in_flight == 0 && r->slot >= 0) {
      if (!r->finished) finish_req(s, r, KDE_ECANCELLED);
      release_req(s, r);
    }
  }
  cudaEventDestroy(st.done);
  s->inflight.pop_front();
  s->cv_done.notify_all();
  return true;
}

void worker_main(kde_server* s) {
  cudaSetDevice(s->cfg.device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (!s->stop) {
    // release cancelled or failed requests that no step references
    for (int k = 0; k < s->cfg.max_slots; ++k) {
      if (!s->slot_owner[k]) continue;
      Req* r = s->reqs[s->slot_owner[k]];
      if ((r->cancel || r->failed) && r->in_flight == 0) {
        if (!r->finished) finish_req(s, r, KDE_ECANCELLED);
        release_req(s, r);
        s->cv_done.notify_all();
      }
    }
    admit(s);
    int active = 0;
    for (int k = 0; k < s->cfg.max_slots; ++k) active += s->slot_owner[k] != 0;
    s->active_max = std::max(s->active_max, active);
    bool launched = false;
    if (s->inflight.size() < 2) {
      int err = 0;
      launched = launch_step(s, &err);
      if (err) s->worker_error = err;
    }
    bool reaped = reap_step(s, false);
    if (!launched && !reaped) {
      if (s->inflight.empty() && s->queue.empty() && active == 0) {
        s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
      } else {
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(50));
        lk.lock();
      }
    }
  }
  while (!s->inflight.empty()) reap_step(s, true);
}

}  // namespace

extern "C" {

int kde_serve_create(const kde_serve_config* cfg, kde_server** out) {
  if (!cfg || !out) return fail(KDE_EINVAL, "serve: NULL argument");
  *out = nullptr;
  if (!cfg->arena || reinterpret_cast<uintptr_t>(cfg->arena) % 256) return fail(KDE_EINVAL, "serve: arena NULL or misaligned");
  if (cfg->max_slots < 1 || cfg->max_slots > kMaxSlots) return fail(KDE_EINVAL, "serve: max_slots outside [1, %d]", kMaxSlots);
  int rc = check_opts(cfg->opts);
  if (rc) return rc;
  kde_server* s = new (std::nothrow) kde_server();
  if (!s) return fail(KDE_ENOMEM, "serve: host memory");
  s->cfg = *cfg;
  if (cfg->opts) {
    s->opts = *cfg->opts;
    s->has_opts = true;
  }
  s->cfg.opts = nullptr;
  cudaSetDevice(cfg->device);
  s->sms = device_sms();
  s->arena = static_cast<unsigned char*>(cfg->arena);
  const int S = cfg->max_slots;
  size_t o = 0;
  s->table_off = o;
  o += (sizeof(DsDev) * S + 255) / 256 * 256;
  s->params_bytes = (params_block_bytes(S) + 255) / 256 * 256;
  s->params_off[0] = o;
  o += s->params_bytes;
  s->params_off[1] = o;
  o += s->params_bytes;
  s->heap_off = o;
  if (cfg->arena_bytes <= o + 4096) {
    delete s;
    return fail(KDE_ENOMEM, "serve: arena of %zu bytes is smaller than the %zu-byte table", cfg->arena_bytes, o);
  }
  s->heap.init(cfg->arena_bytes - o);
  s->slot_owner.assign(S, 0);
  bool ok = cudaStreamCreateWithFlags(&s->comp[0], cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&s->comp[1], cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking) == cudaSuccess;
  for (int b = 0; b < 2 && ok; ++b)
    ok = cudaMallocHost(&s->pin_params[b], s->params_bytes) == cudaSuccess &&
         cudaMallocHost(&s->pin_table[b], sizeof(DsDev) * S) == cudaSuccess;
  for (int b = 0; b < 2 && ok; ++b) {
    ok = cudaEventCreateWithFlags(&s->ev_fork[b], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&s->ev_kdone[b], cudaEventDisableTiming) == cudaSuccess;
    for (int k = 0; k < kSideStreams && ok; ++k)
      ok = cudaStreamCreateWithFlags(&s->side[b][k], cudaStreamNonBlocking) == cudaSuccess &&
           cudaEventCreateWithFlags(&s->ev_join[b][k], cudaEventDisableTiming) == cudaSuccess;
  }
  if (!ok) {
    kde_serve_destroy(s);
    return fail(KDE_ECUDA, "serve: streams or pinned staging");
  }
  // every kernel variant's shared-memory attribute up front
  for (int d : {1, 2, 3, 4, 8, 12, 16})
    for (int B : {2, 8, 16})
      for (int R : {1, 4})
        for (int k = 0; k < 2; ++k)
          if (d <= 4 || R == 1) {
            prepare_lscv(d, B, R, k == 0, false);
            if (B == 16) prepare_lscv(d, B, R, k == 0, true);
          }
  s->worker = std::thread(worker_main, s);
  *out = s;
  return KDE_OK;
}

int kde_serve_submit(kde_server* s, const kde_request* q, uint64_t* ticket) {
  if (!s || !q || !ticket) return fail(KDE_EINVAL, "serve: NULL argument");
  if (!q->x) return fail(KDE_EINVAL, "serve: x is NULL");
  if (q->dtype != KDE_F32 && q->dtype != KDE_F64) return fail(KDE_EINVAL, "serve: dtype");
  if (q->n < 2 || q->n > ((int64_t)1 << 31) || q->d < 1 || q->d > KDE_MAX_D) return fail(KDE_EINVAL, "serve: n or d");
  if (!(q->methods & 3) || (q->methods & ~3) || ((q->methods & KDE_METHOD_PLUGIN) && q->d != 1))
    return fail(KDE_EINVAL, "serve: methods %d for d = %d", q->methods, q->d);
  Req* r = new (std::nothrow) Req();
  if (!r) return fail(KDE_ENOMEM, "serve: host memory");
  r->methods = q->methods;
  r->dtype = q->dtype;
  r->d = q->d;
  r->n = q->n;
  int n_h = 0;
  if (q->methods & KDE_METHOD_LSCV) {
    int rc = build_grid(&q->grid, q->n, q->d, &r->grid);
    if (rc) {
      delete r;
      return rc;
    }
    n_h = (int)r->grid.size();
  }
  // items of at most a twelfth of a CTA's share of one step: every step spans
  // all CTAs and launch tails stay short
  const int cps = (s->has_opts && s->opts.ctas_per_sm) ? s->opts.ctas_per_sm : 2;
  const double max_item = step_budget(s) / (12.0 * std::max(1, s->sms) * cps);
  int rc = make_geometry(q->n, q->d, n_h, s->has_opts ? &s->opts : nullptr, s->sms, &r->geo, max_item);
  if (rc) {
    delete r;
    return rc;
  }
  if (n_h) apply_octave(&r->geo, r->grid);
  r->region_bytes = r->geo.total;
  if (n_h) {
    r->nc.assign(r->geo.n_h_pad, -1.0f);
    for (int k = 0; k < n_h; ++k) r->nc[k] = (float)(-1.0 / (r->grid[k] * r->grid[k]));
  }
  if (r->region_bytes + s->heap_off > s->cfg.arena_bytes) {
    delete r;
    std::lock_guard<std::mutex> lk(s->mu);
    s->rejected++;
    return fail(KDE_EBUSY, "serve: request needs %zu bytes, more than the whole arena", r->region_bytes);
  }
  const size_t bytes = (size_t)q->d * q->n * (q->dtype == KDE_F64 ? 8 : 4);
  r->samples.assign(static_cast<const unsigned char*>(q->x), static_cast<const unsigned char*>(q->x) + bytes);
  r->t_submit = Clock::now();
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->cfg.max_queue > 0 && (int)s->queue.size() >= s->cfg.max_queue) {
    s->rejected++;
    delete r;
    return fail(KDE_EBUSY, "serve: admission queue full");
  }
  r->ticket = s->next_ticket++;
  s->reqs[r->ticket] = r;
  s->queue.push_back(r->ticket);
  s->queue_max = std::max(s->queue_max, (int)s->queue.size());
  s->submitted++;
  if (!s->any_submit) {
    s->any_submit = true;
    s->t_first_submit = r->t_submit;
  }
  *ticket = r->ticket;
  s->cv_work.notify_one();
  return KDE_OK;
}

static int take_result(kde_server* s, uint64_t ticket, kde_result* out, bool erase) {
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return fail(KDE_ENOTFOUND, "serve: ticket %llu unknown", (unsigned long long)ticket);
  Req* r = it->second;
  if (!r->finished) return KDE_EAGAIN;
  if (out) *out = r->result;
  const int st = r->result.status;
  if (erase && r->slot < 0) {
    delete r;
    s->reqs.erase(it);
  }
  return st == KDE_OK ? KDE_OK : fail(st, "serve: request %llu: %s", (unsigned long long)ticket, kde_status_string(st));
}

int kde_serve_poll(kde_server* s, uint64_t ticket, kde_result* out) {
  if (!s) return fail(KDE_EINVAL, "serve: NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->worker_error) return s->worker_error;
  return take_result(s, ticket, out, true);
}

int kde_serve_wait(kde_server* s, uint64_t ticket, int timeout_ms, kde_result* out) {
  if (!s) return fail(KDE_EINVAL, "serve: NULL server");
  std::unique_lock<std::mutex> lk(s->mu);
  const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
  for (;;) {
    if (s->worker_error) return s->worker_error;
    int rc = take_result(s, ticket, out, true);
    if (rc != KDE_EAGAIN) return rc;
    if (timeout_ms >= 0 && Clock::now() >= deadline)
      return fail(KDE_ETIMEDOUT, "serve: request %llu not done after %d ms", (unsigned long long)ticket, timeout_ms);
    s->cv_done.wait_for(lk, std::chrono::milliseconds(2));
  }
}

int kde_serve_cancel(kde_server* s, uint64_t ticket) {
  if (!s) return fail(KDE_EINVAL, "serve: NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return fail(KDE_ENOTFOUND, "serve: ticket unknown");
  Req* r = it->second;
  if (r->finished) return KDE_OK;
  r->cancel = true;
  if (r->slot < 0) {  // still queued: drop now
    s->queue.erase(std::remove(s->queue.begin(), s->queue.end(), ticket), s->queue.end());
    finish_req(s, r, KDE_ECANCELLED);
    r->result.status = KDE_ECANCELLED;
  }
  s->cv_work.notify_one();
  return KDE_OK;
}

static double pct(std::vector<double> v, double p) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double pos = p * (v.size() - 1);
  const size_t i = (size_t)pos;
  const double f = pos - i;
  return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
}

int kde_serve_stats(kde_server* s, kde_serve_stats_t* out) {
  if (!s || !out) return fail(KDE_EINVAL, "serve: NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  memset(out, 0, sizeof(*out));
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->failed = s->failed;
  out->cancelled = s->cancelled;
  out->rejected = s->rejected;
  out->p50_ms = pct(s->lat_ms, 0.50);
  out->p99_ms = pct(s->lat_ms, 0.99);
  out->max_ms = s->lat_ms.empty() ? 0 : *std::max_element(s->lat_ms.begin(), s->lat_ms.end());
  double sum = 0;
  for (double v : s->lat_ms) sum += v;
  out->mean_ms = s->lat_ms.empty() ? 0 : sum / s->lat_ms.size();
  out->p50_wait_ms = pct(s->wait_ms, 0.50);
  out->p99_wait_ms = pct(s->wait_ms, 0.99);
  if (s->completed && s->any_submit) {
    const double secs = std::chrono::duration<double>(s->t_last_done - s->t_first_submit).count();
    out->requests_per_s = secs > 0 ? s->completed / secs : 0;
    out->evals_per_s = secs > 0 ? s->evals_done / secs : 0;
  }
  out->steps = s->steps;
  out->queue_depth_max = s->queue_max;
  out->active_max = s->active_max;
  out->arena_peak_bytes = s->heap.peak() + s->heap_off;
  return KDE_OK;
}

int kde_serve_destroy(kde_server* s) {
  if (!s) return KDE_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv_work.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  for (auto& kv : s->reqs) {
    release_req(s, kv.second);
    delete kv.second;
  }
  for (int b = 0; b < 2; ++b) {
    if (s->pin_params[b]) cudaFreeHost(s->pin_params[b]);
    if (s->pin_table[b]) cudaFreeHost(s->pin_table[b]);
  }
  if (s->copy) cudaStreamDestroy(s->copy);
  for (int b = 0; b < 2; ++b) {
    if (s->comp[b]) cudaStreamDestroy(s->comp[b]);
    for (int k = 0; k < kSideStreams; ++k) {
      if (s->side[b][k]) cudaStreamDestroy(s->side[b][k]);
      if (s->ev_join[b][k]) cudaEventDestroy(s->ev_join[b][k]);
    }
    if (s->ev_fork[b]) cudaEventDestroy(s->ev_fork[b]);
    if (s->ev_kdone[b]) cudaEventDestroy(s->ev_kdone[b]);
  }
  delete s;
  return KDE_OK;
}

}  // extern "C"
