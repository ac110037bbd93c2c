/*
 * gbkde.h -- C ABI of libgbkde, exact kernel-density bandwidth selection on
 * GB300 (sm_103a), following Gramacki & Andrzejewski, "Density Estimations for
 * Approximate Query Processing on SIMD Architectures" (arXiv 1505.01998).
 *
 * The library computes the O(n^2) all-pairs Gaussian-kernel reductions of
 * three bandwidth selectors:
 *   - PLUGIN (Sec. 4.4.1): two-stage plug-in h for univariate data, built on
 *     the density-derivative functionals psi_6 and psi_4;
 *   - LSCV_h (Sec. 4.4.2): the least-squares cross-validation objective g(h)
 *     with bandwidth matrix H = h^2 S (S = sample covariance), evaluated on a
 *     grid of h and minimised by brute force on the grid (Eq. LSCV-finalH);
 *   - LSCV_H (Sec. 4.4.3): the objective g(H) for general bandwidth matrices.
 *
 * Conventions shared by every entry point
 *  - Status: every call returns an int status (KDE_OK = 0 or a KDE_E* code).
 *    kde_last_error() returns a human-readable detail for the calling thread.
 *  - Samples: a d x n matrix with one sample per column, row-major, i.e.
 *    x[k*n + i] is coordinate k of sample i (the paper's input matrix of
 *    Sec. 4.4.2, Eq. LSCV-InputData).  Element type KDE_F32 or KDE_F64.
 *    1 <= d <= 16 (the paper's experiments span d = 1..16, Sec. 7.2), n >= 2,
 *    all values finite.
 *  - Memory: the caller owns every buffer.  Device pointers must be device
 *    memory of the current CUDA device; the workspace must be at least
 *    kde_workspace_size() bytes and 256-byte aligned.  No entry point
 *    allocates device memory.  Host result pointers may be NULL when a result
 *    is not wanted.
 *  - Streams: `stream` is a cudaStream_t (NULL = legacy default stream).  All
 *    device work is queued on it.  Entry points without the _async suffix
 *    copy their results to the host and synchronise that stream before
 *    returning.  _async entry points queue work only and write results to
 *    device memory inside the workspace (see kde_ws_result_offset).
 *  - Arithmetic: pair terms in FP32 (exp by ex2.approx), per-thread sums in
 *    FP32 with Kahan compensation (KDE_FP32_KAHAN, default) or plain FP32
 *    (KDE_FP32_PLAIN); every reduction across threads and blocks, the scalar
 *    plug-in chain, g(h) and the argmin in FP64.
 */
#ifndef GBKDE_H
#define GBKDE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define KDE_OK 0
#define KDE_EINVAL 1      /* invalid argument (sizes, pointers, d, n, grid)    */
#define KDE_ENOMEM 2      /* workspace or arena too small                      */
#define KDE_ECUDA 3       /* a CUDA runtime call failed                        */
#define KDE_EDEGENERATE 4 /* the method is undefined for these data (see below) */
#define KDE_EBUSY 5       /* server full: no slot or HBM budget for a request  */
#define KDE_EAGAIN 6      /* result not ready yet                              */
#define KDE_ETIMEDOUT 7   /* wait timed out                                    */
#define KDE_ECANCELLED 8  /* request was cancelled                             */
#define KDE_ENOTFOUND 9   /* unknown ticket                                    */
#define KDE_EINTERNAL 10  /* internal consistency check failed                 */

/* sample element types */
#define KDE_F32 0
#define KDE_F64 1

/* per-thread summation modes of the pair kernels */
#define KDE_FP32_KAHAN 0
#define KDE_FP32_PLAIN 1

/* bandwidth grid kinds */
#define KDE_GRID_DEFAULT_Z 0 /* h_k = (h0/4) 16^(k/n_h), k < n_h: log-spaced over Z(h0) = [h0/4, 4 h0) */
#define KDE_GRID_EXPLICIT 1  /* the n_h values in h[] (need not be sorted)       */
#define KDE_GRID_LOG 2       /* n_h log-spaced points over [h_min, h_max]        */

#define KDE_MAX_D 16
#define KDE_MAX_NH 1024

/* result flags */
#define KDE_FLAG_MIN_AT_LOWER_EDGE 1 /* argmin is the first grid point */
#define KDE_FLAG_MIN_AT_UPPER_EDGE 2 /* argmin is the last grid point  */

/* methods (for batch / serving requests) */
#define KDE_METHOD_LSCV 1
#define KDE_METHOD_PLUGIN 2

/* A grid of bandwidth multipliers h (H = h^2 S).  For DEFAULT_Z, h0 is the
 * normal-scale rule (4/((d+2) n))^(1/(d+4)) (Eq. LSCV-h0; equal to the
 * printed constants at d = 1) and the range is Eq. LSCV-Zh0. */
typedef struct kde_grid {
  int kind;
  int n_h;          /* 1 .. KDE_MAX_NH */
  const double* h;  /* host array of n_h values, for KDE_GRID_EXPLICIT */
  double h_min;     /* for KDE_GRID_LOG */
  double h_max;
} kde_grid;

/* Tuning knobs; zero means "choose automatically". */
typedef struct kde_opts {
  int precision;      /* KDE_FP32_KAHAN (0) or KDE_FP32_PLAIN                  */
  int tile;           /* LSCV pair tile edge T: 32 or 128 samples               */
  int bw_per_thread;  /* LSCV bandwidths per thread B: 2, 8 or 16 (0: 2 for grids
                         of 1 or 2 points, else the tuner's or the default rule) */
  int tiles_per_item; /* tiles per work item K (1 .. 4096)                      */
  int ctas_per_sm;    /* resident CTAs per SM of the persistent pair kernels    */
  int cv;             /* LSCV weights: KDE_CV_PAPER (0) or KDE_CV_LOO           */
} kde_opts;

/* LSCV objective weights.  KDE_CV_PAPER: n^-2 on the pair sum as printed in
 * Eq. LSCV-gh (reading R2).  KDE_CV_LOO: exact leave-one-out cross-validation,
 * g = h^-d A [n^-1 + 2 n^-2 S1 - 2^(2+d/2) S2 / (n (n-1))]. */
#define KDE_CV_PAPER 0
#define KDE_CV_LOO 1

/* Result of one selection.  Fields that do not apply are 0. */
typedef struct kde_result {
  int status;     /* KDE_OK or KDE_EDEGENERATE                                  */
  int method;     /* KDE_METHOD_LSCV or KDE_METHOD_PLUGIN                       */
  int argmin;     /* LSCV: first grid index attaining the minimum of g          */
  int flags;      /* KDE_FLAG_*                                                 */
  int n_h;
  int d;
  double h;       /* LSCV: selected multiplier (H = h^2 S); PLUGIN: h (data units) */
  double h_data;  /* d = 1: selected bandwidth in data units                    */
  double g_min;   /* LSCV: g at the argmin                                      */
  double sigma;   /* d = 1: sample standard deviation (Eq. PLUGIN-StdDevEstimator) */
  double psi8_ns; /* PLUGIN: Eq. PLUGIN-Psi8Estimate                            */
  double g1;      /* PLUGIN: Eq. PLUGIN-g1                                      */
  double psi6;    /* PLUGIN: Eq. PLUGIN-Psi6Estimate (reading R1)               */
  double g2;      /* PLUGIN: Eq. PLUGIN-g2                                      */
  double psi4;    /* PLUGIN: Eq. PLUGIN-Psi4Estimate (reading R1)               */
  double logdet_S;/* log det S                                                  */
  double h_plugin;/* PLUGIN: h (data units), also when LSCV ran on the same data  */
} kde_result;

/* ------------------------------------------------------------- utilities */

/* Library version string (static storage). */
const char* kde_version(void);

/* Copies the calling thread's last error detail into buf (NUL-terminated,
 * truncated to len).  Returns the status of that error (KDE_OK if none). */
int kde_last_error(char* buf, size_t len);

/* Static description of a status code. */
const char* kde_status_string(int status);

/* Number of tiles of the upper pair triangle for n samples and tile edge T:
 * NT (NT + 1) / 2 with NT = ceil(n / T) (Sec. 5.4.1, pair triangle in k x k
 * tiles with zero padding of n to a multiple of k). */
int kde_tile_count(int64_t n, int tile, int64_t* tiles);

/* The tile map of Sec. 5.4.2 (Eqs. colInTriangleMatrix, rowInTriangleMatrix;
 * Appendix A): tile number bx -> column l and row q, q <= l, of the upper
 * triangle, column l holding tiles l(l+1)/2 .. l(l+1)/2 + l.  The float
 * square-root formula is followed by an exact integer correction.  This is
 * the same function the kernels run, compiled for the host. */
int kde_tile_coords(int64_t bx, int64_t* l, int64_t* q);

/* The library's default grid for n samples in d dimensions (host output). */
int kde_default_grid(int64_t n, int d, int n_h, double* h_out);

/* ------------------------------------------------------------ workspace */

/* Bytes of workspace needed by kde_lscv / kde_plugin / kde_lscv_tile_sums /
 * kde_psi_tile_sums / kde_lscv_H for n samples in d dimensions and n_h
 * bandwidths (use n_h = 1 for plug-in only) with the given options (NULL =
 * defaults).  The workspace also holds the device-side copy of a host input
 * (the *_host entry points). */
int kde_workspace_size(int64_t n, int d, int n_h, const kde_opts* opts, size_t* bytes);

/* Offset, in bytes from the workspace base, of the kde_result written by
 * the last _async call that used that workspace, and of its g[n_h] array. */
int kde_ws_result_offset(size_t* result_offset, size_t* g_offset);

/* ------------------------------------------------------------- LSCV_h */

/* LSCV_h bandwidth selection (Sec. 4.4.2; GPU design of Sec. 6.2 replaced by a
 * fused all-pairs, all-bandwidths kernel).  Computes the covariance S
 * (Eq. LSCV-covariance), its Cholesky factor, and for every grid point
 * g(h) = h^-d [2 n^-2 sum_{i<j} T((X_i - X_j)/h) + n^-1 R(K)] (Eq. LSCV-gh,
 * R(K) = (4 pi)^(-d/2) |S|^(-1/2)); then the argmin over the grid.
 *   x_dev   device samples, d x n row-major, element type dtype
 *   g_host  optional host output, n_h values of g in grid order
 *   h_host  optional host output, the n_h grid values used
 *   out     host result (required)
 * Errors: KDE_EINVAL (bad sizes/pointers/grid), KDE_ENOMEM (workspace too
 * small), KDE_EDEGENERATE (S singular or not positive definite; also
 * reported in out->status), KDE_ECUDA. */
int kde_lscv(const void* x_dev, int dtype, int64_t n, int d, const kde_grid* grid,
             const kde_opts* opts, void* ws, size_t ws_bytes, void* stream,
             double* g_host, double* h_host, kde_result* out);

/* As kde_lscv, queue only: the result and g[] stay in the workspace. */
int kde_lscv_async(const void* x_dev, int dtype, int64_t n, int d, const kde_grid* grid,
                   const kde_opts* opts, void* ws, size_t ws_bytes, void* stream);

/* As kde_lscv with HOST samples: copies x_host into the workspace on the
 * stream (pageable or pinned host memory), runs, copies the result back. */
int kde_lscv_host(const void* x_host, int dtype, int64_t n, int d, const kde_grid* grid,
                  const kde_opts* opts, void* ws, size_t ws_bytes, void* stream,
                  double* g_host, kde_result* out);

/* Raw LSCV pair sums over the tiles [tile_begin, tile_end) of the pair
 * triangle (tile edge opts->tile, tile numbering of kde_tile_coords), for the
 * n_h multipliers h_host[]:
 *   s1[k] = sum exp(-S(v)/(4 h_k^2)),  s2[k] = sum exp(-S(v)/(2 h_k^2))
 * over pairs i < j < n in those tiles, S(v) = v^T S^-1 v (Eq. LSCV_MOD-Pv).
 * The sums over disjoint tile ranges add up to the full sums: this is the
 * unit of multi-GPU sharding and of sampled parity checks. */
int kde_lscv_tile_sums(const void* x_dev, int dtype, int64_t n, int d, const double* h_host,
                       int n_h, int64_t tile_begin, int64_t tile_end, const kde_opts* opts,
                       void* ws, size_t ws_bytes, void* stream, double* s1_host,
                       double* s2_host);

/* log det S of the samples (the prologue of kde_lscv, FP64 on the device):
 * what kde_lscv_merge needs besides the summed exponential sums. */
int kde_lscv_logdet(const void* x_dev, int dtype, int64_t n, int d, void* ws, size_t ws_bytes,
                    void* stream, double* logdet_S);

/* Finishes a sharded LSCV_h selection on the host in FP64: from the full
 * exponential sums s1, s2 (the element-wise sum of kde_lscv_tile_sums over
 * shards that cover the tile range exactly once) computes
 * g(h) = h^-d A [2 n^-2 (s1 - 2^(1+d/2) s2) + n^-1], A = (4 pi)^(-d/2) exp(-logdet_S/2)
 * (Eq. LSCV-gh) and the first-index argmin (Eq. LSCV-finalH).  g_out may be
 * NULL; out receives argmin, h, g_min, flags. */
int kde_lscv_merge(int64_t n, int d, double logdet_S, const double* h, int n_h, const double* s1,
                   const double* s2, double* g_out, kde_result* out);

/* Tile edge and tiles per work item of the single-GPU geometry for n
 * samples in d dimensions on the LSCV grid h[n_h] (NULL: the default grid of
 * n_h points; the grid's shape picks the octave or the direct kernel, whose
 * item sizes differ) and of the psi kernels, on the current device with the
 * given options (NULL = defaults).  Shards whose tile ranges start on
 * multiples of the item size evaluate exactly the items of the single
 * launch.  Any output may be NULL. */
int kde_item_tiles(int64_t n, int d, const double* h, int n_h, const kde_opts* opts, int* lscv_tile,
                   int* lscv_K, int* psi_tile, int* psi_K);

/* Bracketing search for argmin g(h) over [h_lo, h_hi] (<= 0: Z(h0), Eq.
 * LSCV-Zh0): the golden-section alternative to the dense grid named in
 * Sec. 4.4.2, evaluated 8 interior points per round (log-spaced) in one pass;
 * the bracket becomes the neighbours of the best point (log-width x 2/9 per
 * round) until it is within 2 rel_tol (log) or after max_rounds.  out->h and
 * out->g_min hold the best evaluated point (a local minimum if g is not
 * unimodal); out->flags has KDE_FLAG_MIN_AT_LOWER_EDGE (UPPER_EDGE) when every
 * round kept the bracket's lower (upper) end, i.e. g still falls towards that
 * end of [h_lo, h_hi]; rounds_out (optional) the rounds taken.  Workspace:
 * kde_workspace_size(n, d, 8).  Synchronises the stream every round. */
int kde_lscv_search(const void* x_dev, int dtype, int64_t n, int d, double h_lo, double h_hi,
                    double rel_tol, int max_rounds, const kde_opts* opts, void* ws, size_t ws_bytes,
                    void* stream, kde_result* out, int* rounds_out);

/* ------------------------------------------------------------- PLUGIN */

/* PLUGIN bandwidth selection for univariate data (Sec. 4.4.1, steps 1-8; GPU
 * composition of Sec. 6.1 with the scalar steps on the device in FP64):
 * variance, sigma, psi_8^NS, g1, psi_6(g1) over all pairs, g2, psi_4(g2) over
 * all pairs, h.  psi_r(g) = n^-2 g^-(r+1) [2 sum_{i<j} K^(r)((x_i-x_j)/g) +
 * n K^(r)(0)] (reading R1 of the garbled Eqs. PLUGIN-Psi6Estimate/Psi4Estimate).
 * Errors: KDE_EINVAL, KDE_ENOMEM, KDE_EDEGENERATE (sigma = 0, psi_6 >= 0 or
 * psi_4 <= 0; also in out->status), KDE_ECUDA. */
int kde_plugin(const void* x_dev, int dtype, int64_t n, const kde_opts* opts, void* ws,
               size_t ws_bytes, void* stream, kde_result* out);

/* As kde_plugin, queue only (result stays in the workspace). */
int kde_plugin_async(const void* x_dev, int dtype, int64_t n, const kde_opts* opts, void* ws,
                     size_t ws_bytes, void* stream);

/* As kde_plugin with HOST samples (copied into the workspace on the stream). */
int kde_plugin_host(const void* x_host, int dtype, int64_t n, const kde_opts* opts, void* ws,
                    size_t ws_bytes, void* stream, kde_result* out);

/* Raw psi pair sum over the tiles [tile_begin, tile_end) of the pair
 * triangle (tile edge 64, 256 or 512 by n, see kde_psi_tile_edge):
 *   sum K^(r)((x_i - x_j)/g) over pairs i < j < n in those tiles, r in {4,6,8}. */
int kde_psi_tile_sums(const void* x_dev, int dtype, int64_t n, int r, double g,
                      int64_t tile_begin, int64_t tile_end, const kde_opts* opts, void* ws,
                      size_t ws_bytes, void* stream, double* sum_host);

/* Tile edge used by the psi kernels for n samples (for kde_psi_tile_sums). */
int kde_psi_tile_edge(int64_t n, const kde_opts* opts, int* tile);

/* One scalar step of a sharded PLUGIN selection on the host in FP64
 * (Sec. 4.4.1, readings as in kde_plugin), updating *res in place:
 *   stage 8: value = sigma (> 0): resets *res, sets sigma, psi_8^NS
 *            (Eq. PLUGIN-Psi8Estimate) and g1 (Eq. PLUGIN-g1);
 *   stage 6: value = sum_{i<j} K^(6)((x_i - x_j)/g1) over all pairs (the sum
 *            of kde_psi_tile_sums over shards covering the tiles once): psi_6
 *            (Eq. PLUGIN-Psi6Estimate) and g2 (Eq. PLUGIN-g2);
 *   stage 4: value = the same sum of K^(4) at g2: psi_4 (Eq. PLUGIN-Psi4Estimate)
 *            and h (Eq. PLUGIN-Final_h) into h, h_data and h_plugin.
 * Errors: KDE_EINVAL (arguments, stages out of order), KDE_EDEGENERATE
 * (sigma <= 0, psi_6 >= 0, psi_4 <= 0; res->status is set too). */
int kde_plugin_merge(int64_t n, int stage, double value, kde_result* res);

/* ------------------------------------------------------------- LSCV_H */

/* Workspace bytes for kde_lscv_H with m bandwidth matrices. */
int kde_lscv_H_workspace_size(int64_t n, int d, int m, const kde_opts* opts, size_t* bytes);

/* The LSCV_H objective g(H) (Sec. 4.4.3, Eqs. LSCV_MULTI-gh, LSCV_MULTI-Tx,
 * LSCV_MULTI-Kx, LSCV_MULTI-KKx, LSCV_MULTI-rk) for m symmetric positive-
 * definite bandwidth matrices H_host[m][d][d] (row-major, host), in one
 * batched pass over the pairs: each H whitens the samples by its Cholesky
 * factor, so (X_i - X_j)^T H^-1 (X_i - X_j) is a squared distance.  g_host
 * receives m values.  Errors: KDE_EINVAL (m outside [1, KDE_MAX_NH], H not
 * finite or not symmetric), KDE_EDEGENERATE (an H not positive definite),
 * KDE_ENOMEM, KDE_ECUDA.  Synchronises the stream. */
int kde_lscv_H(const void* x_dev, int dtype, int64_t n, int d, const double* H_host, int m,
               const kde_opts* opts, void* ws, size_t ws_bytes, void* stream, double* g_host);

/* Sample covariance S (d x d, row-major, n-1 denominator; Eq. LSCV-covariance,
 * two-pass) computed by the device prologue.  Workspace: kde_workspace_size(n,
 * d, 1).  Synchronises the stream. */
int kde_sample_covariance(const void* x_dev, int dtype, int64_t n, int d, void* ws, size_t ws_bytes,
                          void* stream, double* cov);

/* Minimises g(H) over symmetric positive-definite H (Sec. 4.4.3) by
 * Nelder-Mead over vech of the Cholesky factor of H with log-diagonal entries
 * (every simplex point is positive definite), starting from H_start (NULL:
 * the normal-scale (4/(d+2))^(2/(d+4)) n^(-2/(d+4)) S, reading R5 of
 * Eq. LSCV-H-start).  Every iteration evaluates reflection, expansion and
 * both contractions in one batched kde_lscv_H pass; a shrink in one more.
 * Stops when max |g - g_best| over the simplex <= ftol |g_best| or after
 * max_iter iterations.  H_out (d x d) and g_out receive the best point;
 * evals_out (optional) the number of g(H) evaluations.  Workspace: the larger
 * of kde_workspace_size(n, d, 1) and kde_lscv_H_workspace_size(n, d,
 * max(4, d(d+1)/2 + 1)). */
int kde_lscv_H_minimize(const void* x_dev, int dtype, int64_t n, int d, const double* H_start,
                        int max_iter, double ftol, const kde_opts* opts, void* ws, size_t ws_bytes,
                        void* stream, double* H_out, double* g_out, int* evals_out);

/* -------------------------------------------------------------- batches */

/* One selection request of a batch (device samples) or of the server (host
 * samples).  methods: KDE_METHOD_LSCV and/or KDE_METHOD_PLUGIN (PLUGIN needs
 * d = 1); grid: the LSCV grid (ignored without KDE_METHOD_LSCV). */
typedef struct kde_request {
  const void* x;
  int dtype;
  int d;
  int64_t n;
  int methods;
  kde_grid grid;
} kde_request;

typedef struct kde_batch_plan kde_batch_plan;

/* Plans a batch: per-dataset geometry (the same as a single call would use,
 * so results are bitwise identical alone and batched), kernel-variant groups
 * and the workspace layout; *ws_bytes receives the workspace size.  The
 * request array may be freed afterwards; the sample buffers must stay valid
 * for every run. */
int kde_batch_plan_create(const kde_request* reqs, int n_req, const kde_opts* opts,
                          kde_batch_plan** plan, size_t* ws_bytes);

/* Queues one batched selection of all requests on `stream`: one upload of
 * descriptors, the prologue for every dataset, one persistent launch per
 * kernel variant and phase (LSCV and psi_6 / psi_4 of the PLUGIN method), the
 * fixed-order reductions, the scalar chains and one download of the results.
 * The sequence is captured into a CUDA graph on the first run (and again when
 * the workspace changes) and replayed afterwards. */
int kde_batch_run_async(kde_batch_plan* plan, void* ws, size_t ws_bytes, void* stream);

/* kde_batch_run_async + stream synchronisation + kde_batch_results. */
int kde_batch_run(kde_batch_plan* plan, void* ws, size_t ws_bytes, void* stream, kde_result* outs);

/* Results of the last completed run (outs has n_req entries). */
int kde_batch_results(const kde_batch_plan* plan, kde_result* outs);

/* The LSCV objective g[n_h] of request `req` after a completed run. */
int kde_batch_g(const kde_batch_plan* plan, const void* ws, int req, double* g_host);

int kde_batch_plan_destroy(kde_batch_plan* plan);

/* Workspace bytes of a batch (same layout as kde_batch_plan_create). */
int kde_batch_workspace_size(const kde_request* reqs, int n_req, const kde_opts* opts,
                             size_t* bytes);

/* One-shot batch: plan, run without a graph, synchronise, results, free. */
int kde_select_batch(const kde_request* reqs, int n_req, const kde_opts* opts, void* ws,
                     size_t ws_bytes, void* stream, kde_result* outs);

/* -------------------------------------------------------------- serving */

/* Server configuration.  The arena is device memory owned by the caller (for
 * example a torch tensor); its size is the HBM budget: the slot table and the
 * step parameter blocks sit at its start, request regions (samples, prepared
 * samples, partial sums) are carved from the rest. */
typedef struct kde_serve_config {
  void* arena;            /* 256-byte aligned device memory                         */
  size_t arena_bytes;     /* HBM budget                                              */
  int max_slots;          /* requests resident at once, 1 .. 1024                    */
  int max_queue;          /* waiting requests before submit returns KDE_EBUSY (0 = unbounded) */
  double quantum_evals;   /* work per scheduling step, in evaluations of the direct
                             LSCV kernel: an octave-grid LSCV evaluation counts 0.55,
                             a psi_6 / psi_4 evaluation 1.65 / 1.35 (0 = 1.3e11, ~14 ms) */
  int step_deadline_ms;   /* a step still running after this fails its requests with
                             KDE_ETIMEDOUT (host-side detection; 0 = no deadline)     */
  int device;             /* CUDA device index                                       */
  const kde_opts* opts;   /* geometry options for every request (NULL = defaults)    */
} kde_serve_config;

typedef struct kde_serve_stats_t {
  uint64_t submitted, completed, failed, cancelled, rejected;
  double p50_ms, p99_ms, mean_ms, max_ms; /* submit -> result, completed requests */
  double p50_wait_ms, p99_wait_ms;        /* submit -> admission                   */
  double requests_per_s;                  /* completed / (last result - first submit) */
  double evals_per_s;                     /* pair evaluations of completed requests / same span */
  int64_t steps;
  int queue_depth_max, active_max;
  size_t arena_peak_bytes;
} kde_serve_stats_t;

typedef struct kde_server kde_server;

/* Starts a server: one scheduler thread, one compute and one copy stream on
 * cfg->device.  Requests are advanced together in steps (continuous
 * batching).  A request's work items depend only on the request and the
 * server configuration (items are capped so one step spans every CTA), so
 * its result is bitwise the same whether it runs alone or among others; it
 * equals the single-request entry points' result within the 1e-5 tolerance
 * (those use larger items, so FP32 partial sums are grouped differently). */
int kde_serve_create(const kde_serve_config* cfg, kde_server** server);

/* Queues a request with HOST samples (copied at submit: the caller may reuse
 * its buffer on return).  Admission waits for a free slot and arena space.
 * Errors: KDE_EINVAL, KDE_EBUSY (queue full, or the request alone exceeds the
 * arena). */
int kde_serve_submit(kde_server* server, const kde_request* req, uint64_t* ticket);

/* Result of a finished request (then forgotten): KDE_OK, or the request's
 * failure status (KDE_EDEGENERATE, KDE_ECANCELLED, KDE_ETIMEDOUT ...);
 * KDE_EAGAIN while it is still queued or running; KDE_ENOTFOUND. */
int kde_serve_poll(kde_server* server, uint64_t ticket, kde_result* out);

/* As kde_serve_poll, waiting up to timeout_ms (< 0: no limit); KDE_ETIMEDOUT
 * if the request is still running then (it keeps running). */
int kde_serve_wait(kde_server* server, uint64_t ticket, int timeout_ms, kde_result* out);

/* Cancels a request: dropped at once if queued, at the next step boundary if
 * running; its arena region is released when no launched step references it. */
int kde_serve_cancel(kde_server* server, uint64_t ticket);

int kde_serve_stats(kde_server* server, kde_serve_stats_t* out);

/* Stops the scheduler after the steps in flight complete and frees host
 * resources (the arena stays the caller's). */
int kde_serve_destroy(kde_server* server);

/* ------------------------------------------------ no-allocation variant */

/* Size of the scratch buffer built into the library for kde_lscv_noalloc. */
#define KDE_NOALLOC_MAX_BYTES (16 << 20)

/* kde_lscv without a caller workspace, for callers that cannot allocate
 * device memory: code inside an application whose allocator owns the whole
 * device heap, latency-critical code that must not take cudaMalloc's implicit
 * synchronisation, plain C callers without a tensor library.  The paper has no
 * counterpart; this is a convenience of this library.
 * Arguments and results are those of kde_lscv.  Scratch comes from one
 * KDE_NOALLOC_MAX_BYTES (16 MiB) buffer compiled into the library; every GPU
 * that loads the library holds it until the process exits.  Problems whose
 * workspace (kde_workspace_size) exceeds it are rejected with KDE_ENOMEM
 * before anything is queued.  The first call in each CUDA context (per
 * device, and again after cudaDeviceReset or a re-created primary context,
 * which can load the buffer at another address) looks up the buffer's device
 * address with that context current; make it before any stream capture.
 * Every call shares the buffer, which keeps the previous
 * call's contents (nothing in it needs to start at zero); calls that overlap
 * on the GPU race on it and must be serialised by the caller.  Allocates no
 * device memory; synchronises the stream like kde_lscv. */
int kde_lscv_noalloc(const void* x_dev, int dtype, int64_t n, int d, const kde_grid* grid,
                     const kde_opts* opts, void* stream, double* g_host, double* h_host,
                     kde_result* out);

/* ------------------------------------------- consumers of a bandwidth */

/* Workspace for kde_eval of n samples in d dimensions at m query points. */
int kde_eval_workspace_size(int64_t n, int d, int64_t m, size_t* bytes);

/* Density estimate at query points (Sec. 4.2, the kernel estimator with a
 * bandwidth matrix H and the Gaussian K_H): for every query q_j,
 *   f(q_j) = n^-1 sum_i (2 pi)^-d/2 |H|^-1/2 exp(-(q_j - x_i)^T H^-1 (q_j - x_i) / 2).
 * x_dev: d x n samples (x[k*n + i], as everywhere), KDE_F32 or KDE_F64.
 * H_host: d x d symmetric positive definite bandwidth matrix, row-major host
 * array (for d = 1, h^2; from kde_lscv with H = h^2 S, or kde_lscv_H).
 * q_dev: d x m queries (q[k*m + j]), same dtype as x.  f_host: m doubles.
 * Pairs are evaluated in FP32 (one exp2 per pair) with FP32 Kahan runs per
 * thread and FP64 sums across threads; the result is deterministic.
 * Synchronises the stream.  Errors: KDE_EINVAL (arguments, H not finite or
 * not symmetric), KDE_ENOMEM (workspace too small), KDE_EDEGENERATE (H not
 * positive definite), KDE_ECUDA. */
int kde_eval(const void* x_dev, int dtype, int64_t n, int d, const double* H_host,
             const void* q_dev, int64_t m, void* ws, size_t ws_bytes, void* stream,
             double* f_host);

/* Workspace for kde_aqp of n samples and m ranges. */
int kde_aqp_workspace_size(int64_t n, int m, size_t* bytes);

/* Approximate range aggregates of one numeric column from its sample and a
 * bandwidth h (Sec. 4.3, the Count and Sum estimators over the density
 * estimate).  For every range [lo_k, hi_k], with a = (lo_k - x_i)/h,
 * b = (hi_k - x_i)/h and Phi, phi the standard normal cdf and pdf:
 *   count_k = sum_i [Phi(b) - Phi(a)],
 *   sum_k   = sum_i [x_i (Phi(b) - Phi(a)) + h (phi(a) - phi(b))],
 * i.e. the sample's share of the range and of its total; multiply by
 * N / n for a table of N rows.  x_dev: n samples (KDE_F32 / KDE_F64) in device
 * memory; lo_host, hi_host: m <= KDE_MAX_NH bounds with lo <= hi (either may
 * be infinite; NaN is rejected), rounded to FP32.
 * count_host / sum_host: m doubles each, either may be NULL.  Arithmetic per
 * sample in FP32 (cdf differences taken from the smaller tails; a range end
 * more than 7 h from a sample counts as infinitely far, which changes a term
 * by at most Phi(-7) = 1.3e-12, below its FP32 rounding), FP32 runs per
 * thread and range, FP64 across threads; deterministic.  Synchronises the stream.  Errors: KDE_EINVAL, KDE_ENOMEM,
 * KDE_ECUDA. */
int kde_aqp(const void* x_dev, int dtype, int64_t n, double h, const double* lo_host,
            const double* hi_host, int m, void* ws, size_t ws_bytes, void* stream,
            double* count_host, double* sum_host);

/* ------------------------------------------------------------ autotuner */

#define KDE_TUNE_LATENCY 0    /* one dataset alone on the GPU                    */
#define KDE_TUNE_THROUGHPUT 1 /* the dataset replicated until a launch fills the GPU */

/* Times the LSCV pair kernel for every candidate geometry -- tile edge T in
 * {32, 128}, bandwidths per thread B in {8, 16}, CTAs per SM in {1, 2}, tiles
 * per item at 1x or 2x the default rule -- on the caller's samples and an
 * n_h-point grid (CUDA events around the kernel, best of two runs), and
 * caches the fastest per (device, mode, d, n_h bucket, n bucket; buckets are
 * ceil(log2)).  From then on every entry point of this process uses the
 * cached geometry for options the caller leaves at 0 (throughput entries
 * first).  best receives the winner, best_evals_per_s its rate.  Needs a
 * workspace large enough for the candidates (kde_batch_workspace_size of the
 * replicated dataset); candidates that do not fit are skipped.  Synchronises
 * the stream.  Errors: KDE_EINVAL, KDE_ENOMEM (no candidate fits), KDE_ECUDA. */
int kde_autotune(const void* x_dev, int dtype, int64_t n, int d, int n_h, int mode, void* ws,
                 size_t ws_bytes, void* stream, kde_opts* best, double* best_evals_per_s);

/* Forget every cached tuning of this process. */
int kde_autotune_clear(void);

/* Write / read the tuning cache as text, one line per entry:
 * device mode d nh_bucket n_bucket tile bw ctas_per_sm k_scale evals_per_s. */
int kde_autotune_save(const char* path);
int kde_autotune_load(const char* path);

/* ------------------------------------------------------- measurement aids */

/* Kernel timing hook for the calling thread.  When set (non-NULL cudaEvent_t
 * handles created by the caller), the next LSCV_h / PLUGIN calls of this
 * thread record lscv_begin / lscv_end on their stream immediately around the
 * launch of the all-pairs LSCV kernel, and psi_begin / psi_end around the
 * first all-pairs psi kernel; kde_eval and kde_aqp record lscv_begin /
 * lscv_end around their query x sample (range x sample) kernel.  Pass NULLs to clear.  Never fails. */
int kde_set_kernel_events(void* lscv_begin, void* lscv_end, void* psi_begin, void* psi_end);

/* Sustained per-SM throughput of the units the pair kernels are bound by,
 * measured with clock64() on the current device: MUFU ex2 results, FP32 FMA
 * lanes (scalar FFMA), packed FP32x2 FMA lanes, and packed FP32x2
 * multiply-then-add lanes (the squaring and accumulation of the octave-grid
 * kernel), each per SM per clock.  Also returns the SM count and the
 * effective SM clock (MHz) seen by the probe.  Device-synchronous; allocates
 * nothing (uses the workspace). */
int kde_probe_alu(void* ws, size_t ws_bytes, void* stream, double* mufu_ex2_per_clk_sm,
                  double* ffma_lanes_per_clk_sm, double* ffma2_lanes_per_clk_sm,
                  double* fmul2_fadd2_lanes_per_clk_sm, int* sm_count, double* sm_mhz);

#ifdef __cplusplus
}
#endif
#endif /* GBKDE_H */
