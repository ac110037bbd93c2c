// Host-side declarations shared by the C-ABI translation units.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include "internal.cuh"

namespace gbkde {

// Geometry and workspace layout of one selection (see make_geometry).
struct Geometry {
  int64_t n;
  int d;
  int dk;  // kernel dimension: d for d <= 4, else d rounded up to a multiple of 4
  int n_h;
  int64_t n_pad;
  bool kahan;
  int cv_loo;  // KDE_CV_LOO requested
  int ctas;      // persistent CTAs of the pair kernels
  int ctas_oct;  // persistent CTAs of the octave LSCV kernel (2 or 3 per SM)
  int K_oct;     // tiles per item of the octave LSCV kernel (apply_octave switches to it)
  int64_t rows_oct;
  int64_t item_target;  // LSCV block items aimed at (the tiles-per-item rule)
  // LSCV: tile T = 32 R, B bandwidths per thread, K tiles per item
  int T, R, B, n_h_pad, n_chunks, G, K;
  int64_t tiles, rows, items;
  // psi: tile Tp = 32 Rp, Kp tiles per item
  int Tp, Rp, Kp;
  int64_t ptiles, prows;
  // workspace offsets (bytes)
  int prep_parts;  // CTAs of the prologue (prep_parts_for(n))
  int oct_P;       // > 0: octave grid with this many points per octave (apply_octave)
  size_t off_ds, off_off, off_h, off_nc, off_g, off_sum, off_x, off_y, off_xc, off_lpart,
      off_ppart, off_prep, total;
};

int fail(int status, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* where);
int device_sms();
int check_opts(const kde_opts* o);
int check_common(const void* x, int dtype, int64_t n, int d, void* ws);
// max_item_evals > 0 caps the pair evaluations of one work item (tiles per
// item shrink accordingly): the serving scheduler needs items small enough
// that one step of a fixed evaluation budget spans every CTA.
int make_geometry(int64_t n, int d, int n_h, const kde_opts* o, int sms, Geometry* g,
                  double max_item_evals = 0);
int build_grid(const kde_grid* grid, int64_t n, int d, std::vector<double>* h);
DsDev make_desc(const Geometry& g, const void* x, int dtype, int methods, unsigned char* ws);
// Marks g for the octave-grid kernel when the grid h (ascending) has n_h a
// multiple of 16 (n_h / 8 points per octave of 1/h^2, to 1e-12) and g already
// takes 16 bandwidths per thread; the workspace layout does not change.
void apply_octave(Geometry* g, const std::vector<double>& h);

// CTAs per SM the octave LSCV kernel can hold for dk coordinates: its d <= 4
// instances fit 3 (80 registers), the others 2.  Batches and the server use
// it when the caller gave no CTA count; single calls choose 2 or 3 by the
// balance of their items (make_geometry).
inline int oct_ctas_per_sm(int dk) { return dk <= 4 ? 3 : 2; }
PsiCoef psi_coef(int r);

// Records the caller's timing event k (kde_set_kernel_events) on `st`, if set.
cudaError_t mark_event(int k, cudaStream_t st);

// Cached autotuning of the LSCV geometry (mode 0 latency, 1 throughput);
// out->tiles_per_item holds minus the multiple of the default K rule.
bool tuned_lookup(int mode, int d, int n_h, int64_t n, kde_opts* out);

// Batch machinery shared with the autotuner and the LSCV_H minimiser (batch.cu).
int batch_run(kde_batch_plan* p, void* ws, size_t ws_bytes, cudaStream_t st, bool use_graph);
void batch_free(kde_batch_plan* p);
int lscv_H_eval(kde_batch_plan** plan, bool keep, const void* x_dev, int dtype, int64_t n, int d,
                const double* H, int m, const kde_opts* opts, void* ws, size_t ws_bytes, cudaStream_t st,
                double* g_host);

}  // namespace gbkde
