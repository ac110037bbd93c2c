// Internal declarations shared by the CUDA translation units of libgbkde.
// Device descriptors, the triangular tile map, and small device helpers.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "gbkde.h"

namespace gbkde {

constexpr int kThreads = 256;  // threads per CTA of every pair kernel (8 warps)
constexpr int kWarps = kThreads / 32;
constexpr int kPadTo = 512;    // sample arrays are zero-padded to a multiple of this (the largest tile edge)

// Per-dataset descriptor, resident in device memory for the whole selection.
// Host code fills the geometry; the prologue kernel fills the statistics; the
// finishing kernels fill `res`.
struct DsDev {
  // ---- input
  const void* x;    // d x n samples, row-major (coordinate-major)
  int64_t n;
  int32_t d;
  int32_t dtype;    // KDE_F32 / KDE_F64
  int64_t n_pad;    // n rounded up to kPadTo
  int32_t methods;  // KDE_METHOD_* bits to run
  int32_t given_H;  // 1: whiten by the matrix in cov[] (LSCV_H) instead of the sample covariance
  int32_t dk;       // coordinates of y the pair kernel walks: d, or d rounded up to 8/12/16 (zeros)
  int32_t cv_loo;   // 1: exact leave-one-out weights in g(h) (KDE_CV_LOO)
  // ---- prepared samples
  float* y;   // [d][n_pad]  sqrt(log2(e)/4) L^-1 (x - mean), zero padded   (LSCV)
  float* xc;  // [n_pad]     x - mean, zero padded                           (d = 1)
  // ---- LSCV geometry
  int32_t n_h, n_h_pad;    // grid size and size padded to a multiple of B
  int32_t n_chunks;        // n_h_pad / B
  int32_t n_groups;        // ceil(n_chunks / kWarps): one CTA item covers one group
  int32_t lscv_tile;       // T
  int32_t lscv_K;          // tiles per item
  int64_t lscv_tiles;      // end of the tile range walked (NT (NT+1)/2 for a full selection)
  int64_t lscv_rows;       // ceil((lscv_tiles - lscv_t0) / lscv_K)
  int64_t lscv_t0;         // first tile of the range walked (0 for a full selection)
  double* h;               // [n_h]   bandwidth multipliers
  float* nc;               // [n_h_pad] -1/h^2 (padded entries -1)
  double* lscv_part;       // [lscv_rows][2 n_h_pad] per-item (S1, S2) partials
  double* lscv_sum;        // [2 n_h_pad] reduced (S1, S2)
  double* g;               // [n_h] objective
  // ---- psi geometry
  int32_t psi_tile;
  int32_t psi_K;
  int64_t psi_tiles;
  int64_t psi_rows;
  int64_t psi_t0;
  double* psi_part;        // [psi_rows]
  float psi_scale;         // sqrt(log2(e)/2) / g for the pilot g of the running phase
  int32_t prep_parts;      // CTAs of the prologue: the samples are cut into this many ranges
  double* prep_part;       // [prep_parts][kPrepRecord] per-range count, mean, centred moments
  uint32_t prep_count;     // ranges finished (the last CTA combines them and resets it to 0)
  uint32_t pair_count;     // CTAs of a fused pair-kernel launch finished (the last one finishes)
  uint32_t reduce_count;   // column strips of the LSCV reduction finished (the last one finishes)
  uint32_t strip_count[2 * KDE_MAX_NH / 32];  // row chunks of each strip finished
  int32_t oct_P;           // > 0: the grid is P points per octave of 1/h^2 (octave kernel)
  // ---- statistics (written on the device)
  double mean[KDE_MAX_D];
  double cov[KDE_MAX_D * KDE_MAX_D];
  double logdet;
  double sigma;
  double A;                // (4 pi)^(-d/2) |S|^(-1/2)
  double c_A;              // (4 pi)^(-d/2), from the host
  double c_g1;             // g1 / sigma of the PLUGIN pilot, (-2 K6(0) 32 sqrt(pi) / (105 n))^(1/9), from the host
  float M[KDE_MAX_D * KDE_MAX_D];  // sqrt(log2(e)/4) L^-1, row-major, lower triangular
  kde_result res;
};

// One launch of a pair kernel walks the items of several datasets:
// item k belongs to dataset i with off[i] <= k < off[i+1].
struct Phase {
  DsDev* ds;
  const int64_t* off;
  const int64_t* base;  // optional: first local item of each dataset in this launch
  int32_t n_ds;
  int32_t fuse;         // 0: finishing kernels follow; else (one dataset) the CTA that
                        // finishes last reduces the partials and finishes: LSCV 1, psi r
  int64_t total;
};

// Horner coefficients of the psi kernel polynomial (see psi kernels).
// The monic polynomial p_r(y) of degree M = r/2 in shifted form: with
// w = y + shift (shift = one M-th of p's y^(M-1) coefficient, so that w^(M-1)
// drops out), p_r(y) = q(w) = ((w w + c0) w + c1) w ... (M - 1 coefficients),
// and p_r(y) 2^-y = post * q(w) 2^-w with post = 2^shift.
struct PsiCoef {
  float c[4];
  float shift;
  double post;
};

// Tile map of the upper pair triangle (Sec. 5.4.2, Eqs. colInTriangleMatrix,
// rowInTriangleMatrix; Appendix A): column l holds the l+1 tiles numbered
// l(l+1)/2 .. l(l+1)/2 + l, row q = bx - l(l+1)/2.  The single-precision
// square root can land one column off for large bx; an exact integer
// correction follows.
__host__ __device__ inline void tile_coords(int64_t bx, int64_t& l, int64_t& q) {
  float s = sqrtf(8.0f * (float)bx + 9.0f);
  int64_t L = (int64_t)ceilf((s - 3.0f) * 0.5f);
  if (L < 0) L = 0;
  while (L > 0 && L * (L + 1) / 2 > bx) --L;
  while ((L + 1) * (L + 2) / 2 <= bx) ++L;
  l = L;
  q = bx - L * (L + 1) / 2;
}

// Role of warp `warp` of an LSCV CTA when its item's bandwidth group has
// cg (1..8) chunks of B bandwidths: the chunk it evaluates and the slice of
// the tile's columns it walks.  S = kWarps / cg slices per chunk, so
// S * cg <= kWarps; warps with slice >= S idle.
// Pair-kernel shapes whose items are walked by single warps (k_lscv_warp):
// wide samples (d > 4, padded to 8/12/16 coordinates) with 2 bandwidths per
// thread (grids of one or two points).  The geometry sizes their items for
// 8 times as many workers.
__host__ __device__ constexpr bool lscv_warp_items(int dk, int B) { return dk > 4 && B == 2; }

struct WarpRole {
  int chunk, slice, S;
  bool active;
};
__host__ __device__ inline WarpRole warp_role(int warp, int cg) {
  WarpRole r;
  r.S = kWarps / cg;
  r.chunk = warp % cg;
  r.slice = warp / cg;
  r.active = r.slice < r.S;
  return r;
}

__host__ __device__ inline int64_t tri_tiles(int64_t n, int tile) {
  int64_t nt = (n + tile - 1) / tile;
  return nt * (nt + 1) / 2;
}

#ifdef __CUDACC__
// 2^a by the MUFU unit (PTX ex2.approx.ftz.f32).
__device__ __forceinline__ float ex2(float a) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
  return r;
}

// 2^-a: the negation sits in the same asm block as the ex2, so that it can
// be taken as an operand modifier of the MUFU instruction instead of costing
// a separate FP32 instruction.
__device__ __forceinline__ float ex2_neg(float a) {
  float r;
  asm("{\n\t.reg .f32 t;\n\tneg.f32 t, %1;\n\tex2.approx.ftz.f32 %0, t;\n\t}" : "=f"(r) : "f"(a));
  return r;
}

// Kahan compensated update of (s, c) by v; the running total is s - c.
__device__ __forceinline__ void kahan_add(float& s, float& c, float v) {
  float y = v - c;
  float t = s + y;
  c = (t - s) - y;
  s = t;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Warp sum of values hi + lo carried as FP32 pairs (double-float): at every
// butterfly step the two heads are added by Knuth's TwoSum, whose rounding
// error joins the tails, and the pair is renormalised by Dekker's Fast2Sum.
// The result carries about 44 bits; FP32 arithmetic only, since the FP64
// pipe of this part runs at a small fraction of the FP32 rate.  Every lane
// ends with the same pair (each step is symmetric in its two operands).
// (hi, lo) += (h2, l2) in double-float arithmetic: Knuth's TwoSum of the
// high parts, the low parts and the rounding error added, then renormalised.
__device__ __forceinline__ void ff_add(float& hi, float& lo, float h2, float l2) {
  const float s = __fadd_rn(hi, h2);
  const float bb = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(h2, bb));
  const float t = __fadd_rn(__fadd_rn(lo, l2), e);
  hi = __fadd_rn(s, t);
  lo = __fsub_rn(t, __fsub_rn(hi, s));
}

__device__ __forceinline__ float2 warp_sum_ff(float hi, float lo) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
    const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
    ff_add(hi, lo, h2, l2);
  }
  return make_float2(hi, lo);
}

// Warp totals of nsum double-float values per lane held in shared memory as
// Kahan pairs: sum q of lane L is (v.x, -v.y) (q even) or (v.z, -v.w) (q odd)
// of v = slots[(q >> 1) * 32 + L].  One lane adds each sum over the 32 lanes
// (for nsum <= 16, two lanes over 16 lanes each, then the upper half into the
// lower), in double-float arithmetic, starting at lane q and wrapping around
// (a fixed order per sum; staggered starts keep the concurrent shared-memory
// reads on different banks).  Lane q (< nsum) returns the total of sum q.
// Far fewer instructions than nsum butterflies.
__device__ __forceinline__ float2 warp_sums_ff_transposed(const float4* slots, int nsum, int lane) {
  const bool two = nsum <= 16;
  const int q = two ? (lane & 15) : lane;
  const int base = two ? (lane >> 4) * 16 : 0;
  const int cnt = two ? 16 : 32;
  float hi = 0.f, lo = 0.f;
  if (q < nsum) {
    const float4* v = slots + (q >> 1) * 32 + base;
    for (int i = 0; i < cnt; ++i) {
      const float4 k = v[(i + q) & (cnt - 1)];
      if (q & 1)
        ff_add(hi, lo, k.z, -k.w);
      else
        ff_add(hi, lo, k.x, -k.y);
    }
  }
  if (two) {
    const float h2 = __shfl_xor_sync(0xffffffffu, hi, 16);
    const float l2 = __shfl_xor_sync(0xffffffffu, lo, 16);
    if (lane < 16) ff_add(hi, lo, h2, l2);
  }
  return make_float2(hi, lo);
}

__device__ __forceinline__ double ff_value(float2 p) { return (double)p.x + (double)p.y; }

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Holds a kernel launched with programmatic stream serialisation until the
// kernel before it in the stream has completed and its writes are visible
// (PTX griddepcontrol.wait).  Every kernel that single selections launch
// calls it first, before touching global memory; launched the plain way
// (batches, the server, graph replays), it returns at once.
__device__ __forceinline__ void dependent_launch_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// w^K for a small positive integer K by squarings (K = 7: w^2, w^3, w^6, w^7).
template <int K>
__device__ __forceinline__ double ipow(double w) {
  if constexpr (K == 1)
    return w;
  else if constexpr (K % 2 == 0) {
    const double s = ipow<K / 2>(w);
    return s * s;
  } else {
    return ipow<K - 1>(w) * w;
  }
}

// y = x^(1/K) and its reciprocal for a normal x > 0, in FP64 without pow,
// exp or log (each a long FP64 sequence on this part, whose FP64 unit runs at
// a small fraction of the FP32 rate; a dependent FP64 operation costs about
// 45 clocks).  With x = m 2^(K q), m in [1, 2^K) (an exact exponent split),
// Newton's method for f(w) = w^-K - m, whose step w <- w + w (1 - m w^K) / K
// needs no division, converges quadratically to w = m^(-1/K).  The seed
// 2^(-log2(m) / K) comes from the FP32 MUFU log2 and exp2 (about 20 correct
// bits), so two steps reach FP64 rounding; then m^(1/K) = m w^(K-1) and both
// results are scaled by 2^(+-q).  Other x (zero, negative, subnormal,
// infinite, NaN) take the library pow.
template <int K>
__device__ __forceinline__ double root_newton(double x, double* inv) {
  static_assert(K >= 2 && K <= 9, "small integer roots");
  if (!(x >= 2.2250738585072014e-308 && x <= 1.7976931348623157e308)) {
    const double y = pow(x, 1.0 / K);
    *inv = 1.0 / y;
    return y;
  }
  const long long bits = __double_as_longlong(x);
  const int e = (int)((bits >> 52) & 0x7ff) - 1023;
  int q = e / K, r = e - q * K;
  if (r < 0) {
    r += K;
    --q;
  }
  const double m = __longlong_as_double((bits & 0x000fffffffffffffLL) | ((long long)(1023 + r) << 52));
  float l2, s;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l2) : "f"((float)m));
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(s) : "f"(l2 * (-1.0f / K)));
  double w = (double)s;
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const double t = fma(-m, ipow<K>(w), 1.0);
    w = fma(w * t, 1.0 / K, w);
  }
  const double y = m * ipow<K - 1>(w);
  *inv = w * __longlong_as_double((long long)(1023 - q) << 52);  // |q| <= 511
  return y * __longlong_as_double((long long)(1023 + q) << 52);
}

// Index of the dataset owning global item `it` (largest i with off[i] <= it).
__device__ __forceinline__ int find_ds(const int64_t* off, int n, int64_t it) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= it)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}
#endif

// Prologue ranges: at most 128, about 1,024 samples each; per range one
// record of kPrepRecord doubles: count, mean[KDE_MAX_D], the centre the
// moments were taken about[KDE_MAX_D], centred moments[kNPairs].
constexpr int kNPairs = KDE_MAX_D * (KDE_MAX_D + 1) / 2;  // covariance entries a <= b
constexpr int kPrepRecord = 1 + 2 * KDE_MAX_D + kNPairs;
inline int prep_parts_for(int64_t n) {
  const int64_t p = (n + 1023) / 1024;
  return (int)(p < 1 ? 1 : (p > 128 ? 128 : p));
}

// ------------------------------------------------------------- launchers
// Programmatic dependent launch for the short launch sequences of single
// selections: while a DependentLaunchScope lives on the calling thread,
// launch_kernel asks for programmatic stream serialisation, so that a
// kernel's CTAs are scheduled while the kernel before it drains (each such
// kernel waits in dependent_launch_wait before touching global memory).
// Measured on this part: about 2.3 us less per kernel boundary.
extern thread_local bool t_dependent_launch;
struct DependentLaunchScope {
  bool prev;
  DependentLaunchScope() : prev(t_dependent_launch) { t_dependent_launch = true; }
  ~DependentLaunchScope() { t_dependent_launch = prev; }
  DependentLaunchScope(const DependentLaunchScope&) = delete;
  DependentLaunchScope& operator=(const DependentLaunchScope&) = delete;
};

template <typename... P, typename... A>
cudaError_t launch_kernel(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                          A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = t_dependent_launch ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<P>(args)...);
}

// (defined in the .cu files; return a cudaError_t)
// ids: optional list of dataset indices into ds (one CTA each); NULL = ds[0..n_ds)
// parts_max: the largest prep_parts among the datasets launched
cudaError_t launch_prep(DsDev* ds, int n_ds, const int* ids, int parts_max, cudaStream_t st);
// oct: the octave-grid variant (B = 16; every dataset of the phase has oct_P > 0)
cudaError_t launch_lscv(const Phase& ph, int d, int B, int R, bool kahan, bool oct, int grid,
                        cudaStream_t st);
size_t lscv_smem_bytes(int d, int B, int R, bool kahan, bool oct);
// sets the kernel's shared-memory attribute without launching (call before a graph capture)
cudaError_t prepare_lscv(int d, int B, int R, bool kahan, bool oct);
// Reduction of the LSCV item rows and the finish (g(h), argmin) of n_ds
// datasets: rows_max = the largest lscv_rows among them.
cudaError_t launch_lscv_reduce(DsDev* ds, int n_ds, const int* ids, int n_h_pad_max, int64_t rows_max,
                               cudaStream_t st);
cudaError_t launch_psi(const Phase& ph, int r, int R, bool kahan, const PsiCoef& cf, int grid,
                       cudaStream_t st);
// stage: 6 -> reduce psi_6, set g2; 4 -> reduce psi_4, set h; 0 -> raw sum only (into res.g_min)
cudaError_t launch_psi_finish(DsDev* ds, int n_ds, const int* ids, int stage, int r, cudaStream_t st);
// Descriptor setup and prologue of one dataset: one launch when its prologue
// is a single range, else launch_setup then launch_prep.
cudaError_t launch_setup_prep(DsDev* dst, const DsDev& init, const double* h, int n_h, int64_t* off_dst,
                              const int64_t* off_src, int n_off, cudaStream_t st);
cudaError_t launch_setup(DsDev* dst, const DsDev& init, const double* h, int n_h,
                         int64_t* off_dst, const int64_t* off_src, int n_off, cudaStream_t st);
cudaError_t launch_probe_mode(int mode, double* out, int iters, int grid, cudaStream_t st);

}  // namespace gbkde
