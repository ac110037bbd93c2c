// All-pairs kernel of the plug-in functionals psi_r (Sec. 4.4.1,
// Eqs. PLUGIN-Psi6Estimate, PLUGIN-Psi4Estimate) and the device-side scalar
// chain of the PLUGIN method (steps 5-8).
//
// With z = x sqrt(log2 e / 2) / g and y = (z_i - z_j)^2 we have
// u^2 = ((x_i - x_j)/g)^2 = kappa y (kappa = 2 ln 2) and exp(-u^2/2) = 2^-y, so
// K^(r)(u) = He_r(u) phi(u) = kappa^(r/2) p_r(y) 2^-y / sqrt(2 pi), where p_r is
// He_r rewritten in y and made monic (host code derives its coefficients from
// the Hermite recurrence).  The kernel sums q(w) 2^-w over pairs, where
// w = y + shift removes the y^(r/2 - 1) term of p_r (so p_r(y) 2^-y =
// 2^shift q(w) 2^-w, the constant applied in FP64 by the finish): per pair one
// subtraction, one FMA for w, one ex2, r/2 - 1 Horner FMAs in w (Sec. 7.1
// uses Horner's rule as well) and one accumulating FMA, packed two rows at a
// time in FP32x2 -- r/2 + 2 FP32 lane-operations per pair.
//
// Schedule: T x T tiles of the pair triangle in the numbering of Sec. 5.4.2;
// items of K consecutive tiles; persistent CTAs of 8 warps in RG row groups
// of 32 R rows (R per lane, in registers), T = 32 R RG; each warp covers its
// group's rows against a slice of RG T / 8 columns staged in shared memory.
// Two row groups (T = 512) give each warp four times the pairs per tile of
// one (T = 256), so the per-tile work (row loads, scaling, Kahan fold, tile
// bookkeeping) is spread over more evaluations.  Per-lane FP32 runs over a
// tile are folded into a Kahan pair; item totals are reduced in FP64 and
// written to a per-item slot.
#include "host.hpp"
#include "internal.cuh"

namespace gbkde {

namespace {

constexpr double kSqrtHalfLog2e = 0.8493218002880191;  // sqrt(log2(e) / 2) in FP64
constexpr double kRK = 0.28209479177387814;  // R(K) = 1 / (2 sqrt(pi)) of the Gaussian kernel, FP64

// Columns [j_lo, j_hi) of one tile for this lane's R rows, CPI columns per
// iteration.  Edge tiles mask by tile-local 32-bit indices: row il0 + 64 p
// (+ 32 for the second of a packed pair) and column jj + c, kept when
// il < jl < jlim.  il0 is the lane's first row relative to the column tile
// (negative for tiles off the diagonal, whose rows all precede their
// columns) and jlim the number of real columns of the tile.
template <int RD, int R, int CPI, bool EDGE>
__device__ __forceinline__ void psi_columns(const float* __restrict__ sF, int j_lo, int j_hi,
                                            const float2 (&z)[R / 2], float2 (&acc)[R / 2],
                                            const PsiCoef& cf, int il0, int jlim) {
  constexpr int M = RD / 2;
  float2 cc[M - 1];
#pragma unroll
  for (int m = 0; m < M - 1; ++m) cc[m] = make_float2(cf.c[m], cf.c[m]);
  const float2 sh2 = make_float2(cf.shift, cf.shift);
  // sF holds each column sample as the pair (-v, -v): two columns per 16 bytes
#pragma unroll 1
  for (int jj = j_lo; jj < j_hi; jj += CPI) {
    float2 nfs[CPI];
#pragma unroll
    for (int u = 0; u < CPI / 2; ++u) {
      const float4 v = *reinterpret_cast<const float4*>(sF + 2 * jj + 4 * u);
      nfs[2 * u] = make_float2(v.x, v.y);
      nfs[2 * u + 1] = make_float2(v.z, v.w);
    }
#pragma unroll
    for (int c = 0; c < CPI; ++c) {
      const float2 nf = nfs[c];
#pragma unroll
      for (int p = 0; p < R / 2; ++p) {
        const float2 dl = __fadd2_rn(z[p], nf);
        const float2 w = __ffma2_rn(dl, dl, sh2);  // y + shift
        float2 e = make_float2(ex2_neg(w.x), ex2_neg(w.y));
        if (EDGE) {
          const int il = il0 + 64 * p, jl = jj + c;
          if (!(il < jl && jl < jlim)) e.x = 0.f;
          if (!(il + 32 < jl && jl < jlim)) e.y = 0.f;
        }
        float2 q = __ffma2_rn(w, w, cc[0]);
#pragma unroll
        for (int m = 1; m < M - 1; ++m) q = __ffma2_rn(q, w, cc[m]);
        acc[p] = __ffma2_rn(q, e, acc[p]);
      }
    }
  }
}

__device__ void psi_finish_body(DsDev* ds, int stage, int r, double post);

// Fused single-dataset launches: the CTA that finishes last (a counter in the
// descriptor; no CTA waits) reduces the item partials and advances the chain
// with the code and order of k_psi_finish, so results are bitwise the same.
__device__ __noinline__ void psi_fused_finish(const Phase& ph, int r, double post) {
  __shared__ int sLast;
  DsDev* ds = ph.ds;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) sLast = atomicAdd(&ds->pair_count, 1u) == gridDim.x - 1u;
  __syncthreads();
  if (!sLast) return;
  __threadfence();
  psi_finish_body(ds, ph.fuse, r, post);
  if (threadIdx.x == 0) ds->pair_count = 0u;
}

template <int RD, int R, int RG, bool KAHAN>
__global__ void __launch_bounds__(kThreads, 2) k_psi(Phase ph, PsiCoef cf) {
  dependent_launch_wait();
  constexpr int T = 32 * R * RG;
  constexpr int SL = kWarps / RG;     // column slices per tile
  constexpr int CPI = R >= 8 ? 8 : 4;  // columns per inner iteration
  static_assert(kWarps % RG == 0 && (T / SL) % CPI == 0, "psi warp layout");
  __shared__ __align__(16) float sF[2 * T];  // (-v, -v) per column
  __shared__ double sRed[kWarps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rg = warp / SL;
  constexpr int cols = T / SL;
  const int j_lo = (warp % SL) * cols, j_hi = j_lo + cols;
  const int r0 = rg * 32 * R + lane;  // the lane's first row within a tile

  for (int64_t it = blockIdx.x; it < ph.total; it += gridDim.x) {
    const int di = find_ds(ph.off, ph.n_ds, it);
    const DsDev* ds = ph.ds + di;
    if (ds->res.status != KDE_OK) continue;
    const int64_t row = it - ph.off[di] + (ph.base ? ph.base[di] : 0);
    const int64_t t0 = ds->psi_t0 + row * ds->psi_K;
    const int64_t t1 = min(t0 + (int64_t)ds->psi_K, ds->psi_tiles);
    const int64_t n = ds->n;
    const float sc = ds->psi_scale;
    const float* __restrict__ X = ds->xc;
    float s = 0.f, c = 0.f;
    float2 acc[R / 2];
#pragma unroll
    for (int p = 0; p < R / 2; ++p) acc[p] = make_float2(0.f, 0.f);
    int64_t l, q;
    tile_coords(t0, l, q);
    int64_t l_loaded = -1;
    // row samples of the current tile; those of the next tile are loaded
    // before the current one is evaluated (a tile is only ~6k clocks of work,
    // so an exposed global-load latency per tile would cost ~10 %)
    float zr[R];
#pragma unroll
    for (int k = 0; k < R; ++k) zr[k] = X[q * T + r0 + 32 * k];
    for (int64_t t = t0; t < t1; ++t) {
      if (l != l_loaded) {
        __syncthreads();
        for (int jj = threadIdx.x; jj < T; jj += kThreads) {
          const float v = X[l * T + jj] * sc;
          reinterpret_cast<float2*>(sF)[jj] = make_float2(-v, -v);
        }
        __syncthreads();
        l_loaded = l;
      }
      float2 z[R / 2];
#pragma unroll
      for (int p = 0; p < R / 2; ++p) z[p] = make_float2(zr[2 * p] * sc, zr[2 * p + 1] * sc);
      {
        const int64_t qn = (q + 1 > l) ? 0 : q + 1;
        if (t + 1 < t1) {
#pragma unroll
          for (int k = 0; k < R; ++k) zr[k] = X[qn * T + r0 + 32 * k];
        }
      }
      const bool edge = (q == l) || ((l + 1) * T > n);
      if (edge) {
        const int il0 = (q == l) ? r0 : -(1 << 30);
        const int jlim = (int)min((int64_t)T, n - l * T);
        psi_columns<RD, R, CPI, true>(sF, j_lo, j_hi, z, acc, cf, il0, jlim);
      } else {
        psi_columns<RD, R, CPI, false>(sF, j_lo, j_hi, z, acc, cf, 0, 0);
      }
      if (KAHAN) {
        float run = 0.f;
#pragma unroll
        for (int p = 0; p < R / 2; ++p) {
          run += acc[p].x + acc[p].y;
          acc[p] = make_float2(0.f, 0.f);
        }
        kahan_add(s, c, run);
      }
      if (++q > l) {
        ++l;
        q = 0;
      }
    }
    float vh, vl;  // the lane's total as a double-float pair
    if (KAHAN) {
      vh = s, vl = -c;
    } else {
      float run = 0.f;
#pragma unroll
      for (int p = 0; p < R / 2; ++p) run += acc[p].x + acc[p].y;
      vh = run, vl = 0.f;
    }
    const float2 v = warp_sum_ff(vh, vl);
    __syncthreads();
    if (lane == 0) sRed[warp] = ff_value(v);
    __syncthreads();
    if (threadIdx.x == 0) {
      double tot = 0.0;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) tot += sRed[w];
      ds->psi_part[row] = tot;
    }
  }
  if (ph.fuse) psi_fused_finish(ph, RD, cf.post);
}

// Reduce the per-item psi partials in a fixed order and advance the PLUGIN
// chain on the device in FP64.
//   stage 6: psi_6(g1) (Eq. PLUGIN-Psi6Estimate, reading R1), then g2
//            (Eq. PLUGIN-g2) and the psi_4 sample scale;
//   stage 4: psi_4(g2) (Eq. PLUGIN-Psi4Estimate, reading R1), then h
//            (Eq. PLUGIN-Final_h);
//   stage 0: raw pair sum only (psi tile-sum entry point), into res.g_min.
__device__ void psi_finish_body(DsDev* ds, int stage, int r, double post) {
  __shared__ double sRed[kWarps];
  if (ds->res.status != KDE_OK) return;
  if (stage != 0 && !(ds->methods & KDE_METHOD_PLUGIN)) return;
  double acc = 0.0;
  for (int64_t k = threadIdx.x; k < ds->psi_rows; k += kThreads) acc += __ldcg(ds->psi_part + k);
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sRed[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x != 0) return;
  double P = 0.0;
  for (int w = 0; w < kWarps; ++w) P += sRed[w];
  P *= post;  // sum of p_r(y) 2^-y from the kernel's sum of q(w) 2^-w
  const double kappa = 2.0 * 0.69314718055994530942;
  const double inv_sqrt_2pi = 0.39894228040143267794;
  // sum_{i<j} K^(r)((x_i - x_j)/g) = kappa^(r/2) P / sqrt(2 pi); integer
  // powers by multiplication and the two real roots of the chain by
  // root_newton (FP64 pow is a long sequence on this part: about 5,800
  // clocks against 1,100).  The root's argument is formed from the same
  // numerator and denominator as psi_r, so that its division does not wait
  // for psi_r's.
  double kr = 1.0;
  for (int m = 0; m < r / 2; ++m) kr *= kappa;
  const double sumK = kr * P * inv_sqrt_2pi;
  kde_result& res = ds->res;
  if (stage == 0) {
    res.g_min = sumK;
    return;
  }
  const double n = (double)ds->n;
  if (stage == 6) {
    const double k6_0 = -15.0 * inv_sqrt_2pi;  // K^(6)(0), Eq. PLUGIN-g1
    const double k4_0 = 3.0 * inv_sqrt_2pi;    // K^(4)(0), Eq. PLUGIN-g2
    const double g1 = res.g1;
    const double g1s = g1 * g1, g1q = g1s * g1s;
    const double num = 2.0 * sumK + n * k6_0, den = n * n * (g1q * g1s * g1);
    const double psi6 = num / den;
    // g2 = (-2 K4(0) / (psi6 n))^(1/7)
    const double arg = -2.0 * k4_0 * den / (num * n);
    res.psi6 = psi6;
    if (!(psi6 < 0.0)) {
      res.status = KDE_EDEGENERATE;
      return;
    }
    double inv_g2;
    const double g2 = root_newton<7>(arg, &inv_g2);
    res.g2 = g2;
    ds->psi_scale = (float)(kSqrtHalfLog2e * inv_g2);
  } else {
    const double k4_0 = 3.0 * inv_sqrt_2pi;
    const double g2 = res.g2;
    const double g2s = g2 * g2;
    const double num = 2.0 * sumK + n * k4_0, den = n * n * (g2s * g2s * g2);
    const double psi4 = num / den;
    // h = (R(K) / (psi4 n))^(1/5), R(K) = 1 / (2 sqrt(pi)) (Eq. PLUGIN-Final_h)
    const double arg = kRK * den / (num * n);
    res.psi4 = psi4;
    if (!(psi4 > 0.0)) {
      res.status = KDE_EDEGENERATE;
      return;
    }
    double inv_h;
    const double h = root_newton<5>(arg, &inv_h);
    res.h_plugin = h;
    if (!(ds->methods & KDE_METHOD_LSCV)) {  // otherwise h / h_data hold the LSCV choice
      res.h = h;
      res.h_data = h;
    }
  }
}

__global__ void __launch_bounds__(kThreads) k_psi_finish(DsDev* dsa, const int* ids, int stage, int r,
                                                         double post) {
  dependent_launch_wait();
  DsDev* ds = dsa + (ids ? ids[blockIdx.x] : (int)blockIdx.x);
  psi_finish_body(ds, stage, r, post);
}

template <int RD, int R, int RG>
cudaError_t launch_k(const Phase& ph, bool kahan, const PsiCoef& cf, int grid, cudaStream_t st) {
  if (kahan) return launch_kernel(k_psi<RD, R, RG, true>, dim3(grid), dim3(kThreads), 0, st, ph, cf);
  return launch_kernel(k_psi<RD, R, RG, false>, dim3(grid), dim3(kThreads), 0, st, ph, cf);
}

// Rp = T / 32: 2 (T = 64), 8 (T = 256) or 16 (T = 512: two row groups of 8
// rows per lane).
template <int RD>
cudaError_t launch_r(const Phase& ph, int Rp, bool kahan, const PsiCoef& cf, int grid,
                     cudaStream_t st) {
  switch (Rp) {
    case 2: return launch_k<RD, 2, 1>(ph, kahan, cf, grid, st);
    case 8: return launch_k<RD, 8, 1>(ph, kahan, cf, grid, st);
    case 16: return launch_k<RD, 8, 2>(ph, kahan, cf, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_psi(const Phase& ph, int r, int R, bool kahan, const PsiCoef& cf, int grid,
                       cudaStream_t st) {
  if (ph.total <= 0) return cudaSuccess;
  switch (r) {
    case 4: return launch_r<4>(ph, R, kahan, cf, grid, st);
    case 6: return launch_r<6>(ph, R, kahan, cf, grid, st);
    case 8: return launch_r<8>(ph, R, kahan, cf, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_psi_finish(DsDev* ds, int n_ds, const int* ids, int stage, int r, cudaStream_t st) {
  if (n_ds <= 0) return cudaSuccess;
  return launch_kernel(k_psi_finish, dim3(n_ds), dim3(kThreads), 0, st, ds, ids, stage, r, psi_coef(r).post);
}

}  // namespace gbkde
