// Prologue kernels: descriptor setup, sample statistics, Cholesky whitening
// and the first links of the PLUGIN chain; plus the ALU throughput probe.
#include "internal.cuh"

namespace gbkde {

namespace {

constexpr double kLog2e = 1.4426950408889634074;
constexpr double kPi = 3.14159265358979323846;
constexpr int kPrepThreads = 512;

struct SetupParams {
  DsDev init;
  int64_t off[4];
  int32_t n_off;
  int32_t n_h;
  double h[KDE_MAX_NH];
};

// Copies the host-built descriptor into device memory and expands the grid:
// h[k] and nc[k] = -1/h_k^2 (padded chunk entries get -1).
__global__ void k_setup(DsDev* dst, int64_t* off_dst, SetupParams p) {
  if (threadIdx.x == 0) *dst = p.init;
  if (threadIdx.x < p.n_off) off_dst[threadIdx.x] = p.off[threadIdx.x];
  for (int k = threadIdx.x; k < p.init.n_h_pad; k += blockDim.x) {
    if (k < p.n_h) {
      p.init.h[k] = p.h[k];
      p.init.nc[k] = (float)(-1.0 / (p.h[k] * p.h[k]));
    } else {
      p.init.nc[k] = -1.0f;
    }
  }
}

// Per-thread accumulator: FP32 with Kahan compensation for FP32 input
// (per-thread sums in FP32), FP64 for FP64 input.
template <typename TIN>
struct Acc;
template <>
struct Acc<float> {
  float s = 0.f, c = 0.f;
  __device__ void add(float v) { kahan_add(s, c, v); }
  __device__ double get() const { return (double)s - (double)c; }
};
template <>
struct Acc<double> {
  double s = 0.0;
  __device__ void add(double v) { s += v; }
  __device__ double get() const { return s; }
};

// Block-wide FP64 sum of `cnt` values per thread, deterministic order;
// results land in out[0..cnt) (shared memory) for every thread.
constexpr int kNPairs = KDE_MAX_D * (KDE_MAX_D + 1) / 2;  // covariance entries a <= b

__device__ void block_sum(double* v, int cnt, double (*scratch)[kNPairs], double* out) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = 0; k < cnt; ++k) {
    double s = warp_sum(v[k]);
    if (lane == 0) scratch[warp][k] = s;
  }
  __syncthreads();
  if (threadIdx.x < cnt) {
    double t = 0.0;
    for (int w = 0; w < kPrepThreads / 32; ++w) t += scratch[w][threadIdx.x];
    out[threadIdx.x] = t;
  }
  __syncthreads();
}

// Shared memory of the prologue, declared once in the kernel for every
// (element type, dimension) instance.
struct PrepSmem {
  double scratch[kPrepThreads / 32][kNPairs];
  double sv[kNPairs];
  double sMean[KDE_MAX_D];
  float sM[KDE_MAX_D * KDE_MAX_D];
  float sMeanF[KDE_MAX_D];
  int sOk;
  // centred samples of the pair-parallel covariance pass (D >= 8)
  alignas(16) unsigned char stage[16384];
};

// samples per thread whose loads are issued together (wide samples already
// issue D independent loads per sample)
template <int D>
constexpr int kPrepBatch = D >= 8 ? 1 : 4;

// One CTA per dataset, D = the dataset's kernel dimension (d <= D; coordinates
// d..D-1 are absent).  Pass 1: mean (Eq. LSCV-covariance / PLUGIN-
// VarianceEstimator evaluated two-pass, reading R7).  Pass 2: covariance with
// the n-1 denominator.  Then, on one thread in FP64: Cholesky S = L L^T,
// log|S|, the whitening matrix M = sqrt(log2 e / 4) L^-1, sigma, A and, for
// the PLUGIN method, psi_8^NS (Eq. PLUGIN-Psi8Estimate) and g1
// (Eq. PLUGIN-g1).  Pass 3: y = M (x - mean) and x - mean in FP32.
// Every thread walks samples tid, tid + 512, ... in order; loads are issued
// kPrepBatch samples at a time.  For D >= 8 the covariance is pair-parallel:
// blocks of centred samples are staged in shared memory and thread t adds
// pair t mod P (P = d(d+1)/2) over every G-th sample of the block.
template <typename TIN, int D>
__device__ __forceinline__ void prep_body(DsDev* ds, PrepSmem& sm) {
  double(*scratch)[kNPairs] = sm.scratch;
  double* sv = sm.sv;
  float* sM = sm.sM;
  float* sMeanF = sm.sMeanF;
  double* sMean = sm.sMean;
  int& sOk = sm.sOk;
  const TIN* __restrict__ x = static_cast<const TIN*>(ds->x);
  const int64_t n = ds->n, n_pad = ds->n_pad;
  const int d = ds->d;

  // ---- pass 1: mean
  {
    Acc<TIN> a1[D];
    for (int64_t i0 = threadIdx.x; i0 < n; i0 += (int64_t)kPrepThreads * kPrepBatch<D>) {
      TIN v[kPrepBatch<D>][D];
#pragma unroll
      for (int u = 0; u < kPrepBatch<D>; ++u) {
        const int64_t i = i0 + (int64_t)u * kPrepThreads;
#pragma unroll
        for (int k = 0; k < D; ++k) v[u][k] = (i < n && k < d) ? x[(int64_t)k * n + i] : TIN(0);
      }
#pragma unroll
      for (int u = 0; u < kPrepBatch<D>; ++u)
        if (i0 + (int64_t)u * kPrepThreads < n) {
#pragma unroll
          for (int k = 0; k < D; ++k)
            if (k < d) a1[k].add(v[u][k]);
        }
    }
    double v[D];
#pragma unroll
    for (int k = 0; k < D; ++k) v[k] = a1[k].get();
    block_sum(v, d, scratch, sv);
  }
  if (threadIdx.x < d) {
    sMean[threadIdx.x] = sv[threadIdx.x] / (double)n;
    sMeanF[threadIdx.x] = (float)sMean[threadIdx.x];
  }
  __syncthreads();

  // ---- pass 2: centred cross products, upper triangle a <= b
  const int npairs = d * (d + 1) / 2;
  if constexpr (D <= 4) {
    constexpr int NP = D * (D + 1) / 2;
    Acc<TIN> a2[NP];
    for (int64_t i0 = threadIdx.x; i0 < n; i0 += (int64_t)kPrepThreads * kPrepBatch<D>) {
      TIN c[kPrepBatch<D>][D];
#pragma unroll
      for (int u = 0; u < kPrepBatch<D>; ++u) {
        const int64_t i = i0 + (int64_t)u * kPrepThreads;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const TIN xv = (i < n && k < d) ? x[(int64_t)k * n + i] : TIN(0);
          if constexpr (sizeof(TIN) == 4)
            c[u][k] = xv - sMeanF[k < d ? k : 0];
          else
            c[u][k] = xv - sMean[k < d ? k : 0];
        }
      }
#pragma unroll
      for (int u = 0; u < kPrepBatch<D>; ++u)
        if (i0 + (int64_t)u * kPrepThreads < n) {
          int m = 0;
#pragma unroll
          for (int a = 0; a < D; ++a)
#pragma unroll
            for (int b = a; b < D; ++b) {
              if (b < d) a2[m].add(c[u][a] * c[u][b]);
              ++m;
            }
        }
    }
    // pairs in the order (0,0), (0,1), ..., (1,1), ... of the first d coordinates
    double v[NP];
    {
      int m = 0, mo = 0;
#pragma unroll
      for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = a; b < D; ++b) {
          if (b < d) v[mo++] = a2[m].get();
          ++m;
        }
    }
    block_sum(v, npairs, scratch, sv);
  } else {
    constexpr int SB = 16384 / (D * (int)sizeof(TIN));  // staged samples per block
    TIN(*st)[D] = reinterpret_cast<TIN(*)[D]>(sm.stage);
    const int G = kPrepThreads / npairs;  // threads per pair
    const int t = threadIdx.x;
    const bool active = t < G * npairs;
    const int m = t % npairs, g = t / npairs;
    int pa = 0, rem = m;
    while (rem >= d - pa) {
      rem -= d - pa;
      ++pa;
    }
    const int pb = pa + rem;
    Acc<TIN> acc;
    for (int64_t i0 = 0; i0 < n; i0 += SB) {
      const int cnt = (int)min((int64_t)SB, n - i0);
      __syncthreads();  // previous block consumed
      for (int idx = threadIdx.x; idx < cnt * D; idx += kPrepThreads) {
        const int k = idx / cnt, i = idx - k * cnt;  // coordinate-major: coalesced reads
        TIN c = TIN(0);
        if (k < d) {
          const TIN xv = x[(int64_t)k * n + i0 + i];
          if constexpr (sizeof(TIN) == 4)
            c = xv - sMeanF[k];
          else
            c = xv - sMean[k];
        }
        st[i][k] = c;
      }
      __syncthreads();
      if (active)
        for (int i = g; i < cnt; i += G) acc.add(st[i][pa] * st[i][pb]);
    }
    __syncthreads();
    double* vals = &scratch[0][0];  // kPrepThreads values
    vals[threadIdx.x] = active ? acc.get() : 0.0;
    __syncthreads();
    if (threadIdx.x < npairs) {
      double tsum = 0.0;
      for (int gg = 0; gg < G; ++gg) tsum += vals[gg * npairs + threadIdx.x];
      sv[threadIdx.x] = tsum;
    }
    __syncthreads();
  }

  // ---- scalar work, FP64, one thread
  if (threadIdx.x == 0) {
    kde_result& res = ds->res;
    res.status = KDE_OK;
    res.method = ds->methods;
    res.d = d;
    res.n_h = ds->n_h;
    double S[KDE_MAX_D][KDE_MAX_D];
    int m = 0;
    bool finite = true;
    for (int a = 0; a < d; ++a) {
      ds->mean[a] = sMean[a];
      finite = finite && isfinite(sMean[a]);
      for (int b = a; b < d; ++b) {
        // LSCV_H: whiten by the given bandwidth matrix instead of S
        const double sab = ds->given_H ? ds->cov[a * d + b] : sv[m] / (double)(n - 1);
        S[a][b] = S[b][a] = sab;
        ++m;
      }
    }
    for (int a = 0; a < d; ++a)
      for (int b = 0; b < d; ++b) {
        ds->cov[a * d + b] = S[a][b];
        finite = finite && isfinite(S[a][b]);
      }
    double L[KDE_MAX_D][KDE_MAX_D] = {};
    bool pd = finite;
    for (int j = 0; j < d && pd; ++j) {
      double s = S[j][j];
      for (int k = 0; k < j; ++k) s -= L[j][k] * L[j][k];
      // Numerically singular for FP32 pair arithmetic: a Schur complement below
      // 1e-6 of the variance (the whitened coordinate would be rounding noise),
      // or a spread below 1e-5 of the magnitude of the values.
      const double mag = ds->given_H ? 0.0 : 1e-5 * fabs(sMean[j]);
      if (!(s > 1e-300) || !(s > 1e-6 * S[j][j]) || !(S[j][j] > mag * mag)) {
        pd = false;
        break;
      }
      L[j][j] = sqrt(s);
      for (int i = j + 1; i < d; ++i) {
        double t = S[i][j];
        for (int k = 0; k < j; ++k) t -= L[i][k] * L[j][k];
        L[i][j] = t / L[j][j];
      }
    }
    if (!finite) {
      res.status = KDE_EINVAL;
    } else if (!pd) {
      res.status = KDE_EDEGENERATE;
    } else {
      double W[KDE_MAX_D][KDE_MAX_D] = {};
      double logdet = 0.0;
      for (int i = 0; i < d; ++i) {
        logdet += 2.0 * log(L[i][i]);
        W[i][i] = 1.0 / L[i][i];
        for (int j = 0; j < i; ++j) {
          double t = 0.0;
          for (int k = j; k < i; ++k) t += L[i][k] * W[k][j];
          W[i][j] = -t / L[i][i];
        }
      }
      const double sl = sqrt(0.25 * kLog2e);
      for (int i = 0; i < KDE_MAX_D; ++i)
        for (int j = 0; j < KDE_MAX_D; ++j) {
          const float mv = (i < d && j <= i) ? (float)(sl * W[i][j]) : 0.f;
          ds->M[i * KDE_MAX_D + j] = mv;
          sM[i * KDE_MAX_D + j] = mv;
        }
      ds->logdet = logdet;
      res.logdet_S = logdet;
      ds->A = pow(4.0 * kPi, -0.5 * d) * exp(-0.5 * logdet);
      ds->sigma = sqrt(S[0][0]);
      if (d == 1) res.sigma = ds->sigma;
      if ((ds->methods & KDE_METHOD_PLUGIN) && d == 1) {
        const double sg = ds->sigma;
        const double psi8 = 105.0 / (32.0 * sqrt(kPi) * pow(sg, 9.0));
        const double k6_0 = -15.0 / sqrt(2.0 * kPi);
        const double g1 = pow(-2.0 * k6_0 / (psi8 * (double)n), 1.0 / 9.0);
        res.psi8_ns = psi8;
        res.g1 = g1;
        ds->psi_scale = (float)(sqrt(0.5 * kLog2e) / g1);
      }
    }
    sOk = (res.status == KDE_OK);
  }
  __syncthreads();
  if (!sOk) return;

  // ---- pass 3: whitened (LSCV) and centred (PLUGIN, d = 1) samples
  float* __restrict__ y = ds->y;
  float* __restrict__ xc = ds->xc;
  const int dk = ds->dk;
  for (int64_t i0 = threadIdx.x; i0 < n_pad; i0 += (int64_t)kPrepThreads * kPrepBatch<D>) {
    float c[kPrepBatch<D>][D];
#pragma unroll
    for (int u = 0; u < kPrepBatch<D>; ++u) {
      const int64_t i = i0 + (int64_t)u * kPrepThreads;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        c[u][k] = 0.f;
        if (i < n && k < d) {
          if constexpr (sizeof(TIN) == 4)
            c[u][k] = x[(int64_t)k * n + i] - sMeanF[k];
          else
            c[u][k] = (float)(x[(int64_t)k * n + i] - sMean[k]);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kPrepBatch<D>; ++u) {
      const int64_t i = i0 + (int64_t)u * kPrepThreads;
      if (i >= n_pad) break;
      if (y) {
#pragma unroll
        for (int k = 0; k < D; ++k) {
          float t = 0.f;
#pragma unroll
          for (int j = 0; j <= k; ++j) t = fmaf(sM[k * KDE_MAX_D + j], c[u][j], t);
          if (k < dk) y[(int64_t)k * n_pad + i] = t;  // rows d..dk-1: zero padding (M is 0 there)
        }
      }
      if (xc && d == 1) xc[i] = c[u][0];
    }
  }
}

// One CTA per dataset; `ids` (optional) selects the datasets of a table.
template <typename TIN>
__device__ __forceinline__ void prep_dispatch(DsDev* ds, PrepSmem& sm) {
  switch (ds->dk) {
    case 1: prep_body<TIN, 1>(ds, sm); break;
    case 2: prep_body<TIN, 2>(ds, sm); break;
    case 3: prep_body<TIN, 3>(ds, sm); break;
    case 4: prep_body<TIN, 4>(ds, sm); break;
    case 8: prep_body<TIN, 8>(ds, sm); break;
    case 12: prep_body<TIN, 12>(ds, sm); break;
    default: prep_body<TIN, 16>(ds, sm); break;
  }
}

__global__ void __launch_bounds__(kPrepThreads) k_prep(DsDev* dsa, const int* ids) {
  __shared__ PrepSmem sm;
  DsDev* ds = dsa + (ids ? ids[blockIdx.x] : (int)blockIdx.x);
  if (ds->dtype == KDE_F64)
    prep_dispatch<double>(ds, sm);
  else
    prep_dispatch<float>(ds, sm);
}

constexpr int kProbeThreads = 1024;
constexpr int kProbeSmem = 160 * 1024;  // > half an SM's shared memory: one CTA per SM

// ALU probe: `iters` rounds of 8 independent dependency chains per thread.
// mode 0: MUFU ex2; mode 1: scalar FFMA; mode 2: packed FP32x2 FMA.
// Each CTA records its clock64() span; out[blockIdx.x] = cycles.
template <int MODE>
__global__ void __launch_bounds__(kProbeThreads) k_probe(double* out, int iters, float seed) {
  float a[8];
  float2 p[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    a[k] = seed * (float)(threadIdx.x + k + 1) * 1e-4f;
    p[k] = make_float2(a[k], a[k] + 0.5f);
  }
  const float2 m2 = make_float2(0.9999f, 0.9998f), c2 = make_float2(1e-6f, 2e-6f);
  __syncthreads();
  long long t0 = clock64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        if (MODE == 0) a[k] = ex2(-a[k]);
        if (MODE == 1) a[k] = fmaf(a[k], 0.9999f, 1e-6f);
        if (MODE == 2) p[k] = __ffma2_rn(p[k], m2, c2);
      }
    }
  }
  __syncthreads();
  long long t1 = clock64();
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k] + p[k].x + p[k].y;
  if (s == 12345.678f) out[gridDim.x + blockIdx.x] = s;  // keeps the chains live
  if (threadIdx.x == 0) out[blockIdx.x] = (double)(t1 - t0);
}

}  // namespace

cudaError_t launch_setup(DsDev* dst, const DsDev& init, const double* h, int n_h,
                         int64_t* off_dst, const int64_t* off_src, int n_off, cudaStream_t st) {
  SetupParams p;
  p.init = init;
  p.n_off = n_off;
  for (int k = 0; k < 4; ++k) p.off[k] = k < n_off ? off_src[k] : 0;
  p.n_h = n_h;
  for (int k = 0; k < n_h && k < KDE_MAX_NH; ++k) p.h[k] = h[k];
  k_setup<<<1, 256, 0, st>>>(dst, off_dst, p);
  return cudaGetLastError();
}

cudaError_t launch_prep(DsDev* ds, int n_ds, const int* ids, cudaStream_t st) {
  if (n_ds <= 0) return cudaSuccess;
  k_prep<<<n_ds, kPrepThreads, 0, st>>>(ds, ids);
  return cudaGetLastError();
}

cudaError_t launch_probe_mode(int mode, double* out, int iters, int grid, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_probe<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, kProbeSmem))) return e;
    if ((e = cudaFuncSetAttribute(k_probe<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kProbeSmem))) return e;
    if ((e = cudaFuncSetAttribute(k_probe<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kProbeSmem))) return e;
    attr = true;
  }
  switch (mode) {
    case 0: k_probe<0><<<grid, kProbeThreads, kProbeSmem, st>>>(out, iters, 0.5f); break;
    case 1: k_probe<1><<<grid, kProbeThreads, kProbeSmem, st>>>(out, iters, 0.5f); break;
    default: k_probe<2><<<grid, kProbeThreads, kProbeSmem, st>>>(out, iters, 0.5f); break;
  }
  return cudaGetLastError();
}

}  // namespace gbkde
