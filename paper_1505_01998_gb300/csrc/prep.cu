// Prologue kernels: descriptor setup, sample statistics, Cholesky whitening
// and the first links of the PLUGIN chain; plus the ALU throughput probe.
#include <algorithm>
#include <cstddef>
#include <cstring>

#include "internal.cuh"

namespace gbkde {

namespace {

constexpr double kPsi8Coef = 1.8512470710160756;         // 105 / (32 sqrt(pi)) in FP64
constexpr double kSqrtHalfLog2e = 0.8493218002880191;     // sqrt(log2(e) / 2) in FP64
constexpr double kSqrtQuarterLog2e = 0.6005612043932249;  // sqrt(log2(e) / 4) in FP64
constexpr int kPrepThreads = 512;

constexpr int kDsWords = (int)(sizeof(DsDev) / sizeof(uint64_t));
static_assert(sizeof(DsDev) % sizeof(uint64_t) == 0, "descriptor copied as 8-byte words");

// Kernel parameters of k_setup, sized for grids of up to NH points (the
// parameter block is copied at every launch: 64-point grids and PLUGIN
// calls take the small one).
template <int NH>
struct SetupParams {
  uint64_t init[kDsWords];  // the host-built descriptor, as words
  int64_t off[4];
  int32_t n_off;
  int32_t n_h, n_h_pad;
  double* h_dst;            // the descriptor's h[] and nc[]
  float* nc_dst;
  double h[NH];
  float nc[NH];             // -1/h^2 (FP64, rounded to FP32; padding entries -1)
};

// Words of the descriptor that the host may set: the geometry header (up to
// the strip counters), oct_P, the host constants c_A and c_g1, the result
// block, and the given bandwidth matrix in cov[] (LSCV_H, density estimates).
// Every other word starts at zero.  Parameter words read at distinct
// addresses within a warp are serialised constant-bank accesses, so the copy
// reads only these words (about 70 of about 500 without a given H) and stores
// zeros elsewhere (measured: about 400 clocks less per one-range prologue);
// fill_setup checks on the host that no other word is nonzero.
__host__ __device__ inline bool setup_word_copied(int i, bool given_H) {
  constexpr int w_head = (int)(offsetof(DsDev, strip_count) / 8);
  constexpr int w_oct = (int)(offsetof(DsDev, oct_P) / 8);
  constexpr int w_cov0 = (int)(offsetof(DsDev, cov) / 8), w_cov1 = w_cov0 + KDE_MAX_D * KDE_MAX_D;
  constexpr int w_c0 = (int)(offsetof(DsDev, c_A) / 8), w_c1 = (int)(offsetof(DsDev, M) / 8);
  constexpr int w_res = (int)(offsetof(DsDev, res) / 8);
  static_assert(offsetof(DsDev, c_g1) / 8 < offsetof(DsDev, M) / 8 && sizeof(double) == 8, "layout");
  return i < w_head || i == w_oct || (given_H && i >= w_cov0 && i < w_cov1) || (i >= w_c0 && i < w_c1) ||
         i >= w_res;
}

// Copies the host-built descriptor into device memory, one word per thread,
// and the grid's h[k] and nc[k] = -1/h_k^2 into its arrays.
template <int NH>
__device__ __forceinline__ void setup_copy(DsDev* dst, int64_t* off_dst, const SetupParams<NH>& p) {
  uint64_t* d64 = reinterpret_cast<uint64_t*>(dst);
  const bool given_H = reinterpret_cast<const DsDev*>(p.init)->given_H != 0;
  for (int i = threadIdx.x; i < kDsWords; i += blockDim.x)
    d64[i] = setup_word_copied(i, given_H) ? p.init[i] : 0ull;
  if (threadIdx.x < p.n_off) off_dst[threadIdx.x] = p.off[threadIdx.x];
  for (int k = threadIdx.x; k < p.n_h_pad; k += blockDim.x) {
    if (k < p.n_h) p.h_dst[k] = p.h[k];
    p.nc_dst[k] = p.nc[k];
  }
}

template <int NH>
__global__ void k_setup(DsDev* dst, int64_t* off_dst, SetupParams<NH> p) {
  dependent_launch_wait();
  setup_copy(dst, off_dst, p);
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
  // the lane's total as a double-float pair (value s - c)
  __device__ float2 lane() const { return make_float2(s, -c); }
};
template <>
struct Acc<double> {
  double s = 0.0;
  __device__ void add(double v) { s += v; }
  __device__ double get() const { return s; }
  __device__ double lane() const { return s; }
};

// Warp total of one double-float value per lane (FP32 samples) into *dst
// (lane 0), in FP32 arithmetic.
__device__ __forceinline__ void warp_total(float2 v, double* dst, int lane) {
  const float2 t = warp_sum_ff(v.x, v.y);
  if (lane == 0) *dst = ff_value(t);
}

// Block-wide sum of `cnt` values per thread, deterministic order; results
// land in out[0..cnt) (shared memory, FP64) for every thread.  Double-float
// lanes (FP32 samples): a butterfly per warp, then the warp totals in FP64.
template <typename V>
__device__ void block_sum(const V* v, int cnt, double (*scratch)[kNPairs], double* out) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = 0; k < cnt; ++k) warp_total(v[k], &scratch[warp][k], lane);
  __syncthreads();
  if (threadIdx.x < cnt) {
    double t = 0.0;
    for (int w = 0; w < kPrepThreads / 32; ++w) t += scratch[w][threadIdx.x];
    out[threadIdx.x] = t;
  }
  __syncthreads();
}

// FP64 lanes (FP64 samples): the lane values go through shared memory and one
// warp per value adds them, 16 per lane in order and then a butterfly.  That
// is about a quarter of the FP64 operations of a butterfly in every warp (FP64
// runs at a small fraction of the FP32 rate on this part); measured at
// n = 1,024, about 900 clocks less per moment pass.  Values go in rounds of 4
// (4 x 512 doubles fit the scratch array).
__device__ void block_sum(const double* v, int cnt, double (*scratch)[kNPairs], double* out) {
  constexpr int kPer = 4;
  static_assert(kPer * kPrepThreads <= (kPrepThreads / 32) * kNPairs, "staging fits the scratch array");
  double* stage = &scratch[0][0];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k0 = 0; k0 < cnt; k0 += kPer) {
    const int nk = min(kPer, cnt - k0);
    for (int k = 0; k < nk; ++k) stage[k * kPrepThreads + threadIdx.x] = v[k0 + k];
    __syncthreads();
    if (warp < nk) {
      const double* col = stage + warp * kPrepThreads;
      double t = 0.0;
#pragma unroll
      for (int j = 0; j < kPrepThreads / 32; ++j) t += col[j * 32 + lane];
      t = warp_sum(t);
      if (lane == 0) out[k0 + warp] = t;
    }
    __syncthreads();
  }
}

// Shared memory of the prologue kernels, declared once per kernel for every
// (element type, dimension) instance.
struct PrepSmem {
  double scratch[kPrepThreads / 32][kNPairs];
  double sv[kNPairs];
  double sMean[KDE_MAX_D];
  float sM[KDE_MAX_D * KDE_MAX_D];
  float sMeanF[KDE_MAX_D];
  int last;
  // centred samples of the pair-parallel moment pass (D >= 8)
  alignas(16) unsigned char stage[16384];
};

// samples per thread whose loads are issued together (wide samples already
// issue D independent loads per sample)
template <int D>
constexpr int kPrepBatch = D >= 8 ? 1 : 4;

// The sample range [lo, hi) of part b of a dataset cut into `parts` ranges.
__device__ __forceinline__ void prep_range(int64_t n, int parts, int b, int64_t& lo, int64_t& hi) {
  const int64_t blk = (n + parts - 1) / parts;
  lo = min(n, (int64_t)b * blk);
  hi = min(n, lo + blk);
}

// Mean of samples [lo, hi) into sMean / sMeanF, then the cross products of
// the samples centred about it (in the input precision: FP32 samples take
// the FP32-rounded mean as the centre) into sv, pairs a <= b in order.
// Per-thread sums: FP32 Kahan (FP32 input) or FP64; across threads FP64.
// For D >= 8 the cross products are pair-parallel: blocks of centred samples
// are staged in shared memory and thread t adds pair t mod P (P = d(d+1)/2)
// over every G-th sample of the block.
template <typename TIN, int D>
__device__ __forceinline__ void prep_moments(const DsDev* ds, PrepSmem& sm, int64_t lo, int64_t hi) {
  const TIN* __restrict__ x = static_cast<const TIN*>(ds->x);
  const int64_t n = ds->n;
  const int d = D <= 4 ? D : ds->d;  // dk = d for d <= 4: a compile-time bound there
  const int64_t cnt = hi - lo;
  {
    Acc<TIN> a1[D];
    for (int64_t i0 = lo + threadIdx.x; i0 < hi; i0 += (int64_t)kPrepThreads * kPrepBatch<D>) {
      TIN v[kPrepBatch<D>][D];
#pragma unroll
      for (int u = 0; u < kPrepBatch<D>; ++u) {
        const int64_t i = i0 + (int64_t)u * kPrepThreads;
#pragma unroll
        for (int k = 0; k < D; ++k) v[u][k] = (i < hi && k < d) ? x[(int64_t)k * n + i] : TIN(0);
      }
#pragma unroll
      for (int u = 0; u < kPrepBatch<D>; ++u)
        if (i0 + (int64_t)u * kPrepThreads < hi) {
#pragma unroll
          for (int k = 0; k < D; ++k)
            if (k < d) a1[k].add(v[u][k]);
        }
    }
    decltype(a1[0].lane()) v[D];
#pragma unroll
    for (int k = 0; k < D; ++k) v[k] = a1[k].lane();
    block_sum(v, d, sm.scratch, sm.sv);
  }
  if (threadIdx.x < d) {
    sm.sMean[threadIdx.x] = cnt > 0 ? sm.sv[threadIdx.x] / (double)cnt : 0.0;
    sm.sMeanF[threadIdx.x] = (float)sm.sMean[threadIdx.x];
  }
  __syncthreads();
  const int npairs = d * (d + 1) / 2;
  if (ds->given_H) {  // whitening by a given bandwidth matrix: no sample covariance
    if (threadIdx.x < npairs) sm.sv[threadIdx.x] = 0.0;
    __syncthreads();
    return;
  }
  if constexpr (D <= 4) {
    constexpr int NP = D * (D + 1) / 2;
    Acc<TIN> a2[NP];
    for (int64_t i0 = lo + threadIdx.x; i0 < hi; i0 += (int64_t)kPrepThreads * kPrepBatch<D>) {
      TIN c[kPrepBatch<D>][D];
#pragma unroll
      for (int u = 0; u < kPrepBatch<D>; ++u) {
        const int64_t i = i0 + (int64_t)u * kPrepThreads;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const TIN xv = (i < hi && k < d) ? x[(int64_t)k * n + i] : TIN(0);
          if constexpr (sizeof(TIN) == 4)
            c[u][k] = xv - sm.sMeanF[k < d ? k : 0];
          else
            c[u][k] = xv - sm.sMean[k < d ? k : 0];
        }
      }
#pragma unroll
      for (int u = 0; u < kPrepBatch<D>; ++u)
        if (i0 + (int64_t)u * kPrepThreads < hi) {
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
    decltype(a2[0].lane()) v[NP];
    {
      int m = 0, mo = 0;
#pragma unroll
      for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = a; b < D; ++b) {
          if (b < d) v[mo++] = a2[m].lane();
          ++m;
        }
    }
    block_sum(v, npairs, sm.scratch, sm.sv);
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
    for (int64_t i0 = lo; i0 < hi; i0 += SB) {
      const int c = (int)min((int64_t)SB, hi - i0);
      __syncthreads();  // previous block consumed
      for (int idx = threadIdx.x; idx < c * D; idx += kPrepThreads) {
        const int k = idx / c, i = idx - k * c;  // coordinate-major: coalesced reads
        TIN v = TIN(0);
        if (k < d) {
          const TIN xv = x[(int64_t)k * n + i0 + i];
          if constexpr (sizeof(TIN) == 4)
            v = xv - sm.sMeanF[k];
          else
            v = xv - sm.sMean[k];
        }
        st[i][k] = v;
      }
      __syncthreads();
      if (active)
        for (int i = g; i < c; i += G) acc.add(st[i][pa] * st[i][pb]);
    }
    __syncthreads();
    double* vals = &sm.scratch[0][0];  // kPrepThreads values
    vals[threadIdx.x] = active ? acc.get() : 0.0;
    __syncthreads();
    if (threadIdx.x < npairs) {
      double tsum = 0.0;
      for (int gg = 0; gg < G; ++gg) tsum += vals[gg * npairs + threadIdx.x];
      sm.sv[threadIdx.x] = tsum;
    }
    __syncthreads();
  }
}

// Part b of the prologue of one dataset (grid: parts x datasets).  Each CTA
// takes the moments of its sample range and stores them as a record; the
// CTA that finishes last (a counter in the descriptor; no CTA waits for
// another) combines the records in range order -- the dataset mean
// mu = sum_b n_b m_b / n and the centred cross products
// sum_b [M_b + n_b (u v^T + v u^T + v v^T)], u = m_b - c_b, v = c_b - mu
// (c_b the centre M_b was taken about), which equals the two-pass
// sum (x - mu)(x - mu)^T (Eq. LSCV-covariance / PLUGIN-VarianceEstimator
// evaluated two-pass, reading R7) -- and then, in FP64 across the CTA's
// threads: Cholesky S = L L^T, log|S|, the whitening matrix
// M = sqrt(log2 e / 4) L^-1, sigma, A and, for the PLUGIN method, psi_8^NS
// (Eq. PLUGIN-Psi8Estimate) and g1 (Eq. PLUGIN-g1).
// Returns true (on every thread of the CTA) when this CTA completed the
// dataset's statistics and they are usable (the CTA of a one-range dataset,
// or the last range's CTA).
template <typename TIN, int D>
__device__ __forceinline__ bool prep_stats(DsDev* ds, PrepSmem& sm, int b) {
  const int parts = ds->prep_parts;
  if (b >= parts) return false;
  const int64_t n = ds->n;
  const int d = D <= 4 ? D : ds->d;  // dk = d for d <= 4: a compile-time bound there
  int64_t lo, hi;
  prep_range(n, parts, b, lo, hi);
  prep_moments<TIN, D>(ds, sm, lo, hi);
  const int npairs = d * (d + 1) / 2;
  double* sMean = sm.sMean;
  double* sv = sm.sv;
  float* sM = sm.sM;
  if (parts == 1) {
    // one range: mu is the range mean m (already in sMean), and the moments
    // about mu follow from those about the centre c by one parallel-axis
    // term, M - n u u^T with u = m - c -- the combination below with a single
    // record, without its rounding of n m / n.  c = m for FP64 samples (no
    // term); FP32 samples were centred about the FP32-rounded mean.
    if constexpr (sizeof(TIN) == 4) {
      if (!ds->given_H && threadIdx.x < npairs) {
        int pa = 0, rem = threadIdx.x;
        while (rem >= d - pa) {
          rem -= d - pa;
          ++pa;
        }
        const int pb = pa + rem;
        const double ua = sMean[pa] - (double)sm.sMeanF[pa], ub = sMean[pb] - (double)sm.sMeanF[pb];
        sv[threadIdx.x] -= (double)(hi - lo) * ua * ub;
      }
    }
    __syncthreads();
  } else {
    double* rec = ds->prep_part + (size_t)b * kPrepRecord;
    if (threadIdx.x == 0) rec[0] = (double)(hi - lo);
    if (threadIdx.x < d) {
      rec[1 + threadIdx.x] = sm.sMean[threadIdx.x];
      rec[1 + KDE_MAX_D + threadIdx.x] = sizeof(TIN) == 4 ? (double)sm.sMeanF[threadIdx.x] : sm.sMean[threadIdx.x];
    }
    if (threadIdx.x < npairs) rec[1 + 2 * KDE_MAX_D + threadIdx.x] = sm.sv[threadIdx.x];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) sm.last = (atomicAdd(&ds->prep_count, 1u) == (unsigned)parts - 1u);
    __syncthreads();
    if (!sm.last) return false;
    __threadfence();
    // ---- combine the records in range order (records staged in shared
    // memory, kChunk at a time, by coalesced loads; the sums run in range order)
    const double* recs = ds->prep_part;
    constexpr int kChunk = (int)(sizeof(sm.stage) / (kPrepRecord * sizeof(double)));
    double* cache = reinterpret_cast<double*>(sm.stage);
    int pa = 0, pb = 0;
    if (threadIdx.x < npairs) {
      int rem = threadIdx.x;
      while (rem >= d - pa) {
        rem -= d - pa;
        ++pa;
      }
      pb = pa + rem;
    }
    double tmean = 0.0;
    for (int r0 = 0; r0 < parts; r0 += kChunk) {
      const int nr = min(kChunk, parts - r0);
      __syncthreads();
      for (int idx = threadIdx.x; idx < nr * kPrepRecord; idx += kPrepThreads)
        cache[idx] = __ldcg(recs + (size_t)r0 * kPrepRecord + idx);
      __syncthreads();
      if (threadIdx.x < d)
        for (int r = 0; r < nr; ++r) tmean += cache[r * kPrepRecord] * cache[r * kPrepRecord + 1 + threadIdx.x];
    }
    if (threadIdx.x < d) sMean[threadIdx.x] = tmean / (double)n;
    __syncthreads();
    double tpair = 0.0;
    for (int r0 = 0; r0 < parts && !ds->given_H; r0 += kChunk) {  // a given H needs no S
      const int nr = min(kChunk, parts - r0);
      if (parts > kChunk || r0 > 0) {  // one chunk: still cached from the mean pass
        __syncthreads();
        for (int idx = threadIdx.x; idx < nr * kPrepRecord; idx += kPrepThreads)
          cache[idx] = __ldcg(recs + (size_t)r0 * kPrepRecord + idx);
        __syncthreads();
      }
      if (threadIdx.x < npairs)
        for (int r = 0; r < nr; ++r) {
          const double* q = cache + r * kPrepRecord;
          const double nb = q[0];
          const double ua = q[1 + pa] - q[1 + KDE_MAX_D + pa];
          const double ub = q[1 + pb] - q[1 + KDE_MAX_D + pb];
          const double va = q[1 + KDE_MAX_D + pa] - sMean[pa];
          const double vb = q[1 + KDE_MAX_D + pb] - sMean[pb];
          tpair += q[1 + 2 * KDE_MAX_D + threadIdx.x] + nb * (ua * vb + va * ub + va * vb);
        }
    }
    __syncthreads();
    if (threadIdx.x < npairs) sv[threadIdx.x] = tpair;
    if (threadIdx.x == 0) ds->prep_count = 0u;  // ready for the next run of this descriptor
    __syncthreads();
  }
  // ---- factorisation, FP64, shared by the CTA's threads (the textbook
  // loops; the inverse multiplies by the reciprocal of each diagonal entry)
  double(*S)[KDE_MAX_D] = reinterpret_cast<double(*)[KDE_MAX_D]>(&sm.scratch[0][0]);
  double(*L)[KDE_MAX_D] = S + KDE_MAX_D;
  double(*W)[KDE_MAX_D] = S + 2 * KDE_MAX_D;
  kde_result& res = ds->res;
  bool fin = true;
  for (int t = threadIdx.x; t < KDE_MAX_D * KDE_MAX_D; t += kPrepThreads) {
    const int ra = t / KDE_MAX_D, rb = t % KDE_MAX_D;
    double v = 0.0;
    if (ra < d && rb < d) {
      const int lo_ = min(ra, rb), hi_ = max(ra, rb);
      const int m = lo_ * d - lo_ * (lo_ - 1) / 2 + (hi_ - lo_);  // pair (lo_, hi_) in a <= b order
      // LSCV_H: whiten by the given bandwidth matrix instead of S
      v = ds->given_H ? ds->cov[ra * d + rb] : sv[m] / (double)(n - 1);
      fin = fin && isfinite(v);
    }
    S[ra][rb] = v;
    L[ra][rb] = 0.0;
    W[ra][rb] = 0.0;
  }
  if (threadIdx.x < d) fin = fin && isfinite(sMean[threadIdx.x]);
  const bool finite = __syncthreads_and(fin) != 0;
  if (threadIdx.x == 0) {
    res.status = KDE_OK;
    res.method = ds->methods;
    res.d = d;
    res.n_h = ds->n_h;
    for (int a2 = 0; a2 < d; ++a2) ds->mean[a2] = sMean[a2];
  }
  for (int t = threadIdx.x; t < d * d; t += kPrepThreads) ds->cov[t] = S[t / d][t % d];
  // Cholesky S = L L^T, column by column; the pivot's reciprocal square root
  // scales the column (FP64 divisions and square roots are long sequences on
  // this part, and they sit on the critical path of every column)
  double* rdiag = &W[KDE_MAX_D - 1][0] + KDE_MAX_D;  // [KDE_MAX_D] 1 / L_jj, after W
  double* ldiag = rdiag + KDE_MAX_D;                 // [KDE_MAX_D] log of the pivots L_jj^2
  double* piv = ldiag + KDE_MAX_D;                   // [KDE_MAX_D] the pivots
  if (threadIdx.x == 0) sm.last = finite ? 1 : 0;  // reused as the "positive definite so far" flag
  __syncthreads();
  for (int j = 0; j < d && sm.last; ++j) {
    if (threadIdx.x == 0) {
      double sj = S[j][j];
      for (int k = 0; k < j; ++k) sj -= L[j][k] * L[j][k];
      // Numerically singular for FP32 pair arithmetic: a Schur complement below
      // 1e-6 of the variance (the whitened coordinate would be rounding noise),
      // or a spread below 1e-5 of the magnitude of the values.
      const double mag = ds->given_H ? 0.0 : 1e-5 * fabs(sMean[j]);
      if (!(sj > 1e-300) || !(sj > 1e-6 * S[j][j]) || !(S[j][j] > mag * mag)) {
        sm.last = 0;
      } else {
        const double r = rsqrt(sj);
        L[j][j] = sj * r;
        rdiag[j] = r;
        piv[j] = sj;
      }
    }
    __syncthreads();
    if (!sm.last) break;
    const int i = j + 1 + (int)threadIdx.x;
    if (i < d) {
      double t = S[i][j];
      for (int k = 0; k < j; ++k) t -= L[i][k] * L[j][k];
      L[i][j] = t * rdiag[j];
    }
    __syncthreads();
  }
  const bool pd = finite && sm.last;
  if (!finite || !pd) {
    if (threadIdx.x == 0) res.status = finite ? KDE_EDEGENERATE : KDE_EINVAL;
    return false;
  }
  // W = L^-1, one column per thread (forward substitution, scaled by the
  // reciprocals of the diagonal); the log of each pivot alongside
  // (log|S| = sum_i log L_ii^2, summed in order below)
  if (threadIdx.x < d) ldiag[threadIdx.x] = log(piv[threadIdx.x]);
  // sigma and the PLUGIN pilot on a thread of another warp, alongside the
  // logs: with r = 1 / sigma from one reciprocal square root, sigma = S_00 r,
  // psi_8^NS = 105 / (32 sqrt(pi) sigma^9) = c r^9 and
  // g1 = (-2 K6(0) / (psi_8^NS n))^(1/9) = sigma c_g1 (c_g1 of n from the
  // host): the chain's one long FP64 operation is the reciprocal square root
  // (the division of the psi scale, of two known constants, runs beside it)
  if (threadIdx.x == 32) {
    const double s00 = S[0][0];
    const double rs = rsqrt(s00);
    const double sg = s00 * rs;
    ds->sigma = sg;
    if (d == 1) res.sigma = sg;
    if ((ds->methods & KDE_METHOD_PLUGIN) && d == 1) {
      const double r2 = rs * rs, r4 = r2 * r2, r8 = r4 * r4;
      res.psi8_ns = kPsi8Coef * (r8 * rs);
      res.g1 = sg * ds->c_g1;
      ds->psi_scale = (float)(rs * (kSqrtHalfLog2e / ds->c_g1));
    }
  }
  if (threadIdx.x < d) {
    const int j = threadIdx.x;
    W[j][j] = rdiag[j];
    for (int i = j + 1; i < d; ++i) {
      double t = 0.0;
      for (int k = j; k < i; ++k) t += L[i][k] * W[k][j];
      W[i][j] = -t * rdiag[i];
    }
  }
  __syncthreads();
  const double sl = kSqrtQuarterLog2e;
  for (int t = threadIdx.x; t < KDE_MAX_D * KDE_MAX_D; t += kPrepThreads) {
    const int i = t / KDE_MAX_D, j = t % KDE_MAX_D;
    const float mv = (i < d && j <= i) ? (float)(sl * W[i][j]) : 0.f;
    ds->M[t] = mv;
    sM[t] = mv;
  }
  // log|S| and A = (4 pi)^(-d/2) |S|^(-1/2) = c_A prod_i 1 / L_ii (c_A of d
  // from the host), without FP64 pow or exp
  if (threadIdx.x == 0) {
    double logdet = 0.0, a = ds->c_A;
    for (int i = 0; i < d; ++i) {
      logdet += ldiag[i];
      a *= rdiag[i];
    }
    ds->logdet = logdet;
    res.logdet_S = logdet;
    ds->A = a;
  }
  return true;
}

// Part b of the whitening pass: y = M (x - mean) and x - mean in FP32 for
// the samples of range b (the last range also writes the zero padding up to
// n_pad).
struct WhitenSmem {
  double sMean[KDE_MAX_D];
  float sM[KDE_MAX_D * KDE_MAX_D];
  float sMeanF[KDE_MAX_D];
};

// M and the mean come from srcM / srcMean: the descriptor (a separate
// whitening launch) or, in the CTA that just computed them, its shared memory
// (no read-back of its own global writes).  The caller checks the status.
template <typename TIN, int D>
__device__ __forceinline__ void prep_whiten(const DsDev* ds, WhitenSmem& sm, int b, const float* srcM,
                                            const double* srcMean) {
  const int parts = ds->prep_parts;
  if (b >= parts) return;
  const TIN* __restrict__ x = static_cast<const TIN*>(ds->x);
  const int64_t n = ds->n, n_pad = ds->n_pad;
  const int d = D <= 4 ? D : ds->d, dk = D <= 4 ? D : ds->dk;  // compile-time for d <= 4
  for (int k = threadIdx.x; k < KDE_MAX_D * KDE_MAX_D; k += kPrepThreads) sm.sM[k] = srcM[k];
  if (threadIdx.x < KDE_MAX_D) {
    sm.sMean[threadIdx.x] = threadIdx.x < d ? srcMean[threadIdx.x] : 0.0;
    sm.sMeanF[threadIdx.x] = (float)sm.sMean[threadIdx.x];
  }
  __syncthreads();
  int64_t lo, hi;
  prep_range(n, parts, b, lo, hi);
  if (b == parts - 1) hi = n_pad;
  float* __restrict__ y = ds->y;
  float* __restrict__ xc = ds->xc;
  for (int64_t i0 = lo + threadIdx.x; i0 < hi; i0 += (int64_t)kPrepThreads * kPrepBatch<D>) {
    float c[kPrepBatch<D>][D];
#pragma unroll
    for (int u = 0; u < kPrepBatch<D>; ++u) {
      const int64_t i = i0 + (int64_t)u * kPrepThreads;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        c[u][k] = 0.f;
        if (i < n && k < d) {
          if constexpr (sizeof(TIN) == 4)
            c[u][k] = x[(int64_t)k * n + i] - sm.sMeanF[k];
          else
            c[u][k] = (float)(x[(int64_t)k * n + i] - sm.sMean[k]);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kPrepBatch<D>; ++u) {
      const int64_t i = i0 + (int64_t)u * kPrepThreads;
      if (i >= hi) break;
      if (y) {
        // M is re-read from shared memory per sample (volatile): hoisting its
        // D(D+1)/2 entries out of the loop would exhaust the registers at D = 16
        const volatile float* vM = sm.sM;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          float t = 0.f;
#pragma unroll
          for (int j = 0; j <= k; ++j) t = fmaf(vM[k * KDE_MAX_D + j], c[u][j], t);
          if (k < dk) y[(int64_t)k * n_pad + i] = t;  // rows d..dk-1: zero padding (M is 0 there)
        }
      }
      if (xc && d == 1) xc[i] = c[u][0];
    }
  }
}

template <typename TIN>
__device__ __forceinline__ bool stats_dispatch(DsDev* ds, PrepSmem& sm, int b) {
  switch (ds->dk) {
    case 1: return prep_stats<TIN, 1>(ds, sm, b);
    case 2: return prep_stats<TIN, 2>(ds, sm, b);
    case 3: return prep_stats<TIN, 3>(ds, sm, b);
    case 4: return prep_stats<TIN, 4>(ds, sm, b);
    case 8: return prep_stats<TIN, 8>(ds, sm, b);
    case 12: return prep_stats<TIN, 12>(ds, sm, b);
    default: return prep_stats<TIN, 16>(ds, sm, b);
  }
}

template <typename TIN>
__device__ __forceinline__ void whiten_dispatch(DsDev* ds, WhitenSmem& sm, int b, const float* srcM,
                                                const double* srcMean) {
  switch (ds->dk) {
    case 1: prep_whiten<TIN, 1>(ds, sm, b, srcM, srcMean); break;
    case 2: prep_whiten<TIN, 2>(ds, sm, b, srcM, srcMean); break;
    case 3: prep_whiten<TIN, 3>(ds, sm, b, srcM, srcMean); break;
    case 4: prep_whiten<TIN, 4>(ds, sm, b, srcM, srcMean); break;
    case 8: prep_whiten<TIN, 8>(ds, sm, b, srcM, srcMean); break;
    case 12: prep_whiten<TIN, 12>(ds, sm, b, srcM, srcMean); break;
    default: prep_whiten<TIN, 16>(ds, sm, b, srcM, srcMean); break;
  }
}

// grid: (parts_max, datasets); `ids` (optional) selects the datasets of a table.
// whiten: every dataset of the launch has one range, so its CTA also
// whitens (the statistics it needs are its own) and k_prep_whiten is not
// launched.
__global__ void __launch_bounds__(kPrepThreads) k_prep_stats(DsDev* dsa, const int* ids, int whiten) {
  __shared__ PrepSmem sm;
  dependent_launch_wait();
  DsDev* ds = dsa + (ids ? ids[blockIdx.y] : (int)blockIdx.y);
  const bool ok = ds->dtype == KDE_F64 ? stats_dispatch<double>(ds, sm, blockIdx.x)
                                       : stats_dispatch<float>(ds, sm, blockIdx.x);
  if (whiten && ok) {  // one range: this CTA's M and mean, from its shared memory
    __shared__ WhitenSmem wm;
    __syncthreads();
    if (ds->dtype == KDE_F64)
      whiten_dispatch<double>(ds, wm, blockIdx.x, sm.sM, sm.sMean);
    else
      whiten_dispatch<float>(ds, wm, blockIdx.x, sm.sM, sm.sMean);
  }
}

// Setup, statistics and whitening of one dataset whose prologue is a single
// range (one CTA): the CTA writes the descriptor and the grid itself, so the
// separate k_setup launch is not needed.  (With several ranges every CTA would
// need the descriptor first, and a late copy would reset the range counter.)
template <int NH>
__global__ void __launch_bounds__(kPrepThreads) k_setup_prep1(DsDev* ds, int64_t* off_dst, SetupParams<NH> p) {
  __shared__ PrepSmem sm;
  __shared__ WhitenSmem wm;
  dependent_launch_wait();
  setup_copy(ds, off_dst, p);
  __syncthreads();  // the descriptor this CTA just wrote is read below
  const bool ok = ds->dtype == KDE_F64 ? stats_dispatch<double>(ds, sm, 0) : stats_dispatch<float>(ds, sm, 0);
  if (!ok) return;
  __syncthreads();
  if (ds->dtype == KDE_F64)
    whiten_dispatch<double>(ds, wm, 0, sm.sM, sm.sMean);
  else
    whiten_dispatch<float>(ds, wm, 0, sm.sM, sm.sMean);
}

__global__ void __launch_bounds__(kPrepThreads) k_prep_whiten(DsDev* dsa, const int* ids) {
  __shared__ WhitenSmem sm;
  dependent_launch_wait();
  DsDev* ds = dsa + (ids ? ids[blockIdx.y] : (int)blockIdx.y);
  if (ds->res.status != KDE_OK) return;
  if (ds->dtype == KDE_F64)
    whiten_dispatch<double>(ds, sm, blockIdx.x, ds->M, ds->mean);
  else
    whiten_dispatch<float>(ds, sm, blockIdx.x, ds->M, ds->mean);
}

constexpr int kProbeThreads = 1024;
constexpr int kProbeSmem = 160 * 1024;  // > half an SM's shared memory: one CTA per SM

// ALU probe: `iters` rounds of 8 independent dependency chains per thread.
// mode 0: MUFU ex2; mode 1: scalar FFMA; mode 2: packed FP32x2 FMA; mode 3:
// packed FP32x2 multiplies and adds (independent chains, half each).
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
        // two independent chains (a product and a sum): nothing to contract into an FMA
        if (MODE == 3) {
          if (k & 1)
            p[k] = __fadd2_rn(p[k], c2);
          else
            p[k] = __fmul2_rn(p[k], m2);
        }
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

template <int NH>
static cudaError_t fill_setup(SetupParams<NH>* p, const DsDev& init, const double* h, int n_h,
                              const int64_t* off_src, int n_off) {
  memcpy(p->init, &init, sizeof(DsDev));
  for (int i = 0; i < kDsWords; ++i)  // the device copies only these words (setup_word_copied)
    if (p->init[i] != 0 && !setup_word_copied(i, init.given_H != 0)) return cudaErrorInvalidValue;
  p->n_off = n_off;
  for (int k = 0; k < 4; ++k) p->off[k] = k < n_off ? off_src[k] : 0;
  p->n_h = std::min(n_h, NH);
  p->n_h_pad = std::min(init.n_h_pad, NH);
  p->h_dst = init.h;
  p->nc_dst = init.nc;
  for (int k = 0; k < p->n_h_pad; ++k) {
    p->h[k] = k < p->n_h ? h[k] : 0.0;
    p->nc[k] = k < p->n_h ? (float)(-1.0 / (h[k] * h[k])) : -1.0f;
  }
  return cudaSuccess;
}

template <int NH>
static cudaError_t launch_setup_t(DsDev* dst, const DsDev& init, const double* h, int n_h,
                                  int64_t* off_dst, const int64_t* off_src, int n_off, cudaStream_t st) {
  SetupParams<NH> p;
  const cudaError_t e = fill_setup(&p, init, h, n_h, off_src, n_off);
  if (e != cudaSuccess) return e;
  return launch_kernel(k_setup<NH>, dim3(1), dim3(256), 0, st, dst, off_dst, p);
}

cudaError_t launch_setup(DsDev* dst, const DsDev& init, const double* h, int n_h,
                         int64_t* off_dst, const int64_t* off_src, int n_off, cudaStream_t st) {
  if (std::max(n_h, init.n_h_pad) <= 64)
    return launch_setup_t<64>(dst, init, h, n_h, off_dst, off_src, n_off, st);
  return launch_setup_t<KDE_MAX_NH>(dst, init, h, n_h, off_dst, off_src, n_off, st);
}

template <int NH>
static cudaError_t launch_setup_prep1_t(DsDev* dst, const DsDev& init, const double* h, int n_h,
                                        int64_t* off_dst, const int64_t* off_src, int n_off, cudaStream_t st) {
  SetupParams<NH> p;
  const cudaError_t e = fill_setup(&p, init, h, n_h, off_src, n_off);
  if (e != cudaSuccess) return e;
  return launch_kernel(k_setup_prep1<NH>, dim3(1), dim3(kPrepThreads), 0, st, dst, off_dst, p);
}

cudaError_t launch_setup_prep(DsDev* dst, const DsDev& init, const double* h, int n_h, int64_t* off_dst,
                              const int64_t* off_src, int n_off, cudaStream_t st) {
  if (init.prep_parts > 1) {  // several ranges: the descriptor first, in its own launch
    const cudaError_t e = launch_setup(dst, init, h, n_h, off_dst, off_src, n_off, st);
    if (e != cudaSuccess) return e;
    return launch_prep(dst, 1, nullptr, init.prep_parts, st);
  }
  if (std::max(n_h, init.n_h_pad) <= 64)
    return launch_setup_prep1_t<64>(dst, init, h, n_h, off_dst, off_src, n_off, st);
  return launch_setup_prep1_t<KDE_MAX_NH>(dst, init, h, n_h, off_dst, off_src, n_off, st);
}

cudaError_t launch_prep(DsDev* ds, int n_ds, const int* ids, int parts_max, cudaStream_t st) {
  if (n_ds <= 0) return cudaSuccess;
  const dim3 grid((unsigned)std::max(1, parts_max), (unsigned)n_ds);
  const int fused = parts_max <= 1;
  cudaError_t e = launch_kernel(k_prep_stats, grid, dim3(kPrepThreads), 0, st, ds, ids, fused);
  if (e != cudaSuccess || fused) return e;
  return launch_kernel(k_prep_whiten, grid, dim3(kPrepThreads), 0, st, ds, ids);
}

cudaError_t launch_probe_mode(int mode, double* out, int iters, int grid, cudaStream_t st) {
  static const cudaError_t attr = [] {  // once, thread-safely
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_probe<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, kProbeSmem))) return e;
    if ((e = cudaFuncSetAttribute(k_probe<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kProbeSmem))) return e;
    if ((e = cudaFuncSetAttribute(k_probe<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kProbeSmem))) return e;
    return cudaFuncSetAttribute(k_probe<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, kProbeSmem);
  }();
  if (attr != cudaSuccess) return attr;
  switch (mode) {
    case 0: k_probe<0><<<grid, kProbeThreads, kProbeSmem, st>>>(out, iters, 0.5f); break;
    case 1: k_probe<1><<<grid, kProbeThreads, kProbeSmem, st>>>(out, iters, 0.5f); break;
    case 2: k_probe<2><<<grid, kProbeThreads, kProbeSmem, st>>>(out, iters, 0.5f); break;
    default: k_probe<3><<<grid, kProbeThreads, kProbeSmem, st>>>(out, iters, 0.5f); break;
  }
  return cudaGetLastError();
}

}  // namespace gbkde
