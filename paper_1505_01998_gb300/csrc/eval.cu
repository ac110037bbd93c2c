// Consumers of a selected bandwidth: the density estimate at query points
// (Sec. 4.2, Eqs. kde-def-H, K_H) and the approximate Count / Sum of a
// numeric column over ranges (Sec. 4.3, Eqs. count, sum).
//
// kde_eval: the prologue (with a given H) checks and factors H = L L^T; one CTA
// item is a tile of 128 queries (4 per lane) against a chunk of samples staged
// in shared memory, both whitened by L^-1 relative to the tile's first query
// and scaled so that K_H(q - x) is proportional to 2^-|y_q - y_x|^2; per-query
// FP32 runs fold into Kahan pairs, item totals go to per-chunk FP64 rows
// reduced in fixed order.
// kde_aqp: for every sample and range, the exact integral of its Gaussian
// term over the range (normal cdf differences, tails taken from the nearer
// side); each CTA sorts its chunk of the column so that only the samples near
// a range's ends are evaluated one by one, the inside ones being counted and
// summed through prefix sums; FP64 across threads and CTAs.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "host.hpp"
#include "internal.cuh"

using namespace gbkde;

namespace {

constexpr double kPi = 3.14159265358979323846;
// Queries per lane: 8 for narrow samples (the per-sample shared-memory load
// and loop overhead spread over more evaluations), 4 for wide ones
// (registers).  A query tile is the 32 lanes' queries.
__host__ __device__ constexpr int qpl_of(int dk) { return dk <= 4 ? 8 : 4; }
__host__ __device__ constexpr int qtile_of(int dk) { return 32 * qpl_of(dk); }


// Every query tile t has a centre c_t (its first query).  Queries and samples
// are whitened relative to the centre of the tile they meet, so the FP32
// coordinates the pair loop subtracts are small near the query and the
// rounding of a squared distance is relative to the local, not the global,
// spread of the data.  Scale: sqrt(2) M, so that K_H(q - x) is proportional
// to 2^-|y_q - y_x|^2 (M = sqrt(log2(e)/4) L^-1, H = L L^T).
template <typename TIN>
__global__ void k_eval_queries(const DsDev* ds, const TIN* __restrict__ q, int64_t m, int64_t m_pad,
                               double* __restrict__ cent /* [q_tiles][KDE_MAX_D] */,
                               float* __restrict__ yq /* [dk][m_pad] */) {
  const int d = ds->d, dk = ds->dk, qt = qtile_of(dk);
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m_pad; j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = j / qt, j0 = t * qt;
    float c[KDE_MAX_D] = {};
    for (int k = 0; k < d; ++k) {
      const double ck = (double)q[(int64_t)k * m + j0];  // j0 < m: every tile starts with a query
      if (j == j0) cent[t * KDE_MAX_D + k] = ck;
      if (j < m) c[k] = (float)((double)q[(int64_t)k * m + j] - ck);
    }
    for (int k = 0; k < dk; ++k) {
      float v = 0.f;
      if (k < d)
        for (int i = 0; i <= k; ++i) v = fmaf(ds->M[k * KDE_MAX_D + i], c[i], v);
      yq[(int64_t)k * m_pad + j] = 1.41421356237309505f * v;
    }
  }
}

// Samples staged per pass: wide samples cap the shared memory, narrow ones
// take long passes (fewer barriers per evaluation).
template <int D>
constexpr int kStage = D <= 4 ? 2048 : 512;

// Shared-memory reads of staged samples: one float4 covers 4 / D samples for
// D = 1, 2, one sample for D = 4 k; D = 3 reads single floats.
template <int D>
struct SampleVec {
  static constexpr int per = D == 1 ? 4 : D == 2 ? 2 : 1;   // samples per read group
  static constexpr bool vec = (D % 4 == 0) || D == 1 || D == 2;
  static __device__ __forceinline__ void load(const float* p, float (&v)[per * D]) {
    if constexpr (vec) {
#pragma unroll
      for (int u = 0; u < per * D / 4; ++u) {
        const float4 t = reinterpret_cast<const float4*>(p)[u];
        v[4 * u] = t.x, v[4 * u + 1] = t.y, v[4 * u + 2] = t.z, v[4 * u + 3] = t.w;
      }
    } else {
#pragma unroll
      for (int k = 0; k < per * D; ++k) v[k] = p[k];
    }
  }
};

// One staged sample (negated, whitened: nf = -y_x) against the lane's queries.
template <int D, int NP>
__device__ __forceinline__ void eval_sample(const float* nf, const float2 (&yq2)[NP][D], float2 (&run)[NP]) {
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    float2 q = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const float2 dl = __fadd2_rn(yq2[p][k], make_float2(nf[k], nf[k]));
      q = __ffma2_rn(dl, dl, q);
    }
    run[p] = __fadd2_rn(run[p], make_float2(ex2_neg(q.x), ex2_neg(q.y)));
  }
}

// items: (query tile, sample chunk); part[chunk][m_pad] FP64.  Each staged
// sample is whitened against the tile's centre by the thread that loads it
// and stored negated, so the pair loop forms y_q - y_x with one packed add.
// Each lane holds QPL queries as FP32x2 pairs (lane + 32 i); each warp walks
// a contiguous slice of the staged samples with vector loads.
template <typename TIN, int D>
__global__ void __launch_bounds__(kThreads) k_eval(const DsDev* ds, const float* __restrict__ yq, int64_t m_pad,
                                                   int64_t q_tiles, int64_t chunk, int64_t n_chunks,
                                                   const double* __restrict__ cent,
                                                   double* __restrict__ part) {
  constexpr int ST = kStage<D>;
  constexpr int QPL = qpl_of(D), NP = QPL / 2, QT = 32 * QPL;
  constexpr bool kResident = D <= 4;  // queries stay in registers across passes
  using SV = SampleVec<D>;
  // staged samples during the passes, the per-warp query sums after them
  constexpr int kBuf = ST * D * 4 > kWarps * QT * 8 ? ST * D * 4 : kWarps * QT * 8;
  __shared__ __align__(16) unsigned char sBuf[kBuf];
  float* sS = reinterpret_cast<float*>(sBuf);
  double(*sRed)[QT] = reinterpret_cast<double(*)[QT]>(sBuf);
  __shared__ float sM[D * D];
  __shared__ TIN sC[D];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t n = ds->n;
  const int d = ds->d;
  const TIN* __restrict__ X = static_cast<const TIN*>(ds->x);
  for (int idx = threadIdx.x; idx < D * D; idx += kThreads) {
    const int k = idx / D, i = idx - k * D;
    // sqrt(2) M, negated: staged samples are -y_x
    sM[idx] = (k < d && i <= k) ? -1.41421356237309505f * ds->M[k * KDE_MAX_D + i] : 0.f;
  }
  const int64_t items = q_tiles * n_chunks;
  for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
    const int64_t qt = it % q_tiles, c = it / q_tiles;
    if (threadIdx.x < D) sC[threadIdx.x] = threadIdx.x < d ? (TIN)cent[qt * KDE_MAX_D + threadIdx.x] : TIN(0);
    float2 yq2[NP][D];  // pair p: queries lane + 64 p and lane + 64 p + 32 of the tile
    auto load_queries = [&]() {
#pragma unroll
      for (int p = 0; p < NP; ++p)
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const float* col = yq + (int64_t)k * m_pad + qt * QT + lane + 64 * p;
          yq2[p][k] = make_float2(col[0], col[32]);
        }
    };
    if (kResident) load_queries();
    float s[QPL], cc[QPL];
#pragma unroll
    for (int r = 0; r < QPL; ++r) s[r] = cc[r] = 0.f;
    const int64_t j0 = c * chunk, j1 = min(j0 + chunk, n);
    for (int64_t jb = j0; jb < j1; jb += ST) {
      const int cnt = (int)min((int64_t)ST, j1 - jb);
      __syncthreads();  // previous readers of sS done; sC, sM visible
#pragma unroll 1
      for (int jj = threadIdx.x; jj < cnt; jj += kThreads) {
        float u[D];
#pragma unroll
        for (int k = 0; k < D; ++k) u[k] = k < d ? (float)(X[(int64_t)k * n + jb + jj] - sC[k]) : 0.f;
        // M is re-read from shared memory per sample (volatile): hoisting its
        // D(D+1)/2 entries out of the loop would exhaust the registers at D = 16
        const volatile float* vM = sM;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          float v = 0.f;
#pragma unroll
          for (int i = 0; i <= k; ++i) v = fmaf(vM[k * D + i], u[i], v);
          sS[jj * D + k] = v;
        }
      }
      __syncthreads();
      if (!kResident) load_queries();  // not live while samples are whitened
      float2 run[NP];
#pragma unroll
      for (int p = 0; p < NP; ++p) run[p] = make_float2(0.f, 0.f);
      // warp w: samples [a, b), a contiguous slice in whole read groups
      const int slice = ((cnt + kWarps - 1) / kWarps + SV::per - 1) / SV::per * SV::per;
      const int a = min(cnt, warp * slice), b = min(cnt, a + slice);
      const int bv = a + (b - a) / SV::per * SV::per;
      constexpr int kUnroll = D > 4 ? 1 : 2;
#pragma unroll kUnroll
      for (int jj = a; jj < bv; jj += SV::per) {
        float v[SV::per * D];
        SV::load(sS + jj * D, v);
#pragma unroll
        for (int u = 0; u < SV::per; ++u) eval_sample<D, NP>(v + u * D, yq2, run);
      }
      for (int jj = bv; jj < b; ++jj) eval_sample<D, NP>(sS + jj * D, yq2, run);
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        kahan_add(s[2 * p], cc[2 * p], run[p].x);
        kahan_add(s[2 * p + 1], cc[2 * p + 1], run[p].y);
      }
    }
    // combine the 8 warps (each saw every query of the tile) in fixed order;
    // s[2p], s[2p + 1] hold queries lane + 64 p and lane + 64 p + 32
    __syncthreads();  // the sample buffer becomes sRed
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      sRed[warp][lane + 64 * p] = (double)s[2 * p] - (double)cc[2 * p];
      sRed[warp][lane + 64 * p + 32] = (double)s[2 * p + 1] - (double)cc[2 * p + 1];
    }
    __syncthreads();
    for (int qq = threadIdx.x; qq < QT; qq += kThreads) {
      double t = 0.0;
      for (int w = 0; w < kWarps; ++w) t += sRed[w][qq];
      part[c * m_pad + qt * QT + qq] = t;
    }
  }
}

__global__ void k_eval_finish(const DsDev* ds, const double* __restrict__ part, int64_t m, int64_t m_pad,
                              int64_t n_chunks, double* __restrict__ f) {
  const int d = ds->d;
  const double C = pow(2.0 * kPi, -0.5 * d) * exp(-0.5 * ds->logdet) / (double)ds->n;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
    double t = 0.0;
    for (int64_t c = 0; c < n_chunks; ++c) t += part[c * m_pad + j];
    f[j] = C * t;
  }
}

// Phi(b) - Phi(a) for a <= b, taken from the side with the smaller tails.
__device__ __forceinline__ float cdf_diff(float a, float b) {
  const float r = 0.70710678118654752f;
  if (a >= 0.f) return 0.5f * (erfcf(a * r) - erfcf(b * r));
  if (b <= 0.f) return 0.5f * (erfcf(-b * r) - erfcf(-a * r));
  return 1.f - 0.5f * (erfcf(b * r) + erfcf(-a * r));
}

// Beyond this many bandwidths from a range's end a sample's Gaussian lies on
// one side of it up to Phi(-7) = 1.3e-12 of its mass (phi(7) = 9.1e-12), far
// below the FP32 rounding of a term: that end contributes 0 or 1 to the cdf
// difference and nothing to the pdf difference.
constexpr float kAqpFar = 7.f;
constexpr int kAqpChunk = 8192;  // samples per CTA, sorted in shared memory (96 KB with the prefix sums)

// Count / Sum terms of one sample and range from the normal cdf and pdf.
// With one end far (the usual case) one tail and one pdf suffice, sharing an
// exponential: for a far upper end P = Phi(inf) - Phi(a) = Q(a) and only
// phi(a) remains; for a far lower end P = Phi(b) = Q(-b) and only -phi(b)
// remains.  Both take the same instructions (t = a or -b), so the warp does
// not diverge between them.
// The upper tail Q(t) = erfc(t / sqrt 2) / 2 of the standard normal and the
// exponential e = exp(-t^2 / 2) of its pdf, sharing that exponential: for
// u = |t| / sqrt 2, erfc(u) = (a1 s + ... + a5 s^5) exp(-u^2), s = 1 / (1 + p u),
// the rational approximation of Hastings (Abramowitz & Stegun 7.1.26,
// absolute error of erfc below 1.5e-7; 3e-7 for Q in FP32), and
// Q(-t) = 1 - Q(t).
constexpr float kAsP = 0.3275911f, kAsA1 = 0.254829592f, kAsA2 = -0.284496736f, kAsA3 = 1.421413741f,
                kAsA4 = -1.453152027f, kAsA5 = 1.061405429f;

__device__ __forceinline__ float normal_upper_tail(float t, float& e) {
  const float u = fabsf(t) * 0.70710678118654752f;
  e = expf(-u * u);
  const float sd = __fdividef(1.f, fmaf(kAsP, u, 1.f));
  const float poly = sd * fmaf(sd, fmaf(sd, fmaf(sd, fmaf(sd, kAsA5, kAsA4), kAsA3), kAsA2), kAsA1);
  const float q = 0.5f * poly * e;
  return t >= 0.f ? q : 1.f - q;
}

__device__ __forceinline__ void aqp_full(float xi, float lo, float hi, float inv_h, float h_phi,
                                         float& cnt, float& sum) {
  const float a = (lo - xi) * inv_h, b = (hi - xi) * inv_h;
  const bool up_far = b >= kAqpFar, lo_far = a <= -kAqpFar;
  float P, dphi;
  if (up_far || lo_far) {
    const float t = up_far ? a : -b;
    float e;
    P = normal_upper_tail(t, e);
    dphi = up_far ? e : -e;
  } else {
    P = cdf_diff(a, b);
    // phi(a) - phi(b) as one difference of exponentials: exactly 0 when a == b
    dphi = expf(-0.5f * a * a) - expf(-0.5f * b * b);
  }
  cnt += P;
  sum += fmaf(xi, P, h_phi * dphi);
}

// Sorted keys live in shared memory with one padding slot after every 32
// (element i at i + i/32), so that the per-thread blocks of 8..32 consecutive
// keys of the register stages are read and written without bank conflicts.
__device__ __forceinline__ int kp(int i) { return i + (i >> 5); }

// Bitonic sort of key[0, n2) in shared memory (n2 a power of two), one
// compare-exchange stage per barrier.
__device__ __forceinline__ void bitonic_sort_smem(float* key, int n2) {
  for (int k = 2; k <= n2; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < n2; i += kThreads) {
        const int p = i ^ j;
        if (p > i) {
          const float u = key[kp(i)], v = key[kp(p)];
          if ((u > v) == ((i & k) == 0)) {
            key[kp(i)] = v;
            key[kp(p)] = u;
          }
        }
      }
      __syncthreads();
    }
}

// The same network with n2 = PER * kThreads: each thread holds PER
// consecutive keys in registers; the stages whose partner distance j is
// below PER stay inside a thread (no barrier), the others go through shared
// memory.  Same compare-exchanges, same result.
template <int PER>
__device__ __forceinline__ void bitonic_sort_regs(float* key, int n2) {
  const int base = (int)threadIdx.x * PER;
  float e[PER];
#pragma unroll
  for (int a = 0; a < PER; ++a) e[a] = key[kp(base + a)];
  for (int k = 2; k <= n2; k <<= 1) {
    if ((k >> 1) >= PER) {
#pragma unroll
      for (int a = 0; a < PER; ++a) key[kp(base + a)] = e[a];
      __syncthreads();
      for (int j = k >> 1; j >= PER; j >>= 1) {
        for (int q = threadIdx.x; q < n2 / 2; q += kThreads) {
          const int i = (q / j) * 2 * j + (q % j), p = i + j;
          const float u = key[kp(i)], v = key[kp(p)];
          if ((u > v) == ((i & k) == 0)) {
            key[kp(i)] = v;
            key[kp(p)] = u;
          }
        }
        __syncthreads();
      }
#pragma unroll
      for (int a = 0; a < PER; ++a) e[a] = key[kp(base + a)];
    }
#pragma unroll
    for (int j = PER / 2; j >= 1; j >>= 1) {
      if (j <= (k >> 1)) {
#pragma unroll
        for (int a = 0; a < PER; ++a) {
          const int b = a ^ j;
          if (b > a) {
            const float u = e[a], v = e[b];
            if ((u > v) == (((base + a) & k) == 0)) {
              e[a] = v;
              e[b] = u;
            }
          }
        }
      }
    }
  }
#pragma unroll
  for (int a = 0; a < PER; ++a) key[kp(base + a)] = e[a];
  __syncthreads();
}

// One CTA per chunk of samples, staged in shared memory as FP32 and sorted
// (bitonic), with FP64 prefix sums of the sorted values.  Per range, one
// warp finds by binary search the samples within kAqpFar bandwidths of each
// end (t1 = lo - 7h, t2 = lo + 7h, t3 = hi - 7h, t4 = hi + 7h): those are
// evaluated one by one; the samples between the two windows lie inside the
// range (count: their number, sum: a difference of prefix sums), those
// beyond them outside.  The work per range is two logarithmic searches plus
// the samples near its ends, instead of every sample.  Per-lane FP32 runs,
// FP64 across lanes; part[chunk][range][2].
template <typename TIN>
__global__ void __launch_bounds__(kThreads) k_aqp(const TIN* __restrict__ x, int64_t n, float h,
                                                  const float* __restrict__ rng /* [m][2] */, int m,
                                                  int64_t chunk, double* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char aqp_smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i0 = blockIdx.x * chunk;
  const int cnt = (int)min(chunk, n - i0);
  int n2 = 32;
  while (n2 < cnt) n2 <<= 1;
  double* pre = reinterpret_cast<double*>(aqp_smem);                          // [cnt + 1]
  float* key = reinterpret_cast<float*>(aqp_smem + ((size_t)(cnt + 1) * 8 + 15) / 16 * 16);  // [n2 + n2/32], padded
  __shared__ double sScan[kWarps];
  for (int i = threadIdx.x; i < n2; i += kThreads) key[kp(i)] = i < cnt ? (float)x[i0 + i] : INFINITY;
  __syncthreads();
  // ---- bitonic sort, ascending
  if (n2 == 8 * kThreads)
    bitonic_sort_regs<8>(key, n2);
  else if (n2 == 16 * kThreads)
    bitonic_sort_regs<16>(key, n2);
  else if (n2 == 32 * kThreads)
    bitonic_sort_regs<32>(key, n2);
  else
    bitonic_sort_smem(key, n2);
  // ---- FP64 prefix sums: pre[i] = key[0] + ... + key[i-1]
  {
    const int per = (cnt + kThreads - 1) / kThreads;
    const int b0 = min(cnt, (int)threadIdx.x * per), b1 = min(cnt, b0 + per);
    double run = 0.0;
    for (int i = b0; i < b1; ++i) run += (double)key[kp(i)];
    double incl = run;  // inclusive scan of the thread totals within the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) sScan[warp] = incl;
    __syncthreads();
    double base = incl - run;
    for (int w = 0; w < warp; ++w) base += sScan[w];
    if (threadIdx.x == 0) pre[0] = 0.0;
    for (int i = b0; i < b1; ++i) {
      base += (double)key[kp(i)];
      pre[i + 1] = base;
    }
  }
  __syncthreads();
  const float inv_h = 1.f / h, h_phi = h * 0.39894228040143268f;  // h / sqrt(2 pi)
  const float fh = kAqpFar * h;
  for (int g = warp; g < m; g += kWarps) {
    const float lo = rng[2 * g], hi = rng[2 * g + 1];
    // lanes 0..3: first index with key >= t_(lane+1)
    float t = lo - fh;
    if (lane == 1) t = lo + fh;
    if (lane == 2) t = hi - fh;
    if (lane == 3) t = hi + fh;
    int lb = 0, ub = cnt;
    while (lb < ub) {
      const int mid = (lb + ub) >> 1;
      if (key[kp(mid)] < t) lb = mid + 1; else ub = mid;
    }
    const int i1 = __shfl_sync(0xffffffffu, lb, 0), i2 = __shfl_sync(0xffffffffu, lb, 1);
    const int i3 = __shfl_sync(0xffffffffu, lb, 2), i4 = __shfl_sync(0xffffffffu, lb, 3);
    float c_run = 0.f, s_run = 0.f;
    double c_in = 0.0, s_in = 0.0;
    if (lo + fh <= hi - fh) {  // two windows around the ends, the inside between them
      for (int i = i1 + lane; i < i2; i += 32) aqp_full(key[kp(i)], lo, hi, inv_h, h_phi, c_run, s_run);
      for (int i = i3 + lane; i < i4; i += 32) aqp_full(key[kp(i)], lo, hi, inv_h, h_phi, c_run, s_run);
      if (lane == 0 && i3 > i2) {
        c_in = (double)(i3 - i2);
        s_in = pre[i3] - pre[i2];
      }
    } else {  // a narrow range: one window over both ends
      for (int i = i1 + lane; i < i4; i += 32) aqp_full(key[kp(i)], lo, hi, inv_h, h_phi, c_run, s_run);
    }
    const float2 vc = warp_sum_ff(c_run, 0.f), vs = warp_sum_ff(s_run, 0.f);
    if (lane == 0) {
      part[((int64_t)blockIdx.x * m + g) * 2] = ff_value(vc) + c_in;
      part[((int64_t)blockIdx.x * m + g) * 2 + 1] = ff_value(vs) + s_in;
    }
  }
}

size_t aqp_smem_bytes(int64_t chunk) {
  int n2 = 32;
  while (n2 < chunk) n2 <<= 1;
  return ((size_t)(chunk + 1) * 8 + 15) / 16 * 16 + (size_t)(n2 + n2 / 32) * 4;
}

__global__ void k_aqp_finish(const double* __restrict__ part, int m, int64_t chunks, double* __restrict__ out) {
  for (int j = threadIdx.x; j < 2 * m; j += blockDim.x) {
    double t = 0.0;
    for (int64_t c = 0; c < chunks; ++c) t += part[c * 2 * m + j];
    out[j] = t;
  }
}

struct EvalLayout {
  Geometry g;
  int64_t m_pad, q_tiles, chunk, n_chunks;
  size_t off_yq, off_cent, off_part, off_f, total;
};

int eval_layout(int64_t n, int d, int64_t m, int sms, EvalLayout* L) {
  int rc = make_geometry(n, d, 1, nullptr, sms, &L->g);
  if (rc) return rc;
  const int qt = qtile_of(L->g.dk);
  L->m_pad = (m + qt - 1) / qt * qt;
  L->q_tiles = L->m_pad / qt;
  // sample chunks (multiples of 256): about 16 items per SM over the launch.
  // Finer chunks balance the last round better but cost more per-item work
  // (staging, reductions): 64 items per SM measured 4 % slower at d = 1.
  const int64_t want = std::max<int64_t>(1, (16 * (int64_t)std::max(1, sms) + L->q_tiles - 1) / L->q_tiles);
  L->chunk = std::max<int64_t>(256, ((n + want - 1) / want + 255) / 256 * 256);
  L->n_chunks = (n + L->chunk - 1) / L->chunk;
  size_t o = (L->g.total + 255) / 256 * 256;
  L->off_yq = o;
  o += ((size_t)L->g.dk * L->m_pad * 4 + 255) / 256 * 256;
  L->off_cent = o;
  o += ((size_t)L->q_tiles * KDE_MAX_D * 8 + 255) / 256 * 256;
  L->off_part = o;
  o += ((size_t)L->n_chunks * L->m_pad * 8 + 255) / 256 * 256;
  L->off_f = o;
  o += ((size_t)m * 8 + 255) / 256 * 256;
  L->total = o;
  return KDE_OK;
}

// Persistent grid: every CTA that fits on the device at once (occupancy of
// this instance, looked up once), at most one per item.
template <typename TIN, int D>
cudaError_t eval_launch(cudaStream_t st, const DsDev* ds, const float* yq, const EvalLayout& L,
                        const double* cent, double* part) {
  struct Occupancy {
    cudaError_t e;
    int per_sm;
  };
  // looked up once per instance (thread-safe initialisation of a local static)
  static const Occupancy occ = [] {
    Occupancy o{cudaSuccess, 0};
    o.e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o.per_sm, k_eval<TIN, D>, kThreads, 0);
    o.per_sm = std::max(1, o.per_sm);
    return o;
  }();
  if (occ.e != cudaSuccess) return occ.e;
  const int64_t items = L.q_tiles * L.n_chunks;
  const int grid = (int)std::min<int64_t>(items, (int64_t)std::max(1, device_sms()) * occ.per_sm);
  k_eval<TIN, D><<<grid, kThreads, 0, st>>>(ds, yq, L.m_pad, L.q_tiles, L.chunk, L.n_chunks, cent, part);
  return cudaGetLastError();
}

template <typename TIN>
cudaError_t eval_dispatch(int dk, cudaStream_t st, const DsDev* ds, const float* yq,
                          const EvalLayout& L, const double* cent, double* part) {
  switch (dk) {
    case 1: return eval_launch<TIN, 1>(st, ds, yq, L, cent, part);
    case 2: return eval_launch<TIN, 2>(st, ds, yq, L, cent, part);
    case 3: return eval_launch<TIN, 3>(st, ds, yq, L, cent, part);
    case 4: return eval_launch<TIN, 4>(st, ds, yq, L, cent, part);
    case 8: return eval_launch<TIN, 8>(st, ds, yq, L, cent, part);
    case 12: return eval_launch<TIN, 12>(st, ds, yq, L, cent, part);
    default: return eval_launch<TIN, 16>(st, ds, yq, L, cent, part);
  }
}

struct AqpLayout {
  int64_t chunk, chunks;
  size_t off_part, off_out, total;
};

// One CTA per chunk of at most kAqpChunk samples; chunks sized so that the
// CTAs come in whole waves of 2 per SM (the shared-memory occupancy).
AqpLayout aqp_layout(int64_t n, int m, int sms) {
  AqpLayout L;
  const int64_t ctas = (int64_t)std::max(1, sms) * 2;
  const int64_t waves = std::max<int64_t>(1, (n + ctas * kAqpChunk - 1) / (ctas * kAqpChunk));
  L.chunk = std::min<int64_t>(kAqpChunk, ((n + waves * ctas - 1) / (waves * ctas) + 31) / 32 * 32);
  L.chunk = std::max<int64_t>(L.chunk, kThreads);
  L.chunks = (n + L.chunk - 1) / L.chunk;
  L.off_part = ((size_t)m * 2 * sizeof(float) + 255) / 256 * 256;
  L.off_out = L.off_part + ((size_t)L.chunks * m * 2 * sizeof(double) + 255) / 256 * 256;
  L.total = L.off_out + ((size_t)m * 2 * sizeof(double) + 255) / 256 * 256;
  return L;
}

}  // namespace

extern "C" {

int kde_eval_workspace_size(int64_t n, int d, int64_t m, size_t* bytes) {
  if (!bytes || n < 2 || d < 1 || d > KDE_MAX_D || m < 1) return fail(KDE_EINVAL, "kde_eval_workspace_size: bad arguments");
  EvalLayout L;
  int rc = eval_layout(n, d, m, device_sms(), &L);
  if (rc) return rc;
  *bytes = L.total;
  return KDE_OK;
}

int kde_eval(const void* x_dev, int dtype, int64_t n, int d, const double* H_host, const void* q_dev,
             int64_t m, void* ws, size_t ws_bytes, void* stream, double* f_host) {
  int rc = check_common(x_dev, dtype, n, d, ws);
  if (rc) return rc;
  if (!H_host || !q_dev || !f_host || m < 1) return fail(KDE_EINVAL, "kde_eval: H, q, f or m");
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < d; ++b)
      if (!std::isfinite(H_host[a * d + b]) || H_host[a * d + b] != H_host[b * d + a])
        return fail(KDE_EINVAL, "kde_eval: H not finite and symmetric");
  EvalLayout L;
  rc = eval_layout(n, d, m, device_sms(), &L);
  if (rc) return rc;
  if (ws_bytes < L.total) return fail(KDE_ENOMEM, "workspace %zu bytes < %zu needed", ws_bytes, L.total);
  cudaStream_t st = (cudaStream_t)stream;
  unsigned char* w = static_cast<unsigned char*>(ws);
  DsDev init = make_desc(L.g, x_dev, dtype, KDE_METHOD_LSCV, w);
  init.given_H = 1;
  init.y = nullptr;  // the prologue only checks and factors H; k_eval whitens per query tile
  init.xc = nullptr;
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < d; ++b) init.cov[a * d + b] = H_host[a * d + b];
  DsDev* ds = reinterpret_cast<DsDev*>(w + L.g.off_ds);
  int64_t* off = reinterpret_cast<int64_t*>(w + L.g.off_off);
  const double one = 1.0;
  const int64_t offs[4] = {0, 0, 0, 0};
  float* yq = reinterpret_cast<float*>(w + L.off_yq);
  double* cent = reinterpret_cast<double*>(w + L.off_cent);
  double* part = reinterpret_cast<double*>(w + L.off_part);
  double* f = reinterpret_cast<double*>(w + L.off_f);
  cudaError_t e = launch_setup(ds, init, &one, 1, off, offs, 4, st);
  if (e == cudaSuccess) e = launch_prep(ds, 1, nullptr, L.g.prep_parts, st);
  if (e == cudaSuccess) {
    const int blocks = (int)std::min<int64_t>(1024, (L.m_pad + 255) / 256);
    if (dtype == KDE_F64)
      k_eval_queries<double><<<blocks, 256, 0, st>>>(ds, static_cast<const double*>(q_dev), m, L.m_pad, cent, yq);
    else
      k_eval_queries<float><<<blocks, 256, 0, st>>>(ds, static_cast<const float*>(q_dev), m, L.m_pad, cent, yq);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    e = mark_event(0, st);
    if (e == cudaSuccess)
      e = dtype == KDE_F64 ? eval_dispatch<double>(L.g.dk, st, ds, yq, L, cent, part)
                           : eval_dispatch<float>(L.g.dk, st, ds, yq, L, cent, part);
    if (e == cudaSuccess) e = mark_event(1, st);
  }
  if (e == cudaSuccess) {
    k_eval_finish<<<(int)std::min<int64_t>(1024, (m + 255) / 256), 256, 0, st>>>(ds, part, m, L.m_pad, L.n_chunks, f);
    e = cudaGetLastError();
  }
  kde_result r;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&r, w + L.g.off_ds + offsetof(DsDev, res), sizeof(r), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(f_host, f, sizeof(double) * m, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "kde_eval");
  if (r.status != KDE_OK) return fail(r.status, "kde_eval: %s", kde_status_string(r.status));
  return KDE_OK;
}

int kde_aqp_workspace_size(int64_t n, int m, size_t* bytes) {
  if (!bytes || n < 2 || m < 1 || m > KDE_MAX_NH) return fail(KDE_EINVAL, "kde_aqp_workspace_size: bad arguments");
  *bytes = aqp_layout(n, m, device_sms()).total;
  return KDE_OK;
}

int kde_aqp(const void* x_dev, int dtype, int64_t n, double h, const double* lo_host,
            const double* hi_host, int m, void* ws, size_t ws_bytes, void* stream, double* count_host,
            double* sum_host) {
  int rc = check_common(x_dev, dtype, n, 1, ws);
  if (rc) return rc;
  if (!lo_host || !hi_host || m < 1 || m > KDE_MAX_NH || !(h > 0) || !std::isfinite(h))
    return fail(KDE_EINVAL, "kde_aqp: ranges, m or h");
  for (int k = 0; k < m; ++k)
    if (!(lo_host[k] <= hi_host[k])) return fail(KDE_EINVAL, "kde_aqp: range %d has lo > hi or a NaN bound", k);
  const AqpLayout L = aqp_layout(n, m, device_sms());
  const int64_t chunk = L.chunk, chunks = L.chunks;
  if (ws_bytes < L.total) return fail(KDE_ENOMEM, "workspace %zu bytes < %zu needed", ws_bytes, L.total);
  unsigned char* w = static_cast<unsigned char*>(ws);
  float* rng = reinterpret_cast<float*>(w);
  double* part = reinterpret_cast<double*>(w + L.off_part);
  double* out = reinterpret_cast<double*>(w + L.off_out);
  std::vector<float> r2(2 * m);
  for (int k = 0; k < m; ++k) {
    r2[2 * k] = (float)lo_host[k];
    r2[2 * k + 1] = (float)hi_host[k];
  }
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(rng, r2.data(), sizeof(float) * 2 * m, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = mark_event(0, st);
  const size_t smem = aqp_smem_bytes(chunk);
  static const cudaError_t attr = [] {  // once, thread-safely
    const int mx = (int)aqp_smem_bytes(kAqpChunk);
    cudaError_t a = cudaFuncSetAttribute(k_aqp<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (a == cudaSuccess) a = cudaFuncSetAttribute(k_aqp<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    return a;
  }();
  if (e == cudaSuccess) e = attr;
  if (e == cudaSuccess) {
    if (dtype == KDE_F64)
      k_aqp<double><<<(int)chunks, kThreads, smem, st>>>(static_cast<const double*>(x_dev), n, (float)h, rng, m, chunk, part);
    else
      k_aqp<float><<<(int)chunks, kThreads, smem, st>>>(static_cast<const float*>(x_dev), n, (float)h, rng, m, chunk, part);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = mark_event(1, st);
  if (e == cudaSuccess) {
    k_aqp_finish<<<1, 256, 0, st>>>(part, m, chunks, out);
    e = cudaGetLastError();
  }
  std::vector<double> res(2 * m);
  if (e == cudaSuccess) e = cudaMemcpyAsync(res.data(), out, sizeof(double) * 2 * m, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "kde_aqp");
  for (int k = 0; k < m; ++k) {
    if (count_host) count_host[k] = res[2 * k];
    if (sum_host) sum_host[k] = res[2 * k + 1];
  }
  return KDE_OK;
}

}  // extern "C"
