// Fused all-pairs, all-bandwidths LSCV kernel and its reductions.
//
// For every pair i < j of a dataset and every grid multiplier h it accumulates
//   S1(h) = sum exp(-S(v)/(4 h^2)),   S2(h) = sum exp(-S(v)/(2 h^2)) = sum e^2,
// from which g(h) = h^-d A [2 n^-2 (S1 - 2^(1+d/2) S2) + n^-1] (Sec. 4.4.2,
// Eqs. LSCV-gh, LSCV-Tx, LSCV-Kx, LSCV-KKx with A = (4 pi)^(-d/2)|S|^(-1/2)).
// S(v) = v^T S^-1 v (Eq. LSCV_MOD-Pv) is formed once per pair from samples
// whitened on the device (y = sqrt(log2 e / 4) L^-1 (x - mean), S = L L^T), so
// Q = |y_i - y_j|^2 and e = 2^(-Q/h^2).  The paper precomputes and stores all
// n(n-1)/2 values S(v) and re-reads them once per h (Sec. 5.5, Sec. 6.2); here
// the value lives in a register and feeds a whole chunk of bandwidths.
//
// Work decomposition: the pair triangle is cut into T x T tiles numbered by
// the tile map of Sec. 5.4.2; an item is K consecutive tiles times one group
// of up to 8 chunks of B bandwidths.  A persistent CTA of 8 warps takes items
// in a grid-stride loop; each warp owns one chunk of B bandwidths (and a
// column slice of the tile when a group has fewer than 8 chunks); each lane
// holds R row samples in registers and walks the column samples staged in
// shared memory (broadcast reads).  Per-thread sums: FP32 runs over a tile,
// folded into Kahan-compensated FP32 accumulators; a warp's item total is a
// double-float butterfly in FP32, written as FP64.  Every item writes its
// own partial row, and rows are added in a fixed order, so results do not
// depend on the grid size or on which CTA ran an item.
//
// Variants: on a grid with n_h/8 points per octave of 1/h^2 (the default
// grid) the octave kernel takes 3/8 ex2 per evaluation and squares the rest
// down the octaves; the direct kernel (any grid) takes one ex2 per
// evaluation; grids of one or two points with wide samples (d > 4) walk
// their items one warp per item (k_lscv_warp).
#include "internal.cuh"

namespace gbkde {

namespace {

template <int D>
struct DPad {
  static constexpr int value = (D == 3) ? 4 : D;
};

// Shapes whose squared distances are formed two rows at a time in packed
// FP32x2 (d = 4 with 4 rows per lane): the column tile is staged as
// negated, duplicated pairs (-v, -v), so a difference is one packed add and
// the square-accumulate one packed FMA, half the scalar instructions.
// Measured at n = 16,384 with 128 bandwidths: d = 4 +2 %; d = 3 no change and
// d = 2 -2.4 % (its scalar path walks two columns per 16-byte load), so only
// d = 4 takes it.
template <int D, int R, bool OCT = false>
constexpr bool kPackedQ = (R == 4 && D == 4 && !OCT);

// Wide samples (d > 4, one row per lane; the column tile holds -v): the
// squared distance to column `col` in packed FP32x2 over coordinate pairs,
// two independent chains joined by one add.
template <int DP>
__device__ __forceinline__ float wide_q(const float* __restrict__ sF, int col, const float2 (&y2)[DP / 2]) {
  float2 s2 = make_float2(0.f, 0.f);
#pragma unroll
  for (int u = 0; u < DP / 4; ++u) {
    const float4 v = *reinterpret_cast<const float4*>(sF + col * DP + 4 * u);
    const float2 d0 = __fadd2_rn(y2[2 * u], make_float2(v.x, v.y));
    const float2 d1 = __fadd2_rn(y2[2 * u + 1], make_float2(v.z, v.w));
    s2 = __ffma2_rn(d0, d0, s2);
    s2 = __ffma2_rn(d1, d1, s2);
  }
  return __fadd_rn(s2.x, s2.y);
}

// a * 2^k by an integer add to the exponent field (ALU pipe instead of an
// FP32 multiply).  Exact for normal a whose exponent stays below 255; maps
// -0 and subnormals to values of magnitude below 2^-120, whose ex2 is 1 as
// that of the exact product is.  The octave kernel guarantees |a| < 2^105
// (finite edge mask 2^64, |1/h^2| <= 2^40; see kOctMask).
template <int K>
__device__ __forceinline__ float mul_pow2(float a) {
  return __int_as_float(__float_as_int(a) + (K << 23));
}

// Squared distance given to masked pairs of the octave kernel (diagonal
// tiles, ragged tail): finite, so that the exponent adds of octave_terms
// stay exact, and large enough that 2^64 * |c| >= 2^24 for every grid value
// c = -1/h^2 admitted (|c| in [2^-40, 2^40]): every term is then exactly 0.
constexpr float kOctMask = 18446744073709551616.0f;  // 2^64

// The octave grid's 16 terms of one pair (two residues x 8 octaves) from its
// squared distance qv: three chains per residue, each one ex2 and two
// squarings down (7 -> 6 -> 5, 4 -> 3 -> 2, 1 -> 0 -> one octave below 0);
// the last square of a chain feeds only its sum (FFMA2).  The arguments of
// octaves 4 and 1 are 8 and 64 times that of octave 7 (3 and 6 octaves of
// 1/h^2 up), formed by exponent adds.
__device__ __forceinline__ void octave_terms(float qv, const float2 (&nca)[3], float2 (&acc)[9]) {
  const float2 q2 = make_float2(qv, qv);
  const float2 a7 = __fmul2_rn(q2, nca[0]);
  const float2 a4 = make_float2(mul_pow2<3>(a7.x), mul_pow2<3>(a7.y));
  const float2 a1 = make_float2(mul_pow2<6>(a7.x), mul_pow2<6>(a7.y));
  const float2 e7 = make_float2(ex2(a7.x), ex2(a7.y));
  const float2 e4 = make_float2(ex2(a4.x), ex2(a4.y));
  const float2 e1 = make_float2(ex2(a1.x), ex2(a1.y));
  const float2 e6 = __fmul2_rn(e7, e7), e3 = __fmul2_rn(e4, e4), e0 = __fmul2_rn(e1, e1);
  acc[7] = __fadd2_rn(acc[7], e7);
  acc[6] = __fadd2_rn(acc[6], e6);
  acc[5] = __ffma2_rn(e6, e6, acc[5]);
  acc[4] = __fadd2_rn(acc[4], e4);
  acc[3] = __fadd2_rn(acc[3], e3);
  acc[2] = __ffma2_rn(e3, e3, acc[2]);
  acc[1] = __fadd2_rn(acc[1], e1);
  acc[0] = __fadd2_rn(acc[0], e0);
  acc[8] = __ffma2_rn(e0, e0, acc[8]);
}

// Columns [j_lo, j_hi) of one tile for this lane's R rows and B bandwidths.
// Bandwidths are processed in pairs with packed FP32x2 arithmetic.  ONE (a
// grid of one bandwidth, B = 2, both halves of nc2[0] holding it): the two
// halves of a packed evaluation take two pairs at that bandwidth instead of
// a real and a padding bandwidth -- rows 2p, 2p + 1 (R even) or the two
// columns of an iteration (wide samples) -- so t1/t2 .x and .y hold sums
// of the same bandwidth over different pairs: half the exponentials and
// bandwidth lane-operations of the padded form.
template <int D, int B, int R, bool EDGE, bool ONE = false>
__device__ __forceinline__ void lscv_columns(const float* __restrict__ sF, int j_lo, int j_hi,
                                             const float (&y)[R][D], const float2 (&nc2)[B / 2],
                                             float2 (&t1)[B / 2], float2 (&t2)[B / 2],
                                             int64_t i0, int64_t jg0, int64_t n) {
  constexpr int DP = DPad<D>::value;
  static_assert(!ONE || (B == 2 && (D > 4 || R % 2 == 0)), "one-bandwidth pairing: B = 2, rows two by two");
  if constexpr (kPackedQ<D, R>) {
    // sF holds float2 (-v, -v) per coordinate: [T][DP]
    const float2* __restrict__ sF2 = reinterpret_cast<const float2*>(sF);
    float2 y2[R / 2][D];
#pragma unroll
    for (int p = 0; p < R / 2; ++p)
#pragma unroll
      for (int k = 0; k < D; ++k) y2[p][k] = make_float2(y[2 * p][k], y[2 * p + 1][k]);
#pragma unroll 1
    for (int jj = j_lo; jj < j_hi; ++jj) {
      float2 nv[DP];
#pragma unroll
      for (int u = 0; u < DP / 2; ++u) {
        const float4 v = reinterpret_cast<const float4*>(sF2 + jj * DP)[u];
        nv[2 * u] = make_float2(v.x, v.y);
        nv[2 * u + 1] = make_float2(v.z, v.w);
      }
      float2 q2[R];
#pragma unroll
      for (int p = 0; p < R / 2; ++p) {
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const float2 dl = __fadd2_rn(y2[p][k], nv[k]);
          acc = __ffma2_rn(dl, dl, acc);
        }
        float qa = acc.x, qb = acc.y;
        if (EDGE) {
          const int64_t ia = i0 + 64 * p, ib = ia + 32, j = jg0 + jj;
          if (!(ia < j && j < n)) qa = __int_as_float(0x7f800000);  // +inf -> e = 0
          if (!(ib < j && j < n)) qb = __int_as_float(0x7f800000);
        }
        q2[2 * p] = ONE ? make_float2(qa, qb) : make_float2(qa, qa);
        q2[2 * p + 1] = make_float2(qb, qb);
      }
#pragma unroll
      for (int r = 0; r < R; r += (ONE ? 2 : 1)) {
#pragma unroll
        for (int bp = 0; bp < B / 2; ++bp) {
          const float2 a = __fmul2_rn(q2[r], nc2[bp]);
          const float2 e = make_float2(ex2(a.x), ex2(a.y));
          t1[bp] = __fadd2_rn(t1[bp], e);
          t2[bp] = __ffma2_rn(e, e, t2[bp]);
        }
      }
    }
    return;
  }
  if constexpr (D > 4) {
    // wide samples, one row per lane: sF holds -v.  Two columns per
    // iteration, each squared distance in packed FP32x2 over coordinate
    // pairs (two independent chains joined by one add), so that a warp has
    // four chains in flight instead of one.  Slices of columns are even.
    static_assert(R == 1 && DP % 4 == 0, "wide path: one row per lane");
    float2 y2[DP / 2];
#pragma unroll
    for (int k = 0; k < DP / 2; ++k) y2[k] = make_float2(y[0][2 * k], y[0][2 * k + 1]);
#pragma unroll 1
    for (int jj = j_lo; jj < j_hi; jj += 2) {
      float2 q2[2];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        float qv = wide_q<DP>(sF, jj + c, y2);
        if (EDGE) {
          const int64_t j = jg0 + jj + c;
          if (!(i0 < j && j < n)) qv = __int_as_float(0x7f800000);  // +inf -> e = 0
        }
        q2[c] = make_float2(qv, qv);
      }
      if (ONE) q2[0].y = q2[1].x;
#pragma unroll
      for (int c = 0; c < (ONE ? 1 : 2); ++c)
#pragma unroll
        for (int bp = 0; bp < B / 2; ++bp) {
          const float2 a = __fmul2_rn(q2[c], nc2[bp]);
          const float2 e = make_float2(ex2(a.x), ex2(a.y));
          t1[bp] = __fadd2_rn(t1[bp], e);
          t2[bp] = __ffma2_rn(e, e, t2[bp]);
        }
    }
    return;
  }
  constexpr int CPI = DP <= 4 ? 4 / DP : 1;  // columns per iteration
  constexpr int NV = CPI * DP / 4;           // 16-byte shared-memory loads per iteration
#pragma unroll 1
  for (int jj = j_lo; jj < j_hi; jj += CPI) {
    float vv[4 * NV];
#pragma unroll
    for (int u = 0; u < NV; ++u) {
      const float4 v = *reinterpret_cast<const float4*>(sF + jj * DP + 4 * u);
      vv[4 * u] = v.x;
      vv[4 * u + 1] = v.y;
      vv[4 * u + 2] = v.z;
      vv[4 * u + 3] = v.w;
    }
#pragma unroll
    for (int c = 0; c < CPI; ++c) {
      float2 q2[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const float dl = y[r][k] - vv[c * DP + k];
          acc = fmaf(dl, dl, acc);
        }
        if (EDGE) {
          const int64_t i = i0 + 32 * r, j = jg0 + jj + c;
          if (!(i < j && j < n)) acc = __int_as_float(0x7f800000);  // +inf -> e = 0
        }
        q2[r] = make_float2(acc, acc);
      }
      if constexpr (ONE && R % 2 == 0) {
#pragma unroll
        for (int r = 0; r < R; r += 2) q2[r].y = q2[r + 1].x;
      }
#pragma unroll
      for (int r = 0; r < R; r += (ONE ? 2 : 1)) {
#pragma unroll
        for (int bp = 0; bp < B / 2; ++bp) {
          const float2 a = __fmul2_rn(q2[r], nc2[bp]);
          const float2 e = make_float2(ex2(a.x), ex2(a.y));
          t1[bp] = __fadd2_rn(t1[bp], e);
          t2[bp] = __ffma2_rn(e, e, t2[bp]);
        }
      }
    }
  }
}

// Octave grids (the bandwidths come in octaves of 1/h^2: with P points per
// octave, c_(k-P) = 2 c_k for c = 1/h^2, so e_(k-P) = e_k^2 for every pair).
// A thread owns two residues r, r+1 (mod P) and their 8 octaves: per pair and
// residue three exponentials (octaves 7, 4 and 1) by MUFU ex2, the other
// octaves by squaring down (at most two squarings from an exponential, which
// also bounds the growth of the ex2 error to 4x), including one square below
// octave 0.  Since S2(k) = sum e_k^2 = S1(k-P), the nine running sums
// (octaves 0..7 and "octave -1") give S1 and S2 of all 16 bandwidths.  Per
// evaluation: 3/8 ex2 and 15/8 packed FP32 lane-operations (3/8 of them in
// FFMA2), which balances the FP32 pipe (about 124 lanes/clk/SM) against the
// MUFU pipe (32 ex2/clk/SM).
template <int D, int R, bool EDGE>
__device__ __forceinline__ void lscv_columns_oct(const float* __restrict__ sF, int j_lo, int j_hi,
                                                 const float (&y)[R][D], const float2 (&nca)[3],
                                                 float2 (&acc)[9], int64_t i0, int64_t jg0, int64_t n) {
  constexpr int DP = DPad<D>::value;
  if constexpr (D > 4) {
    // wide samples, one row per lane (sF holds -v): two columns per
    // iteration, each squared distance in packed FP32x2 over coordinate
    // pairs (two chains joined by one add), as in the direct kernel
    static_assert(R == 1 && DP % 4 == 0, "wide path: one row per lane");
    float2 y2[DP / 2];
#pragma unroll
    for (int k = 0; k < DP / 2; ++k) y2[k] = make_float2(y[0][2 * k], y[0][2 * k + 1]);
#pragma unroll 1
    for (int jj = j_lo; jj < j_hi; jj += 2) {
      float qv[2];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        qv[c] = wide_q<DP>(sF, jj + c, y2);
        if (EDGE) {
          const int64_t j = jg0 + jj + c;
          if (!(i0 < j && j < n)) qv[c] = kOctMask;  // every term exactly 0
        }
      }
#pragma unroll
      for (int c = 0; c < 2; ++c) octave_terms(qv[c], nca, acc);
    }
    return;
  }
  constexpr int CPI = DP <= 4 ? 4 / DP : 1;  // columns per iteration
  constexpr int NV = CPI * DP / 4;           // 16-byte shared-memory loads per iteration
#pragma unroll 1
  for (int jj = j_lo; jj < j_hi; jj += CPI) {
    float vv[4 * NV];
#pragma unroll
    for (int u = 0; u < NV; ++u) {
      const float4 v = *reinterpret_cast<const float4*>(sF + jj * DP + 4 * u);
      vv[4 * u] = v.x;
      vv[4 * u + 1] = v.y;
      vv[4 * u + 2] = v.z;
      vv[4 * u + 3] = v.w;
    }
#pragma unroll
    for (int c = 0; c < CPI; ++c) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        float qv = 0.f;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const float dl = y[r][k] - vv[c * DP + k];
          qv = fmaf(dl, dl, qv);
        }
        if (EDGE) {
          const int64_t i = i0 + 32 * r, j = jg0 + jj + c;
          if (!(i < j && j < n)) qv = kOctMask;  // every term exactly 0
        }
        octave_terms(qv, nca, acc);
      }
    }
  }
}

constexpr int kReduceRows = 64;  // item rows per CTA of the LSCV reduction

__device__ double lscv_chunk_total(const DsDev* ds, int c0, int64_t r0, int64_t r1, double* s);
__device__ void lscv_finish_body(DsDev* ds);

// Fused single-dataset launches: the CTA that finishes last (a counter in the
// descriptor; no CTA waits) adds the item rows and finishes, with the same
// code and order as k_lscv_reduce (whose last CTA also finishes), so results
// are bitwise those of the separate reduction.
__device__ __noinline__ void lscv_fused_finish(const Phase& ph) {
  __shared__ double sFin[kThreads];
  __shared__ int sLast;
  DsDev* ds = ph.ds;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) sLast = atomicAdd(&ds->pair_count, 1u) == gridDim.x - 1u;
  __syncthreads();
  if (!sLast) return;
  __threadfence();
  if (ds->res.status == KDE_OK && (ds->methods & KDE_METHOD_LSCV)) {
    const int W = 2 * ds->n_h_pad;
    const int64_t rows = ds->lscv_rows;
    for (int c0 = 0; c0 < W; c0 += 32) {
      double x = 0.0;  // chunk totals in chunk order, as k_lscv_reduce adds them
      for (int64_t r0 = 0; r0 < rows; r0 += kReduceRows)
        x += lscv_chunk_total(ds, c0, r0, min(rows, r0 + kReduceRows), sFin);
      if ((int)threadIdx.x < min(32, W - c0)) ds->lscv_sum[c0 + threadIdx.x] = x;
    }
    __syncthreads();
    lscv_finish_body(ds);
  }
  if (threadIdx.x == 0) ds->pair_count = 0u;
}

// Wide samples (d > 4) on a grid of one or two points, e.g. one g(H) of
// LSCV_H: one warp per item.  With a single chunk of bandwidths the block
// kernel splits each 32 x 32 tile among its 8 warps, four columns each, and a
// warp's share of a tile is small against the tile's fixed costs.  Here each
// warp walks the K tiles of its own item with all 32 columns, staging the
// column samples (negated) in its own slice of shared memory; only warp-level
// synchronisation.  Items are numbered as in the block kernel (one group), so
// the partial rows and their reduction are the same.
template <int D, bool KAHAN>
__global__ void __launch_bounds__(kThreads, 2) k_lscv_warp(Phase ph) {
  dependent_launch_wait();
  constexpr int T = 32, B = 2, DP = DPad<D>::value;
  static_assert(D > 4 && DP % 4 == 0, "wide samples only");
  __shared__ __align__(16) float sFw[kWarps][T * DP];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* sF = sFw[warp];
  const int64_t nw = (int64_t)gridDim.x * kWarps;
  for (int64_t it = (int64_t)blockIdx.x * kWarps + warp; it < ph.total; it += nw) {
    const int di = find_ds(ph.off, ph.n_ds, it);
    const DsDev* ds = ph.ds + di;
    if (ds->res.status != KDE_OK) continue;
    const int64_t row = it - ph.off[di] + (ph.base ? ph.base[di] : 0);
    const int64_t tb = ds->lscv_t0 + row * ds->lscv_K;
    const int64_t te = min(tb + (int64_t)ds->lscv_K, ds->lscv_tiles);
    const bool one = ds->n_h == 1;  // two columns per packed evaluation (see lscv_columns)
    const float2 nc2[1] = {make_float2(ds->nc[0], ds->nc[one ? 0 : 1])};
    float2 t1[1] = {make_float2(0.f, 0.f)}, t2[1] = {make_float2(0.f, 0.f)};
    float ks[4] = {0.f, 0.f, 0.f, 0.f}, kc[4] = {0.f, 0.f, 0.f, 0.f};  // Kahan (s, c): S1 b0, S1 b1, S2 b0, S2 b1
    const int64_t n = ds->n, n_pad = ds->n_pad;
    const float* __restrict__ Y = ds->y;
    int64_t l, q;
    tile_coords(tb, l, q);
    int64_t l_loaded = -1;
    float yn[1][D];
#pragma unroll
    for (int k = 0; k < D; ++k) yn[0][k] = Y[(int64_t)k * n_pad + q * T + lane];
    int run = 0;
    for (int64_t t = tb; t < te; ++t) {
      if (l != l_loaded) {
        __syncwarp();
        for (int idx = lane; idx < T * DP; idx += 32) {
          const int jj = idx / DP, k = idx - jj * DP;
          sF[idx] = (k < D) ? -Y[(int64_t)k * n_pad + l * T + jj] : 0.f;
        }
        __syncwarp();
        l_loaded = l;
      }
      float y[1][D];
      const int64_t qn = (q + 1 > l) ? 0 : q + 1;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        y[0][k] = yn[0][k];
        if (t + 1 < te) yn[0][k] = Y[(int64_t)k * n_pad + qn * T + lane];
      }
      const bool edge = (q == l) || ((l + 1) * T > n);
      const int64_t i0 = q * T + lane, jg0 = l * T;
      if (one) {
        if (edge)
          lscv_columns<D, B, 1, true, true>(sF, 0, T, y, nc2, t1, t2, i0, jg0, n);
        else
          lscv_columns<D, B, 1, false, true>(sF, 0, T, y, nc2, t1, t2, i0, jg0, n);
      } else {
        if (edge)
          lscv_columns<D, B, 1, true>(sF, 0, T, y, nc2, t1, t2, i0, jg0, n);
        else
          lscv_columns<D, B, 1, false>(sF, 0, T, y, nc2, t1, t2, i0, jg0, n);
      }
      if (KAHAN && ++run >= 8) {  // runs of 256 terms
        kahan_add(ks[0], kc[0], t1[0].x);
        kahan_add(ks[1], kc[1], t1[0].y);
        kahan_add(ks[2], kc[2], t2[0].x);
        kahan_add(ks[3], kc[3], t2[0].y);
        t1[0] = t2[0] = make_float2(0.f, 0.f);
        run = 0;
      }
      if (++q > l) {
        ++l;
        q = 0;
      }
    }
    float2 tot[4];
    const float tail[4] = {t1[0].x, t1[0].y, t2[0].x, t2[0].y};
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      if (KAHAN) {
        kahan_add(ks[m], kc[m], tail[m]);
        tot[m] = warp_sum_ff(ks[m], -kc[m]);
      } else {
        tot[m] = warp_sum_ff(tail[m], 0.f);
      }
    }
    if (lane == 0) {
      // row layout of the block kernel: (S1, S2) of bandwidth 0, then of
      // bandwidth 1 (one bandwidth: both halves are bandwidth 0)
      double* out = ds->lscv_part + row * (2 * (int64_t)ds->n_h_pad);
      if (one) {
        out[0] = ff_value(tot[0]) + ff_value(tot[1]);
        out[1] = ff_value(tot[2]) + ff_value(tot[3]);
        out[2] = 0.0;
        out[3] = 0.0;
      } else {
        out[0] = ff_value(tot[0]);
        out[1] = ff_value(tot[2]);
        out[2] = ff_value(tot[1]);
        out[3] = ff_value(tot[3]);
      }
    }
  }
}

// octave instances for d <= 4 are capped at 80 registers: 3 CTAs per SM
// (wide ones spill there and keep 2)
template <int D, int B, int R, bool KAHAN, bool OCT>
__global__ void __launch_bounds__(kThreads, (OCT && D <= 4) ? 3 : 2) k_lscv(Phase ph) {
  dependent_launch_wait();
  constexpr int T = 32 * R;
  constexpr int DP = DPad<D>::value;
  constexpr int FB = T * DP * (kPackedQ<D, R, OCT> ? 8 : 4);  // column tile bytes
  extern __shared__ __align__(16) unsigned char smem[];
  float* sF = reinterpret_cast<float*>(smem);                                 // [T][DP] (pairs if packed)
  double* sRed = reinterpret_cast<double*>(smem + FB);                        // [8][B][2]
  float4* sK = reinterpret_cast<float4*>(smem + FB + kWarps * B * 16);        // [8][B][32]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  for (int64_t it = blockIdx.x; it < ph.total; it += gridDim.x) {
    const int di = find_ds(ph.off, ph.n_ds, it);
    const DsDev* ds = ph.ds + di;
    if (ds->res.status != KDE_OK) continue;
    const int64_t li = it - ph.off[di] + (ph.base ? ph.base[di] : 0);
    const int G = ds->n_groups;
    const int hg = (int)(li % G);
    const int64_t row = li / G;
    const int64_t tb = ds->lscv_t0 + row * ds->lscv_K;
    const int64_t te = min(tb + (int64_t)ds->lscv_K, ds->lscv_tiles);
    const int cg = min(kWarps, ds->n_chunks - hg * kWarps);
    const WarpRole role = warp_role(warp, cg);
    const int S = role.S, my_chunk = role.chunk, my_slice = role.slice;
    const bool active = role.active;
    const int cols = T / S;
    const int j_lo = active ? my_slice * cols : 0;
    const int j_hi = active ? j_lo + cols : 0;
    const int hbase = (hg * kWarps + my_chunk) * B;

    // a grid of one bandwidth (B = 2, rows paired; see lscv_columns)
    constexpr bool kOne = (B == 2) && !OCT && (R % 2 == 0) && D <= 4;
    const bool one = kOne && ds->n_h == 1;
    float2 nc2[B / 2], t1[B / 2], t2[B / 2];
    // octave grids: residues rb, rb + 1 of P; ex2 at octaves 7, 4 and 1; 9 running sums
    const int P = OCT ? ds->oct_P : 0;
    const int rb = 2 * (hg * kWarps + my_chunk);
    float2 nca[3], oacc[9];
    if constexpr (OCT) {
      nca[0] = make_float2(ds->nc[rb + 7 * P], ds->nc[rb + 1 + 7 * P]);
      nca[1] = make_float2(ds->nc[rb + 4 * P], ds->nc[rb + 1 + 4 * P]);
      nca[2] = make_float2(ds->nc[rb + P], ds->nc[rb + 1 + P]);
#pragma unroll
      for (int j = 0; j < 9; ++j) oacc[j] = make_float2(0.f, 0.f);
    } else {
#pragma unroll
      for (int bp = 0; bp < B / 2; ++bp) {
        nc2[bp] = make_float2(ds->nc[hbase + 2 * bp], ds->nc[hbase + 2 * bp + (one ? 0 : 1)]);
        t1[bp] = make_float2(0.f, 0.f);
        t2[bp] = make_float2(0.f, 0.f);
      }
    }
    if (KAHAN) {
#pragma unroll
      for (int b = 0; b < B; ++b) sK[(warp * B + b) * 32 + lane] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const int64_t n = ds->n, n_pad = ds->n_pad;
    const float* __restrict__ Y = ds->y;
    // tiles per Kahan fold: FP32 runs of at least 256 terms per running sum,
    // 1,024 in the octave kernel (its fold of 9 packed sums per tile was
    // 0.35 % of a full-size launch: 30.60 -> 30.49 ms with every other tile)
    const int flush_every = OCT ? max(1, 1024 / (R * cols)) : max(1, 256 / (R * cols));
    int64_t l, q;
    tile_coords(tb, l, q);
    int64_t l_loaded = -1;
    int run = 0;
    // wide samples (d > 4, one row per lane, few columns per warp and tile):
    // the rows of the next tile are loaded while the current one is evaluated
    constexpr bool kPrefetch = D > 4;
    float yn[kPrefetch ? R : 1][kPrefetch ? D : 1];
    if constexpr (kPrefetch) {
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int k = 0; k < D; ++k) yn[r][k] = Y[(int64_t)k * n_pad + q * T + lane + 32 * r];
    }
    for (int64_t t = tb; t < te; ++t) {
      if (l != l_loaded) {
        __syncthreads();
        for (int idx = threadIdx.x; idx < T * DP; idx += kThreads) {
          const int jj = idx / DP, k = idx - jj * DP;
          const float v = (k < D) ? Y[(int64_t)k * n_pad + l * T + jj] : 0.f;
          if constexpr (kPackedQ<D, R, OCT>)
            reinterpret_cast<float2*>(sF)[idx] = make_float2(-v, -v);
          else if constexpr (D > 4)
            sF[idx] = -v;  // the wide paths add -v
          else
            sF[idx] = v;
        }
        __syncthreads();
        l_loaded = l;
      }
      float y[R][D];
      if constexpr (kPrefetch) {
        const int64_t qn = (q + 1 > l) ? 0 : q + 1;
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
          for (int k = 0; k < D; ++k) {
            y[r][k] = yn[r][k];
            if (t + 1 < te) yn[r][k] = Y[(int64_t)k * n_pad + qn * T + lane + 32 * r];
          }
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
          for (int k = 0; k < D; ++k) y[r][k] = Y[(int64_t)k * n_pad + q * T + lane + 32 * r];
      }
      const bool edge = (q == l) || ((l + 1) * T > n);
      const int64_t i0 = q * T + lane, jg0 = l * T;
      if constexpr (OCT) {
        if (edge)
          lscv_columns_oct<D, R, true>(sF, j_lo, j_hi, y, nca, oacc, i0, jg0, n);
        else
          lscv_columns_oct<D, R, false>(sF, j_lo, j_hi, y, nca, oacc, i0, jg0, n);
      } else if (one) {
        if (edge)
          lscv_columns<D, B, R, true, kOne>(sF, j_lo, j_hi, y, nc2, t1, t2, i0, jg0, n);
        else
          lscv_columns<D, B, R, false, kOne>(sF, j_lo, j_hi, y, nc2, t1, t2, i0, jg0, n);
      } else {
        if (edge)
          lscv_columns<D, B, R, true>(sF, j_lo, j_hi, y, nc2, t1, t2, i0, jg0, n);
        else
          lscv_columns<D, B, R, false>(sF, j_lo, j_hi, y, nc2, t1, t2, i0, jg0, n);
      }
      if (KAHAN && OCT && ++run >= flush_every) {
        // slot j: (s, c) of residue rb and of rb + 1 for running sum j
#pragma unroll
        for (int j = 0; j < 9; ++j) {
          float4 k0 = sK[(warp * B + j) * 32 + lane];
          kahan_add(k0.x, k0.y, oacc[j].x);
          kahan_add(k0.z, k0.w, oacc[j].y);
          sK[(warp * B + j) * 32 + lane] = k0;
          oacc[j] = make_float2(0.f, 0.f);
        }
        run = 0;
      }
      if (KAHAN && !OCT && ++run >= flush_every) {
#pragma unroll
        for (int bp = 0; bp < B / 2; ++bp) {
          float4 k0 = sK[(warp * B + 2 * bp) * 32 + lane];
          float4 k1 = sK[(warp * B + 2 * bp + 1) * 32 + lane];
          kahan_add(k0.x, k0.y, t1[bp].x);
          kahan_add(k0.z, k0.w, t2[bp].x);
          kahan_add(k1.x, k1.y, t1[bp].y);
          kahan_add(k1.z, k1.w, t2[bp].y);
          sK[(warp * B + 2 * bp) * 32 + lane] = k0;
          sK[(warp * B + 2 * bp + 1) * 32 + lane] = k1;
          t1[bp] = make_float2(0.f, 0.f);
          t2[bp] = make_float2(0.f, 0.f);
        }
        run = 0;
      }
      if (++q > l) {
        ++l;
        q = 0;
      }
    }
    // ---- item total: lanes (double-float butterfly in FP32), then column
    // slices in fixed order (FP64)
    __syncthreads();
    if constexpr (OCT) {
      // running sums j = 0..8 per residue; local bandwidth b = residue + 2 * octave
      // (butterflies: octave items are long, and the transposed form below
      // raised this kernel's register count and slowed its pair loop)
      float2 vs[9][2];
#pragma unroll
      for (int j = 0; j < 9; ++j) {
        float h0, l0, h1, l1;
        if (KAHAN) {
          float4 k = sK[(warp * B + j) * 32 + lane];
          kahan_add(k.x, k.y, oacc[j].x);  // unflushed tail of the run
          kahan_add(k.z, k.w, oacc[j].y);
          h0 = k.x, l0 = -k.y, h1 = k.z, l1 = -k.w;
        } else {
          h0 = oacc[j].x, l0 = 0.f, h1 = oacc[j].y, l1 = 0.f;
        }
        if (!active) h0 = l0 = h1 = l1 = 0.f;
        vs[j][0] = warp_sum_ff(h0, l0);
        vs[j][1] = warp_sum_ff(h1, l1);
      }
      if (lane == 0) {
#pragma unroll
        for (int oc = 0; oc < 8; ++oc)
#pragma unroll
          for (int rr = 0; rr < 2; ++rr) {
            const int b = rr + 2 * oc;
            sRed[(warp * B + b) * 2] = ff_value(vs[oc][rr]);                        // S1 at octave oc
            sRed[(warp * B + b) * 2 + 1] = ff_value(vs[oc == 0 ? 8 : oc - 1][rr]);  // S2 = S1 an octave below
          }
      }
    }
    if constexpr (!OCT && KAHAN) {
      // fold the unflushed runs into the lane's Kahan pairs (slot b: S1 in
      // x, y and S2 in z, w), then warp totals of the 2B values in lane
      // order: lane q = 2 b + (0: S1, 1: S2)
#pragma unroll
      for (int bp = 0; bp < B / 2; ++bp)
#pragma unroll
        for (int half = 0; half < 2; ++half) {
          const int b = 2 * bp + half;
          float4 k = sK[(warp * B + b) * 32 + lane];
          kahan_add(k.x, k.y, half ? t1[bp].y : t1[bp].x);
          kahan_add(k.z, k.w, half ? t2[bp].y : t2[bp].x);
          if (!active) k = make_float4(0.f, 0.f, 0.f, 0.f);
          sK[(warp * B + b) * 32 + lane] = k;
        }
      __syncwarp();
      const float2 v = warp_sums_ff_transposed(sK + warp * B * 32, 2 * B, lane);
      if (lane < 2 * B) sRed[(warp * B + (lane >> 1)) * 2 + (lane & 1)] = ff_value(v);
    }
#pragma unroll
    for (int bp = 0; bp < B / 2 && !OCT && !KAHAN; ++bp) {
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const int b = 2 * bp + half;
        float h1 = half ? t1[bp].y : t1[bp].x, h2 = half ? t2[bp].y : t2[bp].x;
        if (!active) h1 = h2 = 0.f;
        const float2 v1 = warp_sum_ff(h1, 0.f), v2 = warp_sum_ff(h2, 0.f);
        if (lane == 0) {
          sRed[(warp * B + b) * 2] = ff_value(v1);
          sRed[(warp * B + b) * 2 + 1] = ff_value(v2);
        }
      }
    }
    if (kOne && one) {
      // one bandwidth: the second half's (S1, S2) join the first's; the
      // padding slot is left empty
      __syncwarp();
      if (lane == 0) {
        double* r0 = sRed + warp * B * 2;
        r0[0] += r0[2];
        r0[1] += r0[3];
        r0[2] = 0.0;
        r0[3] = 0.0;
      }
    }
    __syncthreads();
    double* out = ds->lscv_part + row * (2 * (int64_t)ds->n_h_pad) + (OCT ? 0 : (int64_t)hg * kWarps * B * 2);
    for (int o = threadIdx.x; o < cg * B * 2; o += kThreads) {
      const int c = o / (2 * B), rem = o - c * 2 * B;
      double s = 0.0;
      for (int sl = 0; sl < S; ++sl) s += sRed[(sl * cg + c) * B * 2 + rem];
      if constexpr (OCT) {
        // local bandwidth b = residue + 2 * octave of chunk c -> grid index
        const int b = rem >> 1;
        const int k = 2 * (hg * kWarps + c) + (b & 1) + P * (b >> 1);
        out[2 * k + (rem & 1)] = s;
      } else {
        out[o] = s;
      }
    }
  }
  if (ph.fuse) lscv_fused_finish(ph);
}

// Total of item rows [r0, r1) for the columns [c0, c0 + wc) of one strip
// (wc = min(32, 2 n_h_pad - c0)), returned to threads t < wc for column
// c0 + t.  Thread t takes column t % wc and row part t / wc of P = 256 / wc
// parts: it adds rows r0 + part, r0 + part + P, ... in that order, and the
// P part sums of a column are added in order.  The loads of a part are
// issued before its adds (kReduceRows / P <= 8 rows of a full strip).
__device__ double lscv_chunk_total(const DsDev* ds, int c0, int64_t r0, int64_t r1, double* s) {
  const int W = 2 * ds->n_h_pad;
  const int wc = min(32, W - c0);
  const int P = kThreads / wc;
  const int t = threadIdx.x;
  double acc = 0.0;
  if (t < P * wc) {
    const double* p = ds->lscv_part + c0 + t % wc;
    constexpr int U = 8;
    int64_t r = r0 + t / wc;
    for (; r + (U - 1) * P < r1; r += U * P) {
      double v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) v[u] = __ldcg(p + (r + (int64_t)u * P) * W);
#pragma unroll
      for (int u = 0; u < U; ++u) acc += v[u];
    }
    for (; r < r1; r += P) acc += __ldcg(p + r * W);
  }
  s[t] = acc;
  __syncthreads();
  double tot = 0.0;
  if (t < wc)
    for (int part = 0; part < P; ++part) tot += s[part * wc + t];
  __syncthreads();  // s is reused by the next chunk
  return tot;
}

// Sum of the per-item partial rows in two fixed-order levels, then g(h).
// Grid: datasets x strips of 32 columns x chunks of kReduceRows item rows.
// A CTA forms its chunk's totals (lscv_chunk_total); with one chunk they are
// the sums.  With several, the CTA stores them in place of the chunk's first
// row (read by no one else), and the CTA that completes a strip last (a
// counter per strip; nobody waits) adds the chunk totals in chunk order.  The
// CTA that completes the dataset's last strip computes g(h) and the argmin.
// The order of every addition depends only on the dataset's geometry, so a
// selection gets the same bits alone, in a batch, served or fused into its
// pair kernel (which adds in the same order).
__global__ void __launch_bounds__(kThreads) k_lscv_reduce(DsDev* dsa, const int* ids) {
  dependent_launch_wait();
  DsDev* ds = dsa + (ids ? ids[blockIdx.x] : (int)blockIdx.x);
  __shared__ double s[kThreads];
  __shared__ int sLast;
  if (ds->res.status != KDE_OK || !(ds->methods & KDE_METHOD_LSCV)) return;
  const int W = 2 * ds->n_h_pad;
  const int strip = blockIdx.y, c0 = strip * 32;
  if (c0 >= W) return;
  const int64_t rows = ds->lscv_rows;
  const int chunks = (int)((rows + kReduceRows - 1) / kReduceRows);
  const int chunk = blockIdx.z;
  if (chunk >= chunks) return;
  const int t = threadIdx.x, wc = min(32, W - c0);
  const int64_t r0 = (int64_t)chunk * kReduceRows;
  const double tot = lscv_chunk_total(ds, c0, r0, min(rows, r0 + kReduceRows), s);
  if (chunks == 1) {
    if (t < wc) ds->lscv_sum[c0 + t] = tot;
  } else {
    if (t < wc) ds->lscv_part[r0 * W + c0 + t] = tot;
    __threadfence();
    __syncthreads();
    if (t == 0) sLast = atomicAdd(&ds->strip_count[strip], 1u) == (unsigned)chunks - 1u;
    __syncthreads();
    if (!sLast) return;
    __threadfence();
    // the chunk totals are loaded together (one L2 round trip per 256), then
    // added in chunk order
    double x = 0.0;
    for (int k0 = 0; k0 < chunks; k0 += kThreads / wc) {
      const int nk = min(kThreads / wc, chunks - k0);
      if (t < nk * wc)
        s[t] = __ldcg(ds->lscv_part + (int64_t)(k0 + t / wc) * kReduceRows * W + c0 + t % wc);
      __syncthreads();
      if (t < wc)
        for (int k = 0; k < nk; ++k) x += s[k * wc + t];
      __syncthreads();
    }
    if (t < wc) ds->lscv_sum[c0 + t] = x;
    if (t == 0) ds->strip_count[strip] = 0u;
  }
  __threadfence();
  __syncthreads();
  const unsigned strips = (unsigned)((W + 31) / 32);
  if (t == 0) sLast = atomicAdd(&ds->reduce_count, 1u) == strips - 1u;
  __syncthreads();
  if (!sLast) return;
  __threadfence();
  lscv_finish_body(ds);
  if (t == 0) ds->reduce_count = 0u;
}

// Order of (value, index) candidates for a first-index argmin: a number
// before NaN, a smaller number first, equal values (or two NaNs) by index;
// index -1 marks no candidate.
__device__ __forceinline__ bool argmin_before(double g, int k, double h, int j) {
  if (k < 0) return false;
  if (j < 0) return true;
  const bool gn = g != g, hn = h != h;
  if (gn != hn) return hn;
  if (!gn && g != h) return g < h;
  return k < j;
}

// g(h) on the grid and its first-index argmin (Eqs. LSCV-gh, LSCV-finalH),
// by the threads of one CTA.
__device__ void lscv_finish_body(DsDev* ds) {
  const int d = ds->d, n_h = ds->n_h;
  const double n = (double)ds->n;
  // 2^(1 + d/2) exactly: a power of two, times sqrt(2) for odd d (no FP64
  // exp2, a long sequence on this part); one FP64 division for 1/n
  const double c2 = __longlong_as_double((long long)(1024 + d / 2) << 52) * ((d & 1) ? 1.4142135623730951 : 1.0);
  const double inv_n = 1.0 / n, w2 = 2.0 * inv_n * inv_n;
  // K-term weight: the paper's n^-2 (Eq. LSCV-gh) or exact leave-one-out 1/(n(n-1))
  const double wk = ds->cv_loo ? 2.0 * inv_n / (n - 1.0) : w2;
  // g(h_k) per thread (h^-d by d multiplications and one division), and the
  // first index of the minimum: per thread over its k, then lexicographic
  // (g, k) minima across lanes and warps (NaN ranks above every number)
  __shared__ double sg[kWarps];
  __shared__ int sk[kWarps];
  double gb = 0.0;
  int best = -1;
  for (int k = threadIdx.x; k < n_h; k += blockDim.x) {
    const double s1 = __ldcg(ds->lscv_sum + 2 * k), s2 = __ldcg(ds->lscv_sum + 2 * k + 1);
    const double hk = ds->h[k];
    double hd = 1.0;
    for (int i = 0; i < d; ++i) hd *= hk;
    const double gk = ds->A / hd * (w2 * s1 - wk * c2 * s2 + inv_n);
    ds->g[k] = gk;
    if (argmin_before(gk, k, gb, best)) {
      gb = gk;
      best = k;
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const double og = __shfl_xor_sync(0xffffffffu, gb, o);
    const int ok = __shfl_xor_sync(0xffffffffu, best, o);
    if (argmin_before(og, ok, gb, best)) {
      gb = og;
      best = ok;
    }
  }
  if (lane == 0) {
    sg[warp] = gb;
    sk[warp] = best;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    gb = sg[0];
    best = sk[0];
    for (int w = 1; w < kWarps; ++w) {
      const double og = sg[w];
      const int ok = sk[w];
      if (argmin_before(og, ok, gb, best)) {
        gb = og;
        best = ok;
      }
    }
    kde_result& r = ds->res;
    r.method |= KDE_METHOD_LSCV;
    r.argmin = best;
    r.n_h = n_h;
    r.g_min = gb;
    r.h = ds->h[best];
    r.h_data = (d == 1) ? ds->h[best] * ds->sigma : 0.0;
    r.flags = (best == 0 ? KDE_FLAG_MIN_AT_LOWER_EDGE : 0) |
              (best == n_h - 1 ? KDE_FLAG_MIN_AT_UPPER_EDGE : 0);
  }
}


template <int D, int B, int R, bool KAHAN, bool OCT>
cudaError_t launch_t(const Phase& ph, int grid, cudaStream_t st) {
  if constexpr (lscv_warp_items(D, B)) {  // static shared memory: no attribute to set
    if (grid <= 0) return cudaSuccess;
    return launch_kernel(k_lscv_warp<D, KAHAN>, dim3(grid), dim3(kThreads), 0, st, ph);
  } else {
    const size_t smem = lscv_smem_bytes(D, B, R, KAHAN, OCT);
    // set once per instance (a function-local static is initialised once,
    // thread-safely: the server's worker and callers may launch concurrently)
    static const cudaError_t attr = cudaFuncSetAttribute(
        k_lscv<D, B, R, KAHAN, OCT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (attr != cudaSuccess) return attr;
    if (grid <= 0) return cudaSuccess;  // attribute set only (before a graph capture)
    return launch_kernel(k_lscv<D, B, R, KAHAN, OCT>, dim3(grid), dim3(kThreads), smem, st, ph);
  }
}

template <int D, int B, int R>
cudaError_t launch_k(const Phase& ph, bool kahan, bool oct, int grid, cudaStream_t st) {
  if constexpr (B == 16) {
    if (oct) return kahan ? launch_t<D, B, R, true, true>(ph, grid, st) : launch_t<D, B, R, false, true>(ph, grid, st);
  } else {
    if (oct) return cudaErrorInvalidValue;  // octave grids take 16 bandwidths per thread
  }
  return kahan ? launch_t<D, B, R, true, false>(ph, grid, st) : launch_t<D, B, R, false, false>(ph, grid, st);
}

template <int D, int B>
cudaError_t launch_r(const Phase& ph, int R, bool kahan, bool oct, int grid, cudaStream_t st) {
  switch (R) {
    case 1: return launch_k<D, B, 1>(ph, kahan, oct, grid, st);
    case 4:
      if constexpr (D <= 4) return launch_k<D, B, 4>(ph, kahan, oct, grid, st);
      return cudaErrorInvalidValue;  // d > 4 walks one row per lane
    default: return cudaErrorInvalidValue;
  }
}

template <int D>
cudaError_t launch_b(const Phase& ph, int B, int R, bool kahan, bool oct, int grid, cudaStream_t st) {
  switch (B) {
    case 2: return launch_r<D, 2>(ph, R, kahan, oct, grid, st);
    case 8: return launch_r<D, 8>(ph, R, kahan, oct, grid, st);
    case 16: return launch_r<D, 16>(ph, R, kahan, oct, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

size_t lscv_smem_bytes(int d, int B, int R, bool kahan, bool oct) {
  const int dp = (d == 3) ? 4 : d;
  const bool packed = (R == 4 && d == 4 && !oct);  // kPackedQ: the column tile holds pairs
  return (size_t)32 * R * dp * (packed ? 8 : 4) + (size_t)kWarps * B * 16 +
         (kahan ? (size_t)kWarps * B * 32 * 16 : 0);
}

cudaError_t prepare_lscv(int d, int B, int R, bool kahan, bool oct) {
  Phase ph{nullptr, nullptr, nullptr, 0, 0, 0};
  return launch_lscv(ph, d, B, R, kahan, oct, 0, nullptr);
}

cudaError_t launch_lscv(const Phase& ph, int d, int B, int R, bool kahan, bool oct, int grid,
                        cudaStream_t st) {
  if (ph.total <= 0 && grid > 0) return cudaSuccess;
  switch (d) {
    case 1: return launch_b<1>(ph, B, R, kahan, oct, grid, st);
    case 2: return launch_b<2>(ph, B, R, kahan, oct, grid, st);
    case 3: return launch_b<3>(ph, B, R, kahan, oct, grid, st);
    case 4: return launch_b<4>(ph, B, R, kahan, oct, grid, st);
    case 8: return launch_b<8>(ph, B, R, kahan, oct, grid, st);
    case 12: return launch_b<12>(ph, B, R, kahan, oct, grid, st);
    case 16: return launch_b<16>(ph, B, R, kahan, oct, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_lscv_reduce(DsDev* ds, int n_ds, const int* ids, int n_h_pad_max, int64_t rows_max,
                               cudaStream_t st) {
  if (n_ds <= 0) return cudaSuccess;
  int64_t chunks = (rows_max + kReduceRows - 1) / kReduceRows;
  if (chunks < 1) chunks = 1;
  if (chunks > 65535) return cudaErrorInvalidValue;
  dim3 grid(n_ds, (2 * n_h_pad_max + 31) / 32, (unsigned)chunks);
  return launch_kernel(k_lscv_reduce, grid, dim3(kThreads), 0, st, ds, ids);
}

}  // namespace gbkde
