// nyx_roi.cuh -- per-ROI feature kernel (implementation, included by the
// per-dtype translation units nyx_roi_<dtype>.cu).
//
// One thread block processes one ROI at a time, pulling ROI ids from a work
// queue (persistent launch, one queue per size class).  The ROI's bounding
// box is read from global memory (the image and mask are L2-resident after
// the label scan for images up to ~100 MB) and staged in shared memory:
//   raster  : bbox-local GLCM bin per cell (0xFFFF = not in this ROI), with a
//             border of `pad` sentinel cells so neighbour lookups need no
//             bounds checks
//   pc / pv : the ROI's pixels (packed local coordinates, encoded values) in
//             raster order
// Every feature group then runs on shared memory:
//   first-order statistics (Table S1/S5): exact pass-1 sums, then centred
//       power sums (FP32 partials merged with two-sum compensation, or FP64)
//   moments (Table S2 rows 123-135, Table S5 rows 368/370): centred sums
//       about the exact centroid, raw/normalised moments and Hu invariants
//       derived per ROI in FP64
//   histogram features: shared-memory histogram with hist_bins bins
//   GLCM (Table S3 rows 140-174, Table S5 row 361): per offset, a shared
//       hash table of (min bin, max bin) -> count with warp-aggregated
//       inserts; features from the marginals p_x, p_{x+y}, p_{x-y} plus one
//       pass over the non-zero cells (ASM, entropy, max, mutual information)
//   order statistics: block radix sort of the values
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <type_traits>

#include "nyx_internal.cuh"

namespace nyx {

template <int NT_, int PIX_, int CELLS_>
struct RoiClass {
  static constexpr int NT = NT_;
  static constexpr int NW = NT_ / 32;
  static constexpr int PIX = PIX_;      // max pixels of an ROI
  static constexpr int CELLS = CELLS_;  // max padded raster cells
  static constexpr int TAB = 2 * PIX_;  // GLCM hash capacity (power of two); also 2 sort buffers
};
using ClassS = RoiClass<128, 1024, 4096>;
using ClassM = RoiClass<256, 8192, 16384>;

constexpr int RED_MAX = 64;  // max values per block reduction

// shared-memory layout (byte offsets), identical on host and device
struct SmemLayout {
  int raster, pc, pv, tab, rank, hist, marg, red, res, total;
  __host__ __device__ static int align16(int x) { return (x + 15) & ~15; }
  template <class C>
  __host__ __device__ static SmemLayout make(int ng, int hist_bins) {
    SmemLayout L;
    int o = 0;
    L.raster = o; o = align16(o + 2 * C::CELLS);
    L.pc = o;     o = align16(o + 4 * C::PIX);
    L.pv = o;     o = align16(o + 4 * C::PIX);
    L.tab = o;    o = align16(o + 4 * C::TAB);
    L.rank = o;   o = align16(o + 2 * C::PIX);
    L.hist = o;   o = align16(o + 4 * (hist_bins > 0 ? hist_bins : 1));
    int marg = 4 * (4 * (ng > 0 ? ng : 1));
    int cnts = 4 * (C::NW * 256 + 256);
    L.marg = o;   o = align16(o + (marg > cnts ? marg : cnts));
    L.red = o;    o = align16(o + 8 * C::NW * RED_MAX);
    L.res = o;    o = align16(o + 8 * (RED_MAX + 2 * NGLCM + 16));
    L.total = o;
    return L;
  }
};

// ----------------------------------------------------------------------------
// block reductions

template <class C, class A, int NV>
__device__ inline void block_sum(A (&v)[NV], double* scratch, double* out) {
  static_assert(NV <= RED_MAX, "reduction too wide");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    if constexpr (std::is_same<A, float>::value) {
      float hi = v[i], lo = 0.f;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(0xFFFFFFFFu, hi, o);
        const float l2 = __shfl_xor_sync(0xFFFFFFFFu, lo, o);
        float s, e;
        two_sum(hi, h2, s, e);
        hi = s;
        lo = __fadd_rn(__fadd_rn(lo, l2), e);
      }
      if (lane == 0) scratch[warp * NV + i] = (double)hi + (double)lo;
    } else {
      double x = v[i];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
      if (lane == 0) scratch[warp * NV + i] = x;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NV; i += C::NT) {
    double s = 0;
    for (int w = 0; w < C::NW; ++w) s += scratch[w * NV + i];
    out[i] = s;
  }
  __syncthreads();
}

template <class C, int NV>
__device__ inline void block_sum_i64(long long (&v)[NV], double* scratch_d, long long* out) {
  long long* scratch = (long long*)scratch_d;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    long long x = v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
    if (lane == 0) scratch[warp * NV + i] = x;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NV; i += C::NT) {
    long long s = 0;
    for (int w = 0; w < C::NW; ++w) s += scratch[w * NV + i];
    out[i] = s;
  }
  __syncthreads();
}

template <class C>
__device__ inline float block_max(float v, double* scratch_d) {
  float* scratch = (float*)scratch_d;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  float m = scratch[0];
  for (int w = 1; w < C::NW; ++w) m = fmaxf(m, scratch[w]);
  __syncthreads();
  return m;
}

template <class C>
__device__ inline unsigned long long block_max_u64(unsigned long long v, double* scratch_d) {
  unsigned long long* scratch = (unsigned long long*)scratch_d;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long u = __shfl_xor_sync(0xFFFFFFFFu, v, o);
    v = u > v ? u : v;
  }
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  unsigned long long m = scratch[0];
  for (int w = 1; w < C::NW; ++w) m = scratch[w] > m ? scratch[w] : m;
  __syncthreads();
  return m;
}

// exclusive scan of `n` unsigned values in shared memory (single warp)
__device__ inline void warp_exclusive_scan(unsigned* a, int n) {
  const int lane = threadIdx.x & 31;
  unsigned carry = 0;
  for (int base = 0; base < n; base += 32) {
    const int i = base + lane;
    const unsigned v = i < n ? a[i] : 0u;
    unsigned x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    if (i < n) a[i] = carry + x - v;
    carry += __shfl_sync(0xFFFFFFFFu, x, 31);
  }
}

// ----------------------------------------------------------------------------
// helpers

__device__ inline void put(const KParams& p, double* row, int q, double v) {
  const int c = __ldg(p.col_map + q);
  if (c >= 0) row[c] = v;
}

__device__ inline double ipow_d(double x, int k) {
  double r = 1.0;
  for (int i = 0; i < k; ++i) r *= x;
  return r;
}

__device__ inline float alog2(float x) { return log2f(x); }
__device__ inline double alog2(double x) { return log2(x); }

__device__ inline int binom(int n, int k) {
  int r = 1;
  for (int i = 0; i < k; ++i) r = r * (n - i) / (i + 1);
  return r;
}

// moment index <-> exponents (p, q, r), lexicographic with p+q+r <= 3
// (2D: r = 0, 10 entries; 3D: 20 entries)
template <int NDIM>
__host__ __device__ constexpr int midx(int p, int q, int r) {
  if (NDIM == 2) return (p == 0 ? 0 : p == 1 ? 4 : p == 2 ? 7 : 9) + q;
  int base = p == 0 ? 0 : p == 1 ? 10 : p == 2 ? 16 : 19;
  for (int qq = 0; qq < q; ++qq) base += 4 - p - qq;
  return base + r;
}
template <int NDIM>
__device__ inline void mexp(int k, int& p, int& q, int& r) {
  for (int a = 0; a <= 3; ++a)
    for (int b = 0; a + b <= 3; ++b)
      for (int c = 0; c <= (NDIM == 3 ? 3 - a - b : 0); ++c)
        if (midx<NDIM>(a, b, c) == k) {
          p = a;
          q = b;
          r = c;
          return;
        }
  p = q = r = 0;
}

// Hu's seven invariants (Hu 1962) from normalised central moments.
__device__ inline void hu7(double n20, double n02, double n11, double n30, double n21, double n12, double n03,
                           double* h) {
  const double a = n30 - 3 * n12, b = 3 * n21 - n03, s = n30 + n12, t = n21 + n03;
  h[0] = n20 + n02;
  h[1] = (n20 - n02) * (n20 - n02) + 4 * n11 * n11;
  h[2] = a * a + b * b;
  h[3] = s * s + t * t;
  h[4] = a * s * (s * s - 3 * t * t) + b * t * (3 * s * s - t * t);
  h[5] = (n20 - n02) * (s * s - t * t) + 4 * n11 * s * t;
  h[6] = b * s * (s * s - 3 * t * t) - a * t * (3 * s * s - t * t);
}

// normalisation exponent mu00^(1 + o/2) (2D) or mu000^(1 + o/3) (3D)
template <int NDIM>
__device__ inline double norm_pow(double m00, int o) {
  if (NDIM == 2) {
    switch (o) {
      case 0: return m00;
      case 1: return m00 * sqrt(m00);
      case 2: return m00 * m00;
      default: return m00 * m00 * sqrt(m00);
    }
  }
  const double c = cbrt(m00);
  switch (o) {
    case 0: return m00;
    case 1: return m00 * c;
    case 2: return m00 * c * c;
    default: return m00 * m00;
  }
}

// Finalise one weighting's moments from centred sums C[] about (c0,c1,c2)
// (ROI-local), where the exact centroid is (k0,k1,k2): shift, then raw,
// normalised and Hu.  valid = false -> every derived value NaN.
template <int NDIM>
__device__ __noinline__ void finalize_moments(const KParams& p, double* row, int wbase, const double* Cs, double c0, double c1,
                                 double c2, double k0, double k1, double k2, bool valid, double* save_mu) {
  constexpr int NM = NDIM == 3 ? 20 : 10;
  double mu[NM], M[NM];
  const double d0 = c0 - k0, d1 = c1 - k1, d2 = c2 - k2;  // shift from sum centre to exact centroid
  for (int k = 0; k < NM; ++k) {
    int a, b, c;
    mexp<NDIM>(k, a, b, c);
    double s = 0;
    for (int i = 0; i <= a; ++i)
      for (int j = 0; j <= b; ++j)
        for (int l = 0; l <= c; ++l)
          s += binom(a, i) * binom(b, j) * binom(c, l) * ipow_d(d0, a - i) * ipow_d(d1, b - j) * ipow_d(d2, c - l) *
               Cs[midx<NDIM>(i, j, l)];
    mu[k] = s;
  }
  // first-order central moments vanish at the exact centroid
  if (valid) {
    mu[midx<NDIM>(1, 0, 0)] = 0;
    mu[midx<NDIM>(0, 1, 0)] = 0;
    if (NDIM == 3) mu[midx<NDIM>(0, 0, 1)] = 0;
  }
  for (int k = 0; k < NM; ++k) {
    int a, b, c;
    mexp<NDIM>(k, a, b, c);
    double s = 0;
    for (int i = 0; i <= a; ++i)
      for (int j = 0; j <= b; ++j)
        for (int l = 0; l <= c; ++l)
          s += binom(a, i) * binom(b, j) * binom(c, l) * ipow_d(k0, a - i) * ipow_d(k1, b - j) * ipow_d(k2, c - l) *
               mu[midx<NDIM>(i, j, l)];
    M[k] = s;
  }
  const double nan = __longlong_as_double(0x7FF8000000000000ll);
  const double m00 = M[0];
  for (int k = 0; k < NM; ++k) {
    int a, b, c;
    mexp<NDIM>(k, a, b, c);
    const int o = a + b + c;
    put(p, row, Q_MOM + (wbase + F_M) * 20 + k, M[k]);
    put(p, row, Q_MOM + (wbase + F_MU) * 20 + k, valid ? mu[k] : nan);
    if (o >= 2) put(p, row, Q_MOM + (wbase + F_ETA) * 20 + k, valid ? mu[k] / norm_pow<NDIM>(mu[0], o) : nan);
    if (NDIM == 2) put(p, row, Q_MOM + (wbase + F_NU) * 20 + k, valid ? M[k] / norm_pow<NDIM>(m00, o) : nan);
  }
  if (NDIM == 2) {
    double h[7];
    const double g20 = norm_pow<2>(mu[0], 2), g30 = norm_pow<2>(mu[0], 3);
    hu7(mu[midx<2>(2, 0, 0)] / g20, mu[midx<2>(0, 2, 0)] / g20, mu[midx<2>(1, 1, 0)] / g20, mu[midx<2>(3, 0, 0)] / g30,
        mu[midx<2>(2, 1, 0)] / g30, mu[midx<2>(1, 2, 0)] / g30, mu[midx<2>(0, 3, 0)] / g30, h);
    for (int i = 0; i < 7; ++i) put(p, row, Q_MOM + (wbase + F_HU) * 20 + i, valid ? h[i] : nan);
  }
  if (save_mu)
    for (int k = 0; k < NM; ++k) save_mu[k] = mu[k];
}


// Statistics of Table S1 / S5 from the centred power sums S_k = sum (I - c)^k
// about a centring point c close to the mean (exact for integer images); the
// residual offset S_1 / n is removed by a binomial shift.
template <class T, int NDIM>
__device__ __noinline__ void finalize_stats(const KParams& p, double* row, const double* res_st, int n, double mean,
                                            double sumI, double energy, unsigned vmin, unsigned vmax, int64_t bimg,
                                            int x0, int y0, int z0, double cx, double cy, double cz, double bx,
                                            double by, double bz, bool wvalid, double* save) {
  const double nan = __longlong_as_double(0x7FF8000000000000ll);
  const double S1 = res_st[0];
  const double dl = S1 / n;
  double Sk[7];
  Sk[0] = n;
  for (int k = 1; k <= 6; ++k) Sk[k] = res_st[k - 1];
  double m[7];
  m[0] = 1;
  for (int k = 1; k <= 6; ++k) {
    double s = 0;
    for (int j = 0; j <= k; ++j) s += binom(k, j) * ipow_d(-dl, k - j) * Sk[j];
    m[k] = s / n;
  }
  const double m2 = m[2] > 0 ? m[2] : 0.0;
  const double var = n > 1 ? m2 * n / (n - 1) : 0.0;
  const double sd = sqrt(var);
  const double mn = Enc<T>::dec(vmin), mx = Enc<T>::dec(vmax);
  const double imn = Enc<T>::dec(p.img_vmin[bimg]), imx = Enc<T>::dec(p.img_vmax[bimg]);
  put(p, row, Q_STATS + S_MEAN, mean);
  put(p, row, Q_STATS + S_MIN, mn);
  put(p, row, Q_STATS + S_MAX, mx);
  put(p, row, Q_STATS + S_RANGE, mx - mn);
  put(p, row, Q_STATS + S_VAR, var);
  put(p, row, Q_STATS + S_VAR_B, m2);
  put(p, row, Q_STATS + S_STD, sd);
  put(p, row, Q_STATS + S_STD_B, sqrt(m2));
  const bool pos = m2 > 0;
  const double kurt = pos ? m[4] / (m2 * m2) : 0.0;
  put(p, row, Q_STATS + S_SKEW, pos ? m[3] / (m2 * sqrt(m2)) : 0.0);
  put(p, row, Q_STATS + S_KURT, kurt);
  put(p, row, Q_STATS + S_EXKURT, pos ? kurt - 3.0 : 0.0);
  put(p, row, Q_STATS + S_HSKEW, pos ? m[5] / (m2 * m2 * sqrt(m2)) : 0.0);
  put(p, row, Q_STATS + S_HFLAT, pos ? m[6] / (m2 * m2 * m2) : 0.0);
  put(p, row, Q_STATS + S_ENERGY, energy);
  put(p, row, Q_STATS + S_RMS, sqrt(energy / n));
  put(p, row, Q_STATS + S_SE, sd / sqrt((double)n));
  put(p, row, Q_STATS + S_MAD, res_st[6] / n);
  put(p, row, Q_STATS + S_II, sumI);
  const double wcx = wvalid ? x0 + cx : nan, wcy = wvalid ? y0 + cy : nan, wcz = wvalid ? z0 + cz : nan;
  const double gx = x0 + bx, gy = y0 + by, gz = z0 + bz;
  put(p, row, Q_CEN_X, gx);
  put(p, row, Q_CEN_Y, gy);
  put(p, row, Q_CEN_Z, gz);
  put(p, row, Q_STATS + S_WCX, wcx);
  put(p, row, Q_STATS + S_WCY, wcy);
  put(p, row, Q_STATS + S_WCZ, wcz);
  double md = (wcx - gx) * (wcx - gx) + (wcy - gy) * (wcy - gy);
  if (NDIM == 3) md += (wcz - gz) * (wcz - gz);
  put(p, row, Q_STATS + S_MD, sqrt(md));
  put(p, row, Q_STATS + S_COV, mean != 0 ? sd / mean : nan);
  put(p, row, Q_STATS + S_COVERED, imx != imn ? (mx - mn) / (imx - imn) : nan);
  put(p, row, Q_STATS + S_PIU, (mx + mn) != 0 ? 100.0 * (1.0 - (mx - mn) / (mx + mn)) : nan);
  if (save) {
    save[SV_N] = n;
    save[SV_MEAN] = mean;
    for (int k = 2; k <= 6; ++k) save[SV_M2 + k - 2] = m[k];
    save[SV_SGN] = res_st[7];
    save[SV_ENERGY] = energy;
    save[SV_SUMI] = sumI;
    save[SV_CX] = cx;
    save[SV_CY] = cy;
    save[SV_CZ] = cz;
    save[SV_BX] = gx;
    save[SV_BY] = gy;
    save[SV_BZ] = gz;
    save[SV_X0] = x0;
    save[SV_Y0] = y0;
    save[SV_Z0] = z0;
  }
}

// GLCM features of one offset (Table S3 rows 140-174) from the reduced sums
// of the marginals and cells; accumulates the direction mean in gsum.
static __device__ __noinline__ void finalize_glcm(const KParams& p, double* row, const double* r, double mu, double sumave,
                                           double difave, float jmax, int di, int dir, double* gsum) {
  double f[NGLCM];
  const double hx = r[0], var = r[1], sument = r[2], sumvar = r[3], clushade = r[4], cluprom = r[5],
               contrast = r[6], id = r[7], idm = r[8], idn = r[9], idmn = r[10], iv = r[11], difvar = r[12],
               difent = r[13], asmv = r[14], je = r[15], mi = r[16];
  // covariance from the sum and difference marginals:
  // (i+j-2mu)^2 - (i-j)^2 = 4 (i-mu)(j-mu)
  const double cov = (sumvar - contrast) / 4.0;
  f[G_ASM] = asmv;
  f[G_ACOR] = cov + mu * mu;
  f[G_CLUPROM] = cluprom;
  f[G_CLUSHADE] = clushade;
  f[G_CLUTEND] = sumvar;
  f[G_CONTRAST] = contrast;
  f[G_CORR] = var > 0 ? cov / var : 1.0;
  f[G_DIFAVE] = difave;
  f[G_DIFENTRO] = difent;
  f[G_DIFVAR] = difvar;
  f[G_DIS] = difave;
  f[G_ENERGY] = sqrt(asmv);
  f[G_ENTROPY] = je;
  f[G_HOM1] = id;
  f[G_HOM2] = idm;
  f[G_IDM] = idm;
  // HXY1 = HXY2 = HX + HY and HX = HY for a symmetric matrix, so
  // HXY - HXY1 = -MI and HXY2 - HXY = MI (mutual information)
  f[G_INFOMEAS1] = hx > 0 ? -mi / hx : 0.0;
  const double arg = 1.0 - exp(-2.0 * mi);
  f[G_INFOMEAS2] = sqrt(arg > 0 ? arg : 0.0);
  f[G_IDMN] = idmn;
  f[G_ID] = id;
  f[G_IDN] = idn;
  f[G_IV] = iv;
  f[G_JAVE] = mu;
  f[G_JE] = je;
  f[G_JMAX] = jmax;
  f[G_SUMAVE] = sumave;
  f[G_SUMENT] = sument;
  f[G_JVAR] = var;
  f[G_SUMVAR] = sumvar;
  f[G_VARIANCE] = var;
  for (int g = 0; g < NGLCM; ++g) {
    if (p.per_offset) put(p, row, Q_GLCM_O + (di * MAX_DIRS + dir) * NGLCM + g, f[g]);
    gsum[g] += f[g];
  }
  gsum[NGLCM] += 1.0;
}

// Percentiles by linear interpolation at h = (n-1) q on sorted values, and
// the index range of values inside [P10, P90].
template <class T>
__device__ __noinline__ void finalize_percentiles(const KParams& p, double* row, const unsigned* v, int n, double* sc,
                                                  int* idx) {
  const double nan = __longlong_as_double(0x7FF8000000000000ll);
  const double qs[7] = {0.01, 0.10, 0.25, 0.50, 0.75, 0.90, 0.99};
  double pv_[7];
  for (int k = 0; k < 7; ++k) {
    const double h = __dmul_rn((double)(n - 1), qs[k]);
    const int lo = (int)floor(h);
    if (lo >= n - 1) {
      pv_[k] = Enc<T>::dec(v[n - 1]);
    } else {
      const double a = Enc<T>::dec(v[lo]), b = Enc<T>::dec(v[lo + 1]);
      pv_[k] = __dadd_rn(a, __dmul_rn(__dsub_rn(h, (double)lo), __dsub_rn(b, a)));
    }
  }
  sc[0] = pv_[3];
  sc[1] = pv_[1];
  sc[2] = pv_[5];
  put(p, row, Q_STATS + S_P01, pv_[0]);
  put(p, row, Q_STATS + S_P10, pv_[1]);
  put(p, row, Q_STATS + S_P25, pv_[2]);
  put(p, row, Q_STATS + S_MEDIAN, pv_[3]);
  put(p, row, Q_STATS + S_P75, pv_[4]);
  put(p, row, Q_STATS + S_P90, pv_[5]);
  put(p, row, Q_STATS + S_P99, pv_[6]);
  put(p, row, Q_STATS + S_IQR, pv_[4] - pv_[2]);
  put(p, row, Q_STATS + S_QCOD, (pv_[4] + pv_[2]) != 0 ? (pv_[4] - pv_[2]) / (pv_[4] + pv_[2]) : nan);
  int lo = 0, hi = n;
  while (lo < hi) {
    const int m = (lo + hi) >> 1;
    if (Enc<T>::dec(v[m]) < pv_[1]) lo = m + 1;
    else hi = m;
  }
  idx[0] = lo;  // first value >= P10
  lo = 0;
  hi = n;
  while (lo < hi) {
    const int m = (lo + hi) >> 1;
    if (Enc<T>::dec(v[m]) <= pv_[5]) lo = m + 1;
    else hi = m;
  }
  idx[1] = lo;  // one past the last value <= P90
}

// ----------------------------------------------------------------------------
// the kernel

template <class T, int NDIM, class C, class A>
__global__ void __launch_bounds__(C::NT) k_roi(KParams p, int cls) {
  extern __shared__ __align__(16) unsigned char smem[];
  const SmemLayout L = SmemLayout::make<C>(p.ng, p.hist_bins);
  uint16_t* raster = (uint16_t*)(smem + L.raster);
  unsigned* pc = (unsigned*)(smem + L.pc);
  unsigned* pv = (unsigned*)(smem + L.pv);
  unsigned* tab = (unsigned*)(smem + L.tab);
  uint16_t* rank = (uint16_t*)(smem + L.rank);
  unsigned* hist = (unsigned*)(smem + L.hist);
  unsigned* marg = (unsigned*)(smem + L.marg);
  double* red = (double*)(smem + L.red);
  double* res = (double*)(smem + L.res);
  __shared__ RoiInfo s_r;
  __shared__ int s_item;
  __shared__ unsigned s_rowcnt[C::NW], s_rowbase[C::NW + 1];
  __shared__ FastDiv s_fd;
  __shared__ double s_sc[16];
  __shared__ long long s_i64[16];
  __shared__ int s_idx[4];
  __shared__ double s_gsum[NGLCM + 1];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned* qlen = p.qlen + cls;
  const int* queue = p.queue + (int64_t)cls * p.max_rois;
  const int64_t per = p.nx * p.ny * p.nz;
  const bool need_glcm = (p.need & NEED_GLCM) != 0;
  const int pad = need_glcm ? p.pad : 0;
  const double nan = __longlong_as_double(0x7FF8000000000000ll);

  for (;;) {
    if (tid == 0) {
      const unsigned w = atomicAdd(p.qhead + cls, 1u);
      s_item = w < *qlen ? queue[w] : -1;
      if (s_item >= 0) {
        s_r = p.rois[s_item];
        s_fd.init(s_r.vmax > s_r.vmin ? s_r.vmax - s_r.vmin : 1u);
      }
    }
    __syncthreads();
    const int item = s_item;
    if (item < 0) break;
    const RoiInfo r = s_r;
    const int W = r.w, H = r.h, D = NDIM == 3 ? r.d : 1;
    const int Wp = W + 2 * pad, Hp = H + 2 * pad, Dp = NDIM == 3 ? D + 2 * pad : 1;
    const int cells = Wp * Hp * Dp;
    const int n = (int)r.n;
    const int64_t bimg = (int64_t)(r.key >> 32);
    const int label = (int)(r.key & 0xFFFFFFFFu);
    const int64_t origin = bimg * per + ((int64_t)r.z0 * p.ny + r.y0) * p.nx + r.x0;
    const unsigned vmin = r.vmin, vmax = r.vmax;
    double* row = p.table + (int64_t)item * p.n_col;

    // ---- stage the ROI: raster of bins, pixel list, value histogram -------
    for (int i = tid; i < cells; i += C::NT) raster[i] = 0xFFFF;
    for (int i = tid; i < p.hist_bins; i += C::NT) hist[i] = 0;
    if (tid == 0) s_rowbase[C::NW] = 0;
    __syncthreads();
    const int nrows = H * D;
    const T* img = (const T*)p.img;
    for (int rb = 0; rb < nrows; rb += C::NW) {
      const int rr = rb + warp;
      const bool have = rr < nrows;
      const int ry = have ? rr % H : 0, rz = have ? rr / H : 0;
      const int64_t roff = origin + ((int64_t)rz * p.ny + ry) * p.nx;
      unsigned cnt = 0;
      if (have)
        for (int x0 = 0; x0 < W; x0 += 32) {
          const int x = x0 + lane;
          const bool in = x < W && __ldg(p.mask + roff + x) == label;
          cnt += __popc(__ballot_sync(0xFFFFFFFFu, in));
        }
      if (lane == 0) s_rowcnt[warp] = cnt;
      __syncthreads();
      if (tid == 0) {
        unsigned run = s_rowbase[C::NW];
        for (int w = 0; w < C::NW; ++w) {
          s_rowbase[w] = run;
          run += s_rowcnt[w];
        }
        s_rowbase[C::NW] = run;
      }
      __syncthreads();
      unsigned base = s_rowbase[warp];
      if (have)
        for (int x0 = 0; x0 < W; x0 += 32) {
          const int x = x0 + lane;
          const bool in = x < W && __ldg(p.mask + roff + x) == label;
          const unsigned bal = __ballot_sync(0xFFFFFFFFu, in);
          if (in) {
            const unsigned pos = base + __popc(bal & lanemask_lt());
            const unsigned e = Enc<T>::enc(__ldg(img + roff + x));
            if (pos < (unsigned)C::PIX) {
              pc[pos] = NDIM == 3 ? ((unsigned)x | ((unsigned)ry << 11) | ((unsigned)rz << 22))
                                  : ((unsigned)x | ((unsigned)ry << 16));
              pv[pos] = e;
            }
            // GLCM bin and histogram bin (rule a4)
            unsigned gb = 0, hb = 0;
            if (vmax > vmin) {
              if (Enc<T>::INTEGER) {
                const unsigned dv = e - vmin;
                gb = s_fd.div((unsigned)p.ng * dv);
                hb = s_fd.div((unsigned)p.hist_bins * dv);
              } else {
                const double xv = Enc<T>::dec(e), mn = Enc<T>::dec(vmin), mx = Enc<T>::dec(vmax);
                const double den = __dsub_rn(mx, mn), dx = __dsub_rn(xv, mn);
                if (need_glcm) gb = (unsigned)floor(__ddiv_rn(__dmul_rn((double)p.ng, dx), den));
                if (p.need & NEED_HIST) hb = (unsigned)floor(__ddiv_rn(__dmul_rn((double)p.hist_bins, dx), den));
              }
              gb = min(gb, (unsigned)(p.ng - 1));
              hb = min(hb, (unsigned)(p.hist_bins - 1));
            }
            if (need_glcm) raster[((rz + pad) * Hp + (ry + pad)) * Wp + (x + pad)] = (uint16_t)gb;
            if (p.need & NEED_HIST) atomicAdd(&hist[hb], 1u);
          }
          base += __popc(bal);
        }
    }
    __syncthreads();
    if (tid == 0 && s_rowbase[C::NW] != (unsigned)n) atomicOr(p.err, E_INTERNAL);

    // ---- geometry columns ----------------------------------------------------
    if (tid == 0) {
      put(p, row, Q_LABEL, (double)label);
      put(p, row, Q_IMAGE, (double)bimg);
      put(p, row, Q_AREA, (double)n);
      put(p, row, Q_BB_X, (double)r.x0);
      put(p, row, Q_BB_Y, (double)r.y0);
      put(p, row, Q_BB_Z, (double)r.z0);
      put(p, row, Q_BB_W, (double)W);
      put(p, row, Q_BB_H, (double)H);
      put(p, row, Q_BB_D, (double)D);
    }

    // ---- pass 1: exact sums (integers) --------------------------------------
    const unsigned need = p.need;
    const float fbias = std::is_same<T, int16_t>::value ? 32768.f : 0.f;
    {
      // [0] sum I, [1] sum x I, [2] sum y I, [3] sum z I, [4] sum x, [5] sum y, [6] sum z, [7] sum I^2
      long long s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      A fs[5] = {0, 0, 0, 0, 0};  // float images: sum I, x I, y I, z I, I^2
      for (int i = tid; i < n; i += C::NT) {
        const unsigned c = pc[i];
        const int x = NDIM == 3 ? (int)(c & 2047u) : (int)(c & 0xFFFFu);
        const int y = NDIM == 3 ? (int)((c >> 11) & 2047u) : (int)(c >> 16);
        const int z = NDIM == 3 ? (int)(c >> 22) : 0;
        s[4] += x;
        s[5] += y;
        s[6] += z;
        if (Enc<T>::INTEGER) {
          const int v = (int)pv[i] - (int)fbias;
          s[0] += v;
          s[1] += (long long)x * v;
          s[2] += (long long)y * v;
          s[3] += (long long)z * v;
          s[7] += (long long)v * v;
        } else {
          const A v = (A)Enc<T>::decf(pv[i]);
          fs[0] += v;
          fs[1] += (A)x * v;
          fs[2] += (A)y * v;
          fs[3] += (A)z * v;
          fs[4] += v * v;
        }
      }
      block_sum_i64<C, 8>(s, red, s_i64);
      if (!Enc<T>::INTEGER) {
        block_sum<C, A, 5>(fs, red, s_sc);
      } else if (tid == 0) {
        for (int i = 0; i < 4; ++i) s_sc[i] = (double)s_i64[i];
        s_sc[4] = (double)s_i64[7];
      }
      __syncthreads();
    }
    const double sumI = s_sc[0];
    const double energy = s_sc[4];
    const double mean = sumI / n;
    const bool wvalid = sumI != 0;
    // centre of the intensity-weighted sums (exact centroid, or the binary
    // centroid when the weights sum to zero) and the binary centroid
    const double bx = (double)s_i64[4] / n, by = (double)s_i64[5] / n, bz = (double)s_i64[6] / n;
    const double cx = wvalid ? s_sc[1] / sumI : bx, cy = wvalid ? s_sc[2] / sumI : by,
                 cz = wvalid ? s_sc[3] / sumI : bz;

    // ---- pass 2: centred sums (one loop per feature group keeps the live
    // accumulators few) -------------------------------------------------------
    constexpr int NM = NDIM == 3 ? 20 : 10;
    double* res_st = res;            // [8]  statistics
    double* res_mi = res + 8;        // [NM] intensity-weighted moments
    double* res_mb = res + 8 + NM;   // [NM] binary moments
    if (need & (NEED_STATS | NEED_SAVE)) {
      A acc[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) acc[i] = 0;
      const A mu_hi = (A)mean, mu_lo = (A)(mean - (double)mu_hi);
#pragma unroll 1
      for (int i = tid; i < n; i += C::NT) {
        const A v = Enc<T>::INTEGER ? (A)((int)pv[i] - (int)fbias) : (A)Enc<T>::decf(pv[i]);
        const A d = (v - mu_hi) - mu_lo;
        const A d2 = d * d, d3 = d2 * d, d4 = d2 * d2;
        acc[0] += d;
        acc[1] += d2;
        acc[2] += d3;
        acc[3] += d4;
        acc[4] += d4 * d;
        acc[5] += d3 * d3;
        acc[6] += d < 0 ? -d : d;
        acc[7] += d > 0 ? (A)1 : (d < 0 ? (A)-1 : (A)0);
      }
      block_sum<C, A, 8>(acc, red, res_st);
    }
#pragma unroll 1
    for (int w = 0; w < 2; ++w) {
      if (!(need & (w ? NEED_MOM_BIN : (NEED_MOM_INT | NEED_SAVE)))) continue;
      A acc[NM];
#pragma unroll
      for (int i = 0; i < NM; ++i) acc[i] = 0;
      const A c0 = (A)(w ? bx : cx), c1 = (A)(w ? by : cy), c2 = (A)(w ? bz : cz);
#pragma unroll 1
      for (int i = tid; i < n; i += C::NT) {
        const unsigned c = pc[i];
        const A u0 = (A)(NDIM == 3 ? (int)(c & 2047u) : (int)(c & 0xFFFFu)) - c0;
        const A u1 = (A)(NDIM == 3 ? (int)((c >> 11) & 2047u) : (int)(c >> 16)) - c1;
        const A u2 = (A)(NDIM == 3 ? (int)(c >> 22) : 0) - c2;
        const A wt = w ? (A)1 : (Enc<T>::INTEGER ? (A)((int)pv[i] - (int)fbias) : (A)Enc<T>::decf(pv[i]));
        A px[4], py[4], pz[4];
        px[0] = wt;
        py[0] = pz[0] = 1;
#pragma unroll
        for (int e = 1; e < 4; ++e) {
          px[e] = px[e - 1] * u0;
          py[e] = py[e - 1] * u1;
          pz[e] = pz[e - 1] * u2;
        }
#pragma unroll
        for (int a = 0; a <= 3; ++a)
#pragma unroll
          for (int b = 0; a + b <= 3; ++b)
#pragma unroll
            for (int cc = 0; cc <= (NDIM == 3 ? 3 - a - b : 0); ++cc)
              acc[midx<NDIM>(a, b, cc)] += px[a] * py[b] * pz[cc];
      }
      block_sum<C, A, NM>(acc, red, w ? res_mb : res_mi);
    }

    // ---- finalise statistics and moments (FP64, one thread per group) -------
    double* save = (need & NEED_SAVE) ? p.saved + (int64_t)item * SV_WORDS : nullptr;
    if (tid == 0)
      finalize_stats<T, NDIM>(p, row, res_st, n, mean, sumI, energy, vmin, vmax, bimg, r.x0, r.y0, r.z0, cx, cy, cz,
                              bx, by, bz, wvalid, save);
    if (tid == 32 && (need & (NEED_MOM_INT | NEED_SAVE)))
      finalize_moments<NDIM>(p, row, 0, res_mi, (double)(A)cx, (double)(A)cy, (double)(A)cz, cx, cy, cz, wvalid,
                             save ? save + SV_MU : nullptr);
    if (tid == 64 && (need & NEED_MOM_BIN))
      finalize_moments<NDIM>(p, row, 5, res_mb, (double)(A)bx, (double)(A)by, (double)(A)bz, bx, by, bz, true,
                             nullptr);
    __syncthreads();

    // ---- histogram features -------------------------------------------------
    if (need & NEED_HIST) {
      A hv[2] = {0, 0};
      const A inv = (A)1 / (A)n;
      for (int i = tid; i < p.hist_bins; i += C::NT) {
        const unsigned h = hist[i];
        if (h) {
          const A pr = (A)h * inv;
          hv[0] -= pr * alog2(pr);
          hv[1] += pr * pr;
        }
      }
      block_sum<C, A, 2>(hv, red, s_sc + 8);
      if (tid == 0) {
        put(p, row, Q_STATS + S_ENTROPY, s_sc[8]);
        put(p, row, Q_STATS + S_UNIFORMITY, s_sc[9]);
      }
    }

    // ---- GLCM ------------------------------------------------------------------
    if (need_glcm) {
      const int ng = p.ng;
      unsigned* px = marg;
      unsigned* psum = marg + ng;      // index a + b, 0 .. 2ng-2
      unsigned* pdiff = marg + 3 * ng; // index |a - b|
      int cap = 64;
      while (cap < 2 * n && cap < C::TAB) cap <<= 1;
      const bool dbg = p.dbg_roi == (int64_t)item;
      for (int di = 0; di < p.n_dist; ++di) {
        if (tid == 0)
          for (int g = 0; g <= NGLCM; ++g) s_gsum[g] = 0;
        for (int dir = 0; dir < p.n_dirs; ++dir) {
          const int oi = di * p.n_dirs + dir;
          const int dx = p.off[oi][0], dy = p.off[oi][1], dz = p.off[oi][2];
          const int olin = (dz * Hp + dy) * Wp + dx;
          for (int i = tid; i < cap; i += C::NT) tab[i] = 0;
          for (int i = tid; i < 4 * ng; i += C::NT) marg[i] = 0;
          __syncthreads();
          // accumulate pairs (q, q + o) inside the ROI
          for (int i0 = warp * 32; i0 < n; i0 += C::NT) {
            const int i = i0 + lane;
            unsigned key = 0xFFFFFFFFu;
            if (i < n) {
              const unsigned c = pc[i];
              const int x = NDIM == 3 ? (int)(c & 2047u) : (int)(c & 0xFFFFu);
              const int y = NDIM == 3 ? (int)((c >> 11) & 2047u) : (int)(c >> 16);
              const int z = NDIM == 3 ? (int)(c >> 22) : 0;
              const int ci = ((z + pad) * Hp + (y + pad)) * Wp + (x + pad);
              const unsigned a = raster[ci], b = raster[ci + olin];
              if (b != 0xFFFFu) key = a < b ? (a << 8) | b : (b << 8) | a;
            }
            const unsigned peers = __match_any_sync(0xFFFFFFFFu, key);
            if (key != 0xFFFFFFFFu && (peers & lanemask_lt()) == 0) {
              const unsigned add = (unsigned)__popc(peers);
              unsigned h = (key * 2654435761u >> 7) & (unsigned)(cap - 1);
              for (int probe = 0; probe < cap; ++probe) {
                const unsigned wv = tab[h];
                if (wv == 0) {
                  const unsigned old = atomicCAS(&tab[h], 0u, (key << 16) | add);
                  if (old == 0) break;
                  if ((old >> 16) == key) {
                    atomicAdd(&tab[h], add);
                    break;
                  }
                } else if ((wv >> 16) == key) {
                  atomicAdd(&tab[h], add);
                  break;
                }
                h = (h + 1) & (unsigned)(cap - 1);
              }
            }
          }
          __syncthreads();
          // marginals from the non-zero cells
          for (int s = tid; s < cap; s += C::NT) {
            const unsigned wv = tab[s];
            if (!wv) continue;
            const unsigned key = wv >> 16, cnt = wv & 0xFFFFu;
            const unsigned a = key >> 8, b = key & 255u;
            atomicAdd(&px[a], cnt);
            atomicAdd(&px[b], cnt);
            atomicAdd(&psum[a + b], 2 * cnt);
            atomicAdd(&pdiff[b - a], 2 * cnt);
            if (dbg) {
              p.dbg_glcm[(int64_t)oi * ng * ng + a * ng + b] = a == b ? 2 * cnt : cnt;
              p.dbg_glcm[(int64_t)oi * ng * ng + b * ng + a] = a == b ? 2 * cnt : cnt;
            }
          }
          __syncthreads();
          // exact integer first moments: T, sum (a+1) px, sum (s+2) psum, sum k pdiff
          {
            long long iv[4] = {0, 0, 0, 0};
            for (int a = tid; a < ng; a += C::NT) {
              iv[0] += px[a];
              iv[1] += (long long)(a + 1) * px[a];
              iv[3] += (long long)a * pdiff[a];
            }
            for (int s = tid; s < 2 * ng - 1; s += C::NT) iv[2] += (long long)(s + 2) * psum[s];
            block_sum_i64<C, 4>(iv, red, s_i64 + 8);
          }
          const long long Ti = s_i64[8];
          if (Ti == 0) {  // no pair for this offset: every feature NaN
            if (tid == 0 && p.per_offset)
              for (int g = 0; g < NGLCM; ++g) put(p, row, Q_GLCM_O + (di * MAX_DIRS + dir) * NGLCM + g, nan);
            __syncthreads();
            continue;
          }
          const double Td = (double)Ti;
          const double mu = (double)s_i64[9] / Td, sumave = (double)s_i64[10] / Td, difave = (double)s_i64[11] / Td;
          // centred / entropy sums in the accumulation type
          A gv[17];
#pragma unroll
          for (int k = 0; k < 17; ++k) gv[k] = 0;
          float jmax = 0.f;
          const A invT = (A)1 / (A)Td, muA = (A)mu, saA = (A)sumave, daA = (A)difave, ngA = (A)ng;
          for (int a = tid; a < ng; a += C::NT) {
            if (!px[a]) continue;
            const A pr = (A)px[a] * invT, di_ = (A)(a + 1) - muA;
            gv[0] -= pr * alog2(pr);  // HX
            gv[1] += di_ * di_ * pr;            // sigma^2
          }
          for (int s = tid; s < 2 * ng - 1; s += C::NT) {
            if (!psum[s]) continue;
            const A pr = (A)psum[s] * invT, dk = (A)(s + 2) - saA;
            gv[2] -= pr * alog2(pr);  // SUMENT
            gv[3] += dk * dk * pr;              // SUMVAR = CLUTEND
            gv[4] += dk * dk * dk * pr;         // CLUSHADE
            gv[5] += dk * dk * dk * dk * pr;    // CLUPROM
          }
          for (int k = tid; k < ng; k += C::NT) {
            if (!pdiff[k]) continue;
            const A pr = (A)pdiff[k] * invT, kk = (A)k, dk = kk - daA;
            gv[6] += kk * kk * pr;                     // CONTRAST
            gv[7] += pr / ((A)1 + kk);                 // ID = HOM1
            gv[8] += pr / ((A)1 + kk * kk);            // IDM = HOM2
            gv[9] += pr / ((A)1 + kk / ngA);           // IDN
            gv[10] += pr / ((A)1 + kk * kk / (ngA * ngA));  // IDMN
            if (k >= 1) gv[11] += pr / (kk * kk);      // IV
            gv[12] += dk * dk * pr;                    // DIFVAR
            gv[13] -= pr * alog2(pr);        // DIFENTRO
          }
          for (int s = tid; s < cap; s += C::NT) {
            const unsigned wv = tab[s];
            if (!wv) continue;
            const unsigned key = wv >> 16, cnt = wv & 0xFFFFu;
            const unsigned a = key >> 8, b = key & 255u;
            const A mult = a == b ? (A)1 : (A)2;          // cells (a,b) and (b,a)
            const A pr = (A)(a == b ? 2 * cnt : cnt) * invT;
            gv[14] += mult * pr * pr;                                       // ASM
            gv[15] -= mult * pr * alog2(pr);                                // JE
            const A ratio = (A)(a == b ? 2 * cnt : cnt) * (A)Td / ((A)px[a] * (A)px[b]);
            gv[16] += mult * pr * alog2(ratio);                             // mutual information
            jmax = fmaxf(jmax, (float)pr);
          }
          block_sum<C, A, 17>(gv, red, res);
          jmax = block_max<C>(jmax, red);
          if (tid == 0) finalize_glcm(p, row, res, mu, sumave, difave, jmax, di, dir, s_gsum);
          __syncthreads();
        }
        if (tid == 0)
          for (int g = 0; g < NGLCM; ++g)
            put(p, row, Q_GLCM_D + di * NGLCM + g, s_gsum[NGLCM] > 0 ? s_gsum[g] / s_gsum[NGLCM] : nan);
      }
    }

    // ---- order statistics: block radix sort of the encoded values -----------
    if (need & NEED_ORDER) {
      unsigned* src = tab;
      unsigned* dst = tab + C::PIX;
      for (int i = tid; i < n; i += C::NT) src[i] = pv[i];
      unsigned* cnt = marg;                 // [NW][256]
      unsigned* dtot = marg + C::NW * 256;  // [256]
      const int seg = (((n + C::NW - 1) / C::NW) + 31) & ~31;
      for (int shift = 0; shift < Enc<T>::BITS; shift += 8) {
        for (int i = tid; i < C::NW * 256; i += C::NT) cnt[i] = 0;
        __syncthreads();
        const int lo = warp * seg, hi = min(n, lo + seg);
        for (int i0 = lo; i0 < hi; i0 += 32) {
          const int i = i0 + lane;
          const bool act = i < hi;
          const unsigned dg = act ? (src[i] >> shift) & 255u : 256u + lane;
          const unsigned peers = __match_any_sync(0xFFFFFFFFu, dg);
          const unsigned before = __popc(peers & lanemask_lt());
          unsigned b0 = 0;
          if (act) b0 = cnt[warp * 256 + dg];
          __syncwarp();
          if (act) {
            rank[i] = (uint16_t)(b0 + before);
            if (before == 0) cnt[warp * 256 + dg] = b0 + __popc(peers);
          }
          __syncwarp();
        }
        __syncthreads();
        // digit-major, then warp, exclusive offsets
        for (int d = tid; d < 256; d += C::NT) {
          unsigned t = 0;
          for (int w = 0; w < C::NW; ++w) t += cnt[w * 256 + d];
          dtot[d] = t;
        }
        __syncthreads();
        if (warp == 0) warp_exclusive_scan(dtot, 256);
        __syncthreads();
        for (int d = tid; d < 256; d += C::NT) {
          unsigned run = dtot[d];
          for (int w = 0; w < C::NW; ++w) {
            const unsigned c = cnt[w * 256 + d];
            cnt[w * 256 + d] = run;
            run += c;
          }
        }
        __syncthreads();
        for (int i = lo + lane; i < hi; i += 32) {
          const unsigned k = src[i];
          dst[cnt[warp * 256 + ((k >> shift) & 255u)] + rank[i]] = k;
        }
        __syncthreads();
        unsigned* t = src;
        src = dst;
        dst = t;
      }
      const unsigned* v = src;  // sorted, ascending
      if (tid == 0) finalize_percentiles<T>(p, row, v, n, s_sc, s_idx);
      __syncthreads();
      // mode: longest run of equal values, ties -> smallest value.  Each
      // thread owns a contiguous segment; runs entering a segment get their
      // start from an exclusive max-scan of the previous segments.
      const int per_t = (n + C::NT - 1) / C::NT;
      const int s0 = min(n, tid * per_t), s1 = min(n, s0 + per_t);
      int last_start = -1;
      for (int i = s0; i < s1; ++i)
        if (i == 0 || v[i] != v[i - 1]) last_start = i;
      {
        // exclusive max-scan of last_start over threads
        int* sc = (int*)red;
        sc[tid] = last_start;
        __syncthreads();
        if (tid == 0) {
          int run = -1;
          for (int t = 0; t < C::NT; ++t) {
            const int x = sc[t];
            sc[t] = run;
            if (x > run) run = x;
          }
        }
        __syncthreads();
        last_start = sc[tid];
        __syncthreads();
      }
      unsigned long long best = 0;  // (length << 32) | ~value: max = longest, then smallest
      int start = last_start;
      for (int i = s0; i < s1; ++i) {
        if (i == 0 || v[i] != v[i - 1]) start = i;
        if (i == n - 1 || v[i] != v[i + 1]) {
          const unsigned long long cand = ((unsigned long long)(i - start + 1) << 32) | (unsigned)(~v[i]);
          if (cand > best) best = cand;
        }
      }
      best = block_max_u64<C>(best, red);
      // robust mean, median absolute deviation
      const int i10 = s_idx[0], i90 = s_idx[1];
      const double med = s_sc[0];
      const A medA = (A)med;
      A rv[2] = {0, 0};
      for (int i = tid; i < n; i += C::NT) {
        const A x = (A)Enc<T>::dec(v[i]);
        if (i >= i10 && i < i90) rv[0] += x;
        rv[1] += x > medA ? x - medA : medA - x;
      }
      block_sum<C, A, 2>(rv, red, s_sc + 4);
      const int cntV = i90 - i10;
      const double rmean = s_sc[4] / cntV;
      const A rmA = (A)rmean;
      A ra[1] = {0};
      for (int i = i10 + tid; i < i90; i += C::NT) {
        const A x = (A)Enc<T>::dec(v[i]);
        ra[0] += x > rmA ? x - rmA : rmA - x;
      }
      block_sum<C, A, 1>(ra, red, s_sc + 6);
      if (tid == 0) {
        put(p, row, Q_STATS + S_MODE, Enc<T>::dec(~(unsigned)(best & 0xFFFFFFFFu)));
        put(p, row, Q_STATS + S_MODE_PROB, (double)(best >> 32) / n);
        put(p, row, Q_STATS + S_RMEAN, cntV > 0 ? rmean : nan);
        put(p, row, Q_STATS + S_RMAD, cntV > 0 ? s_sc[6] / cntV : nan);
        put(p, row, Q_STATS + S_MEDAD, s_sc[5] / n);
      }
    }
    __syncthreads();
  }
}

}  // namespace nyx

namespace nyx {

// Launch one persistent instantiation of the ROI kernel: as many blocks as
// fit on the device at once (occupancy x SMs); blocks drain the class queue.
template <class T, int NDIM, class C, class A>
cudaError_t launch_roi_one(const KParams& p, int cls, int nsm, cudaStream_t st) {
  auto kern = k_roi<T, NDIM, C, A>;
  const SmemLayout L = SmemLayout::make<C>(p.ng, p.hist_bins);
  const int smem = L.total;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  static int configured[64] = {0};
  if (dev < 64 && configured[dev] < smem) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    configured[dev] = smem;
  }
  int nb = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, C::NT, smem);
  if (e != cudaSuccess) return e;
  if (nb < 1) return cudaErrorInvalidConfiguration;
  kern<<<nb * nsm, C::NT, smem, st>>>(p, cls);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_roi_t(const KParams& p, int cls, int fp64, int nsm, cudaStream_t st) {
  if (p.ndim == 3) {
    if (cls == 0)
      return fp64 ? launch_roi_one<T, 3, ClassS, double>(p, cls, nsm, st) : launch_roi_one<T, 3, ClassS, float>(p, cls, nsm, st);
    return fp64 ? launch_roi_one<T, 3, ClassM, double>(p, cls, nsm, st) : launch_roi_one<T, 3, ClassM, float>(p, cls, nsm, st);
  }
  if (cls == 0)
    return fp64 ? launch_roi_one<T, 2, ClassS, double>(p, cls, nsm, st) : launch_roi_one<T, 2, ClassS, float>(p, cls, nsm, st);
  return fp64 ? launch_roi_one<T, 2, ClassM, double>(p, cls, nsm, st) : launch_roi_one<T, 2, ClassM, float>(p, cls, nsm, st);
}

}  // namespace nyx
