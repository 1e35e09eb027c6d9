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
//   edge intensity statistics (Table S1 rows 3-7): a face-neighbour test on
//       the raster, folded into the two statistics passes
//   NGTDM and GLDM (Table S3 rows 246-264): one visit of each pixel's
//       Chebyshev-1 neighbours in the raster gives the NGTDM level sums and
//       the GLDM dependence; per-level integer / fixed-point sums in shared
//       memory, (level, dependence) cells in the shared hash table
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

template <int NT_, int PIX_, int CELLS_, int MINB_ = 1>
struct RoiClass {
  static constexpr int NT = NT_;
  static constexpr int MINB = MINB_;    // resident blocks per SM the register budget is set for
  static constexpr int NW = NT_ / 32;
  static constexpr int PIX = PIX_;      // max pixels of an ROI
  static constexpr int CELLS = CELLS_;  // max padded raster cells
  static constexpr int TAB = 2 * PIX_;  // GLCM hash capacity (power of two); also 2 sort buffers
};
using ClassW = RoiClass<32, 256, 1024>;    // one warp per ROI
using ClassS = RoiClass<128, 1024, 4096, 6>;  // 6 blocks of ~35 KB shared memory fit an SM
using ClassM = RoiClass<256, 4096, 8192, 2>;  // 2 blocks of ~100 KB fit an SM
using ClassL = RoiClass<512, 8192, 16384>;    // one block of ~200 KB per SM

constexpr int RED_MAX = 32;  // max values per block reduction (and per warp slot of the scratch)

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
    int marg = 4 * (4 * (ng > 0 ? ng : 1) + 32);  // 4 words per grey level + the GLDM column sums
    int cnts = 4 * (C::NW * 256 + 256);
    L.marg = o;   o = align16(o + (marg > cnts ? marg : cnts));
    L.red = o;    o = align16(o + 8 * C::NW * RED_MAX);
    L.res = o;    o = align16(o + 8 * (RED_MAX + 2 * NGLCM + 16));
    L.total = o;
    return L;
  }
};

// ----------------------------------------------------------------------------
// Arithmetic discipline.  GB300's FP64 pipe retires a few thread-operations
// per clock per SM and occupies it for a whole warp instruction even when one
// lane is active, so the fast path keeps every per-pixel AND per-ROI step in
// the accumulation type A (float), converts results to the FP64 table with
// integer bit manipulation, and uses FP64 arithmetic only where an output must
// match a double-precision definition bit for bit (percentile interpolation).
// With A = double (the plain FP64 path) the same code runs in FP64.

// exact float -> double without the FP64 pipe
__device__ inline double f2d(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
  const unsigned ex = (u >> 23) & 0xFFu, man = u & 0x7FFFFFu;
  unsigned long long bits;
  if (ex == 0xFFu) {
    bits = sign | 0x7FF0000000000000ull | ((unsigned long long)man << 29);
  } else if (ex != 0) {
    bits = sign | ((unsigned long long)(ex + 896u) << 52) | ((unsigned long long)man << 29);
  } else if (man == 0) {
    bits = sign;
  } else {  // subnormal float: normalise
    const int lz = __clz(man) - 8;  // leading zeros within the 23-bit field
    const unsigned m = (man << (lz + 1)) & 0x7FFFFFu;
    bits = sign | ((unsigned long long)(896 - lz) << 52) | ((unsigned long long)m << 29);
  }
  return __longlong_as_double((long long)bits);
}

// f * 2^e2 as a double (exact; the result is assumed to be a normal double)
__device__ inline double f2d_scaled(float f, int e2) {
  double d = f2d(f);
  long long b = __double_as_longlong(d);
  const long long ex = (b >> 52) & 0x7FF;
  if (ex == 0 || ex == 0x7FF) return d;  // zero / inf / nan unchanged
  b += (long long)e2 << 52;
  return __longlong_as_double(b);
}

// exact integer -> double for |v| < 2^53 without the FP64 pipe
__device__ inline double i2d(long long v) {
  if (v == 0) return 0.0;
  const unsigned long long sign = v < 0 ? (1ull << 63) : 0ull;
  const unsigned long long a = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
  const int msb = 63 - __clzll((long long)a);
  const unsigned long long man = (a << (52 - msb)) & ((1ull << 52) - 1);
  return __longlong_as_double((long long)(sign | ((unsigned long long)(msb + 1023) << 52) | man));
}

__device__ inline double to_d(float v) { return f2d(v); }
__device__ inline double to_d(double v) { return v; }

__device__ inline void put(const KParams& p, double* row, int q, double v) {
  const int c = __ldg(p.col_map + q);
  if (c >= 0) row[c] = v;
}
template <class A>
__device__ inline void putA(const KParams& p, double* row, int q, A v) {
  const int c = __ldg(p.col_map + q);
  if (c >= 0) row[c] = to_d(v);
}

__device__ inline float alog2(float x) { return log2f(x); }
__device__ inline double alog2(double x) { return log2(x); }
__device__ inline float asqrt(float x) { return sqrtf(x); }
__device__ inline double asqrt(double x) { return sqrt(x); }
__device__ inline float aexp(float x) { return expf(x); }
__device__ inline double aexp(double x) { return exp(x); }
__device__ inline float aexpm1(float x) { return expm1f(x); }
__device__ inline double aexpm1(double x) { return expm1(x); }
__device__ inline float acbrt(float x) { return cbrtf(x); }
__device__ inline double acbrt(double x) { return cbrt(x); }

template <class A>
__device__ inline A anan() {
  if constexpr (std::is_same<A, float>::value) return __int_as_float(0x7FC00000);
  else return __longlong_as_double(0x7FF8000000000000ll);
}

// decode an encoded value straight into the accumulation type
template <class T, class A>
__device__ inline A decA(unsigned e) {
  if constexpr (std::is_same<A, float>::value) return Enc<T>::decf(e);
  else return Enc<T>::dec(e);
}

// Edge test of one ROI pixel (packed bbox-local coordinates c, as in the
// pixel list) on the padded raster (pad >= 1): true when a face neighbour is
// not a cell of the ROI.
template <int NDIM>
__device__ inline bool edge_pixel(const uint16_t* raster, unsigned c, int pad, int Wp, int Hp, int plane) {
  const int x = NDIM == 3 ? (int)(c & 2047u) : (int)(c & 0xFFFFu);
  const int y = NDIM == 3 ? (int)((c >> 11) & 2047u) : (int)(c >> 16);
  const int z = NDIM == 3 ? (int)(c >> 22) : 0;
  const int ri = ((NDIM == 3 ? z + pad : 0) * Hp + (y + pad)) * Wp + (x + pad);
  const unsigned a0 = raster[ri - 1], a1 = raster[ri + 1], a2 = raster[ri - Wp], a3 = raster[ri + Wp];
  bool e = (a0 == 0xFFFFu) | (a1 == 0xFFFFu) | (a2 == 0xFFFFu) | (a3 == 0xFFFFu);
  if (NDIM == 3) {
    const unsigned a4 = raster[ri - plane], a5 = raster[ri + plane];
    e |= (a4 == 0xFFFFu) | (a5 == 0xFFFFu);
  }
  return e;
}

// ----------------------------------------------------------------------------
// block reductions (results are left in shared memory for every thread)

// Slots of a warp reduce-scatter: the power of two at or above NV (<= 32).
template <int NV>
struct RsSlots {
  static constexpr int S = NV <= 1 ? 1 : NV <= 2 ? 2 : NV <= 4 ? 4 : NV <= 8 ? 8 : NV <= 16 ? 16 : 32;
  static constexpr int SH = S == 1 ? 5 : S == 2 ? 4 : S == 4 ? 3 : S == 8 ? 2 : S == 16 ? 1 : 0;  // log2(32 / S)
};

// Warp sums of NV values by recursive halving (reduce-scatter): at partner
// distance o each lane keeps half of its slots and adds the other half
// received from lane ^ o, so S slots cost S - 1 exchanges instead of 5 per
// value; a butterfly over the remaining lane bits finishes.  Afterwards lane
// l holds the warp total of slot l >> SH.  Float values travel as
// compensated (hi, lo) pairs merged with two-sum; the order of operations is
// fixed, so results are deterministic.
template <class A, int NV>
__device__ inline void warp_rs(const A (&v)[NV], A& hi_out, A& lo_out, const A* v_lo = nullptr) {
  constexpr int S = RsSlots<NV>::S;
  const int lane = threadIdx.x & 31;
  A hi[S], lo[S];
#pragma unroll
  for (int i = 0; i < S; ++i) {
    hi[i] = i < NV ? v[i] : (A)0;
    lo[i] = (i < NV && v_lo) ? v_lo[i] : (A)0;
  }
#pragma unroll
  for (int h = S / 2, o = 16; h >= 1; h >>= 1, o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const A sh = up ? hi[i] : hi[i + h], sl = up ? lo[i] : lo[i + h];
      const A kh = up ? hi[i + h] : hi[i], kl = up ? lo[i + h] : lo[i];
      const A rh = __shfl_xor_sync(0xFFFFFFFFu, sh, o);
      if constexpr (std::is_same<A, float>::value) {
        const float rl = __shfl_xor_sync(0xFFFFFFFFu, sl, o);
        float s_, e_;
        two_sum(kh, rh, s_, e_);
        hi[i] = s_;
        lo[i] = __fadd_rn(__fadd_rn(kl, rl), e_);
      } else {
        hi[i] = kh + rh;
        (void)sl;
        (void)kl;
      }
    }
  }
#pragma unroll
  for (int o = 16 >> (5 - RsSlots<NV>::SH); o >= 1; o >>= 1) {  // lane bits below the slot bits
    const A rh = __shfl_xor_sync(0xFFFFFFFFu, hi[0], o);
    if constexpr (std::is_same<A, float>::value) {
      const float rl = __shfl_xor_sync(0xFFFFFFFFu, lo[0], o);
      float s_, e_;
      two_sum(hi[0], rh, s_, e_);
      hi[0] = s_;
      lo[0] = __fadd_rn(__fadd_rn(lo[0], rl), e_);
    } else {
      hi[0] += rh;
    }
  }
  hi_out = hi[0];
  lo_out = lo[0];
}

template <class C, class A, int NV>
__device__ inline void block_sum(A (&v)[NV], double* scratch, A* out) {
  static_assert(NV <= RED_MAX && NV <= 32, "reduction too wide");
  constexpr int SH = RsSlots<NV>::SH;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  A hi, lo;
  warp_rs<A, NV>(v, hi, lo);
  const int slot = lane >> SH;
  if constexpr (std::is_same<A, float>::value) {
    float2* sc = (float2*)scratch;
    if ((lane & ((1 << SH) - 1)) == 0 && slot < NV) sc[warp * NV + slot] = make_float2(hi, lo);
    __syncthreads();
    for (int i = threadIdx.x; i < NV; i += C::NT) {
      float h = 0.f, l = 0.f;
      for (int w = 0; w < C::NW; ++w) {
        const float2 x = sc[w * NV + i];
        float s_, e_;
        two_sum(h, x.x, s_, e_);
        h = s_;
        l = __fadd_rn(__fadd_rn(l, x.y), e_);
      }
      out[i] = __fadd_rn(h, l);
    }
  } else {
    (void)lo;
    if ((lane & ((1 << SH) - 1)) == 0 && slot < NV) scratch[warp * NV + slot] = hi;
    __syncthreads();
    for (int i = threadIdx.x; i < NV; i += C::NT) {
      double t = 0;
      for (int w = 0; w < C::NW; ++w) t += scratch[w * NV + i];
      out[i] = t;
    }
  }
  __syncthreads();
}

// Kahan-compensated running sum (per thread)
template <class A>
struct KSum {
  A s, c;
  __device__ KSum() : s(0), c(0) {}
  __device__ void add(A x) {
    const A y = x - c;
    const A t = s + y;
    c = (t - s) - y;
    s = t;
  }
};

// Block sums of per-thread compensated float pairs (v.s - v.c), kept as
// unrounded (hi, lo) pairs: out_hi[i] + out_lo[i] in FP64 is the total to
// about 2^-44 relative, as the FP64 centroid and mean need.  Results in
// shared memory for every thread.
template <class C, int NV>
__device__ inline void block_sum_pair(const KSum<float> (&v)[NV], double* scratch, float* out_hi, float* out_lo) {
  static_assert(NV <= RED_MAX && NV <= 32, "reduction too wide");
  constexpr int SH = RsSlots<NV>::SH;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float vh[NV], vl[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    vh[i] = v[i].s;
    vl[i] = -v[i].c;
  }
  float hi, lo;
  warp_rs<float, NV>(vh, hi, lo, vl);
  const int slot = lane >> SH;
  float2* sc = (float2*)scratch;
  if ((lane & ((1 << SH) - 1)) == 0 && slot < NV) sc[warp * NV + slot] = make_float2(hi, lo);
  __syncthreads();
  for (int i = threadIdx.x; i < NV; i += C::NT) {
    float h = 0.f, l = 0.f;
    for (int w = 0; w < C::NW; ++w) {
      const float2 x = sc[w * NV + i];
      float s_, e_;
      two_sum(h, x.x, s_, e_);
      h = s_;
      l = __fadd_rn(__fadd_rn(l, x.y), e_);
    }
    two_sum(h, l, out_hi[i], out_lo[i]);  // normalised pair
  }
  __syncthreads();
}

// (hi, lo) float pair -> the nearest double of hi + lo, and a double split
// into a float pair
__device__ inline double pair_d(float hi, float lo) { return f2d(hi) + f2d(lo); }

template <class C, int NV>
__device__ inline void block_sum_i64(long long (&v)[NV], double* scratch_d, long long* out) {
  long long* scratch = (long long*)scratch_d;
  constexpr int SH = RsSlots<NV>::SH;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long hi, lo;
  warp_rs<long long, NV>(v, hi, lo);
  (void)lo;
  const int slot = lane >> SH;
  if ((lane & ((1 << SH) - 1)) == 0 && slot < NV) scratch[warp * NV + slot] = hi;
  __syncthreads();
  for (int i = threadIdx.x; i < NV; i += C::NT) {
    long long t = 0;
    for (int w = 0; w < C::NW; ++w) t += scratch[w * NV + i];
    out[i] = t;
  }
  __syncthreads();
}

// Block minimum and maximum of two unsigned values; results in mn / mx of
// every thread.
template <class C>
__device__ inline void block_minmax_u32(unsigned& mn, unsigned& mx, double* scratch_d) {
  unsigned* scratch = (unsigned*)scratch_d;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  mn = __reduce_min_sync(0xFFFFFFFFu, mn);
  mx = __reduce_max_sync(0xFFFFFFFFu, mx);
  if (lane == 0) {
    scratch[2 * warp] = mn;
    scratch[2 * warp + 1] = mx;
  }
  __syncthreads();
  for (int w = 0; w < C::NW; ++w) {
    mn = min(mn, scratch[2 * w]);
    mx = max(mx, scratch[2 * w + 1]);
  }
  __syncthreads();
}

template <class C>
__device__ inline unsigned long long block_max_u64(unsigned long long v, double* scratch_d) {
  unsigned long long* scratch = (unsigned long long*)scratch_d;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long u = __shfl_xor_sync(0xFFFFFFFFu, v, o);
    v = u > v ? u : v;
  }
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  unsigned long long m = scratch[0];
  for (int w = 1; w < C::NW; ++w) m = scratch[w] > m ? scratch[w] : m;
  __syncthreads();
  return m;
}

// Run-length merge of equal keys held by consecutive lanes (every lane of the
// warp calls it; `invalid` marks lanes without a key).  Returns the run length
// in the first lane of each run of valid keys, 0 elsewhere.  Smooth images
// give long runs of equal co-occurrence cells or histogram bins along x; one
// atomic per run replaces up to 32 conflicting ones on the same address.
__device__ inline unsigned run_leader(unsigned key, unsigned invalid) {
  const int lane = threadIdx.x & 31;
  const unsigned prev = __shfl_up_sync(0xFFFFFFFFu, key, 1);
  const bool lead = lane == 0 || key != prev;
  const unsigned leads = __ballot_sync(0xFFFFFFFFu, lead);
  if (!lead || key == invalid) return 0u;
  const unsigned above = lane == 31 ? 0u : (leads & (0xFFFFFFFFu << (lane + 1)));
  return (unsigned)((above ? __ffs(above) - 1 : 32) - lane);
}

// Add `add` to the count of 16-bit `key` in a shared open-addressing table of
// (key << 16 | count) words (cap a power of two, at most half full, so the
// probe ends); a newly occupied slot is appended to cells[].
__device__ __forceinline__ void tab_add(unsigned* tab, int cap, unsigned key, unsigned add, uint16_t* cells,
                                        unsigned* ncell) {
  unsigned h = (key * 2654435761u >> 7) & (unsigned)(cap - 1);
  for (int probe = 0; probe < cap; ++probe) {
    const unsigned wv = tab[h];
    if (wv == 0) {
      const unsigned old = atomicCAS(&tab[h], 0u, (key << 16) | add);
      if (old == 0) {
        cells[atomicAdd(ncell, 1u)] = (uint16_t)h;
        return;
      }
      if ((old >> 16) == key) {
        atomicAdd(&tab[h], add);
        return;
      }
    } else if ((wv >> 16) == key) {
      atomicAdd(&tab[h], add);
      return;
    }
    h = (h + 1) & (unsigned)(cap - 1);
  }
}

// ----------------------------------------------------------------------------
// moments helpers

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

// binomial coefficients C(n, k) for n <= 6
__device__ __constant__ const signed char c_binom[7][7] = {{1},          {1, 1},          {1, 2, 1},
                                                           {1, 3, 3, 1}, {1, 4, 6, 4, 1}, {1, 5, 10, 10, 5, 1},
                                                           {1, 6, 15, 20, 15, 6, 1}};

// Hu's seven invariants (Hu 1962) from normalised central moments.
template <class A>
__device__ inline void hu7(A n20, A n02, A n11, A n30, A n21, A n12, A n03, A* h) {
  const A a = n30 - 3 * n12, b = 3 * n21 - n03, s = n30 + n12, t = n21 + n03;
  h[0] = n20 + n02;
  h[1] = (n20 - n02) * (n20 - n02) + 4 * n11 * n11;
  h[2] = a * a + b * b;
  h[3] = s * s + t * t;
  h[4] = a * s * (s * s - 3 * t * t) + b * t * (3 * s * s - t * t);
  h[5] = (n20 - n02) * (s * s - t * t) + 4 * n11 * s * t;
  h[6] = b * s * (s * s - 3 * t * t) - a * t * (3 * s * s - t * t);
}

// normalisation mu00^(1 + o/2) (2D) or mu000^(1 + o/3) (3D): a real power of
// a negative mu000 exists only for an integer exponent (NaN otherwise, as
// for the FP64 power function)
template <int NDIM, class A>
__device__ inline A norm_pow(A m00, int o) {
  if (NDIM == 2) {
    switch (o) {
      case 0: return m00;
      case 1: return m00 * asqrt(m00);
      case 2: return m00 * m00;
      default: return m00 * m00 * asqrt(m00);
    }
  }
  if (m00 < 0 && (o == 1 || o == 2)) return anan<A>();
  const A c = acbrt(m00);
  switch (o) {
    case 0: return m00;
    case 1: return m00 * c;
    case 2: return m00 * c * c;
    default: return m00 * m00;
  }
}

// One weighting's moments, one lane per moment (every lane of the warp calls
// it).  Cs[] are the sums sum w (x - s0)^p (y - s1)^q (z - s2)^r about the
// centre s, an FP32 point inside the bounding box: the weighted centroid
// when it lies in the box, else the binary centroid (a signed intensity
// image whose weights nearly cancel puts the weighted centroid far outside,
// where the expansions below would cancel catastrophically).  With W the
// total weight and ci the FP64 weighted centroid, the first-order sums are
// W (ci - s) exactly; raw moments follow by the binomial expansion about s,
// central moments by the expansion about s - ci (zero when s is ci's
// rounding).  valid = false (zero total weight) leaves raw moments finite
// and every derived value NaN.  Hu invariants are evaluated on eta rescaled
// to O(1) and scaled back by an exact power of two, so tiny
// intensity-weighted invariants neither underflow nor lose precision in
// FP32.
template <int NDIM, class A>
__device__ __noinline__ void finalize_moments_warp(const KParams& p, double* row, int wbase, const A* Cs, A s0, A s1,
                                                   A s2, const double* ci, double W, bool valid, double* save_mu,
                                                   bool on = true, int lb = 0) {
  constexpr int NM = NDIM == 3 ? 20 : 10;
  const int lane = (int)(threadIdx.x & 31) - lb;  // index within this lane's group of moments
  const bool act = on && lane >= 0 && lane < NM;
  const A nan = anan<A>();
  int a = 0, b = 0, c = 0;
  if (act) mexp<NDIM>(lane, a, b, c);
  const int o = a + b + c;
  const A f1[3] = {(A)(W * (ci[0] - (double)s0)), (A)(W * (ci[1] - (double)s1)),
                   (A)(NDIM == 3 ? W * (ci[2] - (double)s2) : 0.0)};
  const A d0 = (A)((double)s0 - ci[0]), d1 = (A)((double)s1 - ci[1]), d2 = (A)(NDIM == 3 ? (double)s2 - ci[2] : 0.0);
  const A pw0[4] = {1, s0, s0 * s0, s0 * s0 * s0}, pw1[4] = {1, s1, s1 * s1, s1 * s1 * s1},
          pw2[4] = {1, s2, s2 * s2, s2 * s2 * s2};
  const A pd0[4] = {1, d0, d0 * d0, d0 * d0 * d0}, pd1[4] = {1, d1, d1 * d1, d1 * d1 * d1},
          pd2[4] = {1, d2, d2 * d2, d2 * d2 * d2};
  A M = 0, mu = 0;
  if (act)
    for (int i = 0; i <= a; ++i)
      for (int j = 0; j <= b; ++j)
        for (int l = 0; l <= c; ++l) {
          const int q = i + j + l;
          const A sv = q == 1 ? f1[i ? 0 : (j ? 1 : 2)] : Cs[midx<NDIM>(i, j, l)];
          const A bc = (A)(c_binom[a][i] * c_binom[b][j] * c_binom[c][l]);
          M += bc * pw0[a - i] * pw1[b - j] * pw2[c - l] * sv;
          mu += bc * pd0[a - i] * pd1[b - j] * pd2[c - l] * sv;
        }
  if (o == 1) mu = 0;  // first-order central moments vanish at the centroid
  // the central moments the Hu invariants need, from their lanes
  const A m20 = __shfl_sync(0xFFFFFFFFu, mu, lb + midx<NDIM>(2, 0, 0)),
          m02 = __shfl_sync(0xFFFFFFFFu, mu, lb + midx<NDIM>(0, 2, 0)),
          m11 = __shfl_sync(0xFFFFFFFFu, mu, lb + midx<NDIM>(1, 1, 0)),
          m30 = __shfl_sync(0xFFFFFFFFu, mu, lb + midx<NDIM>(3, 0, 0)),
          m21 = __shfl_sync(0xFFFFFFFFu, mu, lb + midx<NDIM>(2, 1, 0)),
          m12 = __shfl_sync(0xFFFFFFFFu, mu, lb + midx<NDIM>(1, 2, 0)),
          m03 = __shfl_sync(0xFFFFFFFFu, mu, lb + midx<NDIM>(0, 3, 0));
  if (!act) return;
  const A mu00 = Cs[0];
  putA(p, row, Q_MOM + (wbase + F_M) * 20 + lane, M);
  putA(p, row, Q_MOM + (wbase + F_MU) * 20 + lane, valid ? mu : nan);
  if (o >= 2) putA(p, row, Q_MOM + (wbase + F_ETA) * 20 + lane, valid ? mu / norm_pow<NDIM>(mu00, o) : nan);
  if (NDIM == 2) putA(p, row, Q_MOM + (wbase + F_NU) * 20 + lane, valid ? M / norm_pow<NDIM>(mu00, o) : nan);
  if (save_mu) save_mu[lane] = to_d(mu);
  if (NDIM == 2) {  // every active lane computes the invariants, lane i stores the i-th
    const A g20 = norm_pow<2>(mu00, 2), g30 = norm_pow<2>(mu00, 3);
    const A e20 = m20 / g20, e02 = m02 / g20, e11 = m11 / g20;
    // scale lambda = 2^k close to eta20 + eta02: eta_o / lambda^(o/2) = O(1)
    int k = 0;
    if (valid) {
      const A s2 = (e20 > 0 ? e20 : -e20) + (e02 > 0 ? e02 : -e02);
      int ex;
      if constexpr (std::is_same<A, float>::value) (void)frexpf(s2, &ex);
      else (void)frexp(s2, &ex);
      k = s2 > 0 ? ex : 0;
      k &= ~1;  // even, so that lambda^(1/2) and lambda^(3/2) are exact powers of two
    }
    A il, il15;
    if constexpr (std::is_same<A, float>::value) {
      il = ldexpf(1.f, -k);
      il15 = ldexpf(1.f, -(3 * k) / 2);
    } else {
      il = ldexp(1.0, -k);
      il15 = ldexp(1.0, -(3 * k) / 2);
    }
    A h[7];
    hu7<A>(e20 * il, e02 * il, e11 * il, m30 / g30 * il15, m21 / g30 * il15, m12 / g30 * il15, m03 / g30 * il15, h);
    constexpr int deg[7] = {1, 2, 3, 3, 6, 4, 6};  // degree of each invariant in eta20-like units
    A hm = 0;
    int dm = 0;
#pragma unroll
    for (int i = 0; i < 7; ++i)
      if (lane == i) {
        hm = h[i];
        dm = deg[i];
      }
    if (lane < 7) {
      double v;
      if constexpr (std::is_same<A, float>::value) v = f2d_scaled(hm, k * dm);
      else v = ldexp(hm, k * dm);
      put(p, row, Q_MOM + (wbase + F_HU) * 20 + lane, valid ? v : to_d(nan));
    }
  }
}

// Statistics of Table S1 / S5 from the centred power sums S_k = sum (I - c)^k
// about a centring point c close to the mean; the residual offset S_1 / n is
// removed by a binomial shift.  Called by all 32 lanes of a warp.
template <class T, int NDIM, class A>
__device__ __noinline__ void finalize_stats(const KParams& p, double* row, const A* res_st, int n, A mean, A sumI,
                                            A energy, unsigned vmin, unsigned vmax, int64_t bimg, int x0, int y0,
                                            int z0, const double* cd, bool wvalid, double* save) {
  const A nan = anan<A>();
  const A nA = (A)n;
  const A dl = res_st[0] / nA;
  A pd[7];
  pd[0] = 1;
  for (int k = 1; k <= 6; ++k) pd[k] = pd[k - 1] * -dl;
  A m[7];
  m[0] = 1;
  for (int k = 1; k <= 6; ++k) {
    A s = pd[k] * nA;  // j = 0 term: S_0 = n
    for (int j = 1; j <= k; ++j) s += (A)c_binom[k][j] * pd[k - j] * res_st[j - 1];
    m[k] = s / nA;
  }
  const A m2 = m[2] > 0 ? m[2] : (A)0;
  const A var = n > 1 ? m2 * nA / (nA - 1) : (A)0;
  const A sd = asqrt(var);
  const A mn = decA<T, A>(vmin), mx = decA<T, A>(vmax);
  const A imn = decA<T, A>(p.img_vmin[bimg]), imx = decA<T, A>(p.img_vmax[bimg]);
  const bool pos = m2 > 0;
  const A kurt = pos ? m[4] / (m2 * m2) : (A)0;
  // every lane of the warp computes every value; lane j stores value j, so
  // the columns leave in one warp-wide store instead of one after another
  constexpr int NA = 16;
  const A va[NA] = {mean,
                    var,
                    m2,
                    sd,
                    asqrt(m2),
                    pos ? m[3] / (m2 * asqrt(m2)) : (A)0,
                    kurt,
                    pos ? kurt - 3 : (A)0,
                    pos ? m[5] / (m2 * m2 * asqrt(m2)) : (A)0,
                    pos ? m[6] / (m2 * m2 * m2) : (A)0,
                    asqrt(energy / nA),
                    sd / asqrt(nA),
                    res_st[6] / nA,
                    mean != 0 ? sd / mean : nan,
                    imx != imn ? (mx - mn) / (imx - imn) : nan,
                    (mx + mn) != 0 ? (A)100 * ((A)1 - (mx - mn) / (mx + mn)) : nan};
  constexpr int qa[NA] = {S_MEAN, S_VAR, S_VAR_B, S_STD, S_STD_B, S_SKEW, S_KURT, S_EXKURT,
                          S_HSKEW, S_HFLAT, S_RMS, S_SE, S_MAD, S_COV, S_COVERED, S_PIU};
  // centroids in image coordinates: integer origin + the FP64 local centroid;
  // the mass displacement is the FP64 distance of the two centroids, which
  // nearly coincide in symmetric ROIs (an FP32 difference would keep few
  // digits of it)
  double md = (cd[0] - cd[3]) * (cd[0] - cd[3]) + (cd[1] - cd[4]) * (cd[1] - cd[4]);
  if (NDIM == 3) md += (cd[2] - cd[5]) * (cd[2] - cd[5]);
  constexpr int ND = 7;
  const double vd[ND] = {i2d(x0) + cd[3],
                         i2d(y0) + cd[4],
                         i2d(z0) + cd[5],
                         wvalid ? i2d(x0) + cd[0] : to_d(nan),
                         wvalid ? i2d(y0) + cd[1] : to_d(nan),
                         wvalid ? i2d(z0) + cd[2] : to_d(nan),
                         wvalid ? sqrt(md) : to_d(nan)};
  constexpr int qd[ND] = {Q_CEN_X, Q_CEN_Y, Q_CEN_Z, Q_STATS + S_WCX, Q_STATS + S_WCY, Q_STATS + S_WCZ,
                          Q_STATS + S_MD};
  const int lane = threadIdx.x & 31;
  A a_mine = 0;
  double d_mine = 0;
  int q_mine = -1;
#pragma unroll
  for (int j = 0; j < NA; ++j)
    if (lane == j) {
      a_mine = va[j];
      q_mine = Q_STATS + qa[j];
    }
#pragma unroll
  for (int j = 0; j < ND; ++j)
    if (lane == NA + j) q_mine = qd[j];
#pragma unroll
  for (int j = 0; j < ND; ++j)
    if (lane == NA + j) d_mine = vd[j];
  if (lane < NA) putA(p, row, q_mine, a_mine);
  else if (q_mine >= 0) put(p, row, q_mine, d_mine);
  if (save && lane == 0) {
    save[SV_N] = i2d(n);
    save[SV_MEAN] = to_d(mean);
    for (int k = 2; k <= 6; ++k) save[SV_M2 + k - 2] = to_d(m[k]);
    save[SV_SGN] = to_d(res_st[7]);
    save[SV_ENERGY] = to_d(energy);
    save[SV_SUMI] = to_d(sumI);
    save[SV_CX] = cd[0];
    save[SV_CY] = cd[1];
    save[SV_CZ] = cd[2];
    save[SV_BX] = i2d(x0) + cd[3];
    save[SV_BY] = i2d(y0) + cd[4];
    save[SV_BZ] = i2d(z0) + cd[5];
    save[SV_X0] = i2d(x0);
    save[SV_Y0] = i2d(y0);
    save[SV_Z0] = i2d(z0);
  }
}

// int64 / int128 -> float without the FP64 pipe: convert the magnitude (the
// sum of non-negative halves has no cancellation), then apply the sign
__device__ inline float u64f(unsigned long long u) {
  return fmaf((float)(unsigned)(u >> 32), 4294967296.f, (float)(unsigned)(u & 0xFFFFFFFFull));
}
__device__ inline float ll2f(long long x) {
  const float m = u64f(x < 0 ? 0ull - (unsigned long long)x : (unsigned long long)x);
  return x < 0 ? -m : m;
}
__device__ inline float i128f(__int128 x) {
  const unsigned __int128 u = x < 0 ? (unsigned __int128)0 - (unsigned __int128)x : (unsigned __int128)x;
  const float m = fmaf(u64f((unsigned long long)(u >> 64)), 18446744073709551616.f, u64f((unsigned long long)u));
  return x < 0 ? -m : m;
}
template <class A>
__device__ inline A i128A(__int128 x) {
  if constexpr (std::is_same<A, float>::value) {
    return i128f(x);
  } else {  // magnitude first (its two halves are non-negative), then the sign
    const unsigned __int128 u = x < 0 ? (unsigned __int128)0 - (unsigned __int128)x : (unsigned __int128)x;
    const double m = (double)(unsigned long long)(u >> 64) * 18446744073709551616.0 + (double)(unsigned long long)u;
    return x < 0 ? -m : m;
  }
}

// GLCM sums of one offset, reduced over the block; all are integers, so they
// do not depend on the order of the hash table or of the reduction.  With C
// the count of a cell (a, b) of the symmetric matrix, k = a + b + 2 (= i + j,
// 1-based levels) and d = |a - b|:
//   [0] T = sum C            [1..4] sum C k^m      [5..6] sum C d^m
//   [7] sum C i^2            [8] sum C^2           [9] sum C log2 C  (2^-24)
//   [10] sum C log2(C T / (P_i P_j))  (2^-32)      [11] max C
// and over the marginals (c = count of one entry, e = c log2 c):
//   [12] sum e over p_x      [13] over p_{x+y}     [14] over p_{x-y}  (2^-24)
//   [15..19] sum_k c_k w(k) over p_{x-y} for w = 1/(1+k), 1/(1+k^2),
//            1/(1+k/Ng), 1/(1+k^2/Ng^2), 1/k^2 (k >= 1)  (2^-32)
// In the per (ROI, offset) accumulator handed to k_glcm_final, [9] and
// [12..14] are replaced by T log2 T minus the sum (gacc_value).
// Each fixed-point term is one rounding of a value computed in A, except
// c log2 c of counts below CLOG_N, which the plan tabulates from FP64.
constexpr int GI = GI_HOST, GF = GF_HOST, GN = GI + GF;

template <class A>
__device__ inline long long a2ll(A x) {
  if constexpr (std::is_same<A, float>::value) return __float2ll_rn(x);
  else return __double2ll_rn(x);
}
// c log2 c in units of 2^-24
template <class A>
__device__ inline long long ent_fx(unsigned c) {
  const A ca = (A)c;
  return a2ll(ca * alog2(ca) * (A)16777216);
}
// c log2 c (2^-24 units): counts below CLOG_N from the plan's exact table
// (the hot small counts stay in L1), larger ones computed
template <class A>
__device__ inline long long clog_fx(const long long* clog, unsigned c) {
  return c < (unsigned)CLOG_N ? __ldg(clog + c) : ent_fx<A>(c);
}

// T log2 T (2^-24 units) of an offset's total mass T: from the table, or in
// FP64 for the totals of the multi-block class beyond it
__device__ inline long long tlog_fx(const long long* clog, long long T) {
  if (T < CLOG_N) return __ldg(clog + T);
  const double t = (double)T;
  return __double2ll_rn(t * log2(t) * 16777216.0);
}

// The value handed to k_glcm_final for GLCM sum t: the entropy sums (joint,
// p_x, p_{x+y}, p_{x-y}) become the exact integer numerators
// T log2 T - sum c log2 c of T times the entropy, so that the feature kernel
// divides without cancellation (each distribution sums to T).
__device__ inline long long gacc_value(int t, long long v, long long TL) {
  return (t == 9 || t == 12 || t == 13 || t == 14) ? TL - v : v;
}

// the inverse-difference family of one difference-marginal entry (c at k),
// with the weights from the plan's table (rounded once on the host)
template <class A>
__device__ inline void invdiff_fx(const KParams& p, unsigned c, int k, long long* s) {
  const A* w;
  if constexpr (std::is_same<A, float>::value) w = p.wtab_f + 5 * k;
  else w = p.wtab_d + 5 * k;
  const A ca = (A)c * (A)4294967296.0;
#pragma unroll
  for (int i = 0; i < 5; ++i) s[15 + i] += a2ll(ca * __ldg(w + i));
}

// C log2(C T / (P_i P_j)) in units of 2^-32, from the exact integer excess
// C T - P_i P_j through log1p, so that cells of a nearly independent matrix
// (ratio close to 1, mutual information ~1e-7) keep their precision
template <class A>
__device__ inline long long mi_fx(unsigned Cc, long long T, unsigned pa, unsigned pb) {
  const long long pp = (long long)pa * (long long)pb;
  const long long ex = (long long)Cc * T - pp;
  if constexpr (std::is_same<A, float>::value)
    return a2ll<float>((float)Cc * log1pf((float)ex / (float)pp) * 6196328018.7194805f);  // 2^32 / ln 2
  else
    return a2ll<double>((double)Cc * log1p((double)ex / (double)pp) * 6196328018.7194805);
}

// GLCM features of one offset (Table S3 rows 140-174): every moment-type
// feature from exact integer power sums (central moments of the sum /
// difference / row distributions as exact integer numerators over powers of
// T), the entropies from the marginal sums.  Every feature is a quotient of
// exact integer (or fixed-point) numerators, so none cancels in A: the
// entropies come as T log2 T - sum c log2 c, CORR as its exact covariance
// and variance numerators.  Writes f[0..NGLCM) (the caller's shared-memory
// row) and f[NGLCM] = 1 (the offset has pairs).
template <class A>
__device__ __noinline__ void finalize_glcm(const KParams& p, double* row, const long long* iv, int di, int dir,
                                           A* f) {
  typedef __int128 I;
  const long long T = iv[0], S1 = iv[1], S2 = iv[2], S3 = iv[3], S4 = iv[4], D1 = iv[5], D2 = iv[6], Q2 = iv[7];
  const A Ta = i128A<A>(T), invT = (A)1 / Ta;
  // row distribution: mu = sum i p = S1 / (2T), var = (T Q2 - (S1/2)^2) / T^2
  const I R1 = (I)S1;  // 2 * sum i P
  const I var_n = 4 * (I)T * Q2 - R1 * R1;  // 4 T^2 var
  // sum distribution (k = i + j): mean S1/T, central moments via exact numerators
  const I c2n = (I)T * S2 - (I)S1 * S1;                                          // T^2 m2
  const I c3n = (I)T * T * S3 - 3 * (I)T * S1 * S2 + 2 * (I)S1 * S1 * S1;       // T^3 m3
  const I c4n = (I)T * T * T * S4 - 4 * (I)T * T * S1 * S3 + 6 * (I)T * S1 * S1 * S2 -
                3 * (I)S1 * S1 * S1 * S1;                                          // T^4 m4
  const I dvn = (I)T * D2 - (I)D1 * D1;                                          // T^2 var of |i-j|
  // covariance: sum (i-mu)(j-mu) p = ((S2 - D2) T - S1^2) / (4 T^2)
  const I cov_n = ((I)S2 - D2) * T - (I)S1 * S1;                                 // 4 T^2 cov
  const A T2 = Ta * Ta;
  const A mu = i128A<A>(R1) * invT / 2;
  const A var = i128A<A>(var_n) / (4 * T2);
  const A sumave = i128A<A>(S1) * invT;
  const A sumvar = i128A<A>(c2n) / T2;
  const A clushade = i128A<A>(c3n) / (T2 * Ta);
  const A cluprom = i128A<A>(c4n) / (T2 * T2);
  const A contrast = i128A<A>(D2) * invT;
  const A difave = i128A<A>(D1) * invT;
  const A difvar = i128A<A>(dvn) / T2;
  const A asmv = i128A<A>(iv[8]) / T2;
  // entropies from their exact numerators T log2 T - sum c log2 c (2^-24
  // units), mutual information (2^-32 units) and correlation from exact
  // integer numerators: no cancellation in A
  const A E = (A)(1.0 / 16777216.0), Qf = (A)(1.0 / 4294967296.0);
  const A je = i128A<A>(iv[9]) * E * invT;
  const A hx = i128A<A>(iv[12]) * E * invT;
  const A sument = i128A<A>(iv[13]) * E * invT;
  const A difent = i128A<A>(iv[14]) * E * invT;
  const A mi = i128A<A>(iv[10]) * Qf * invT;
  const A corr = var_n > 0 ? i128A<A>(cov_n) / i128A<A>(var_n) : (A)1;
  A fv[5];
  for (int k = 0; k < 5; ++k) fv[k] = i128A<A>(iv[15 + k]) * (A)(1.0 / 4294967296.0) * invT;  // ID, IDM, IDN, IDMN, IV
  f[G_ASM] = asmv;
  f[G_ACOR] = i128A<A>((I)S2 - D2) * invT / 4;
  f[G_CLUPROM] = cluprom;
  f[G_CLUSHADE] = clushade;
  f[G_CLUTEND] = sumvar;
  f[G_CONTRAST] = contrast;
  f[G_CORR] = corr;
  f[G_DIFAVE] = difave;
  f[G_DIFENTRO] = difent;
  f[G_DIFVAR] = difvar;
  f[G_DIS] = difave;
  f[G_ENERGY] = asqrt(asmv);
  f[G_ENTROPY] = je;
  f[G_HOM1] = fv[0];
  f[G_HOM2] = fv[1];
  f[G_IDM] = fv[1];
  // HXY1 = HXY2 = HX + HY and HX = HY for a symmetric matrix, so
  // HXY - HXY1 = -MI and HXY2 - HXY = MI (mutual information)
  f[G_INFOMEAS1] = hx > 0 ? -mi / hx : (A)0;
  {
    const A arg = -aexpm1((A)-2 * mi);  // 1 - exp(-2 MI) without cancellation for small MI
    f[G_INFOMEAS2] = asqrt(arg > 0 ? arg : (A)0);
  }
  f[G_IDMN] = fv[3];
  f[G_ID] = fv[0];
  f[G_IDN] = fv[2];
  f[G_IV] = fv[4];
  f[G_JAVE] = mu;
  f[G_JE] = je;
  f[G_JMAX] = i128A<A>(iv[11]) * invT;
  f[G_SUMAVE] = sumave;
  f[G_SUMENT] = sument;
  f[G_JVAR] = var;
  f[G_SUMVAR] = sumvar;
  f[G_VARIANCE] = var;
  if (p.per_offset)
    for (int g = 0; g < NGLCM; ++g) putA(p, row, Q_GLCM_O + (di * MAX_DIRS + dir) * NGLCM + g, f[g]);
  f[NGLCM] = 1;
}

// Block reduction of the GN GLCM sums (index 11 is a maximum); results in
// out (shared memory) for every thread.  Within a warp the sums use recursive
// halving (reduce-scatter): at lane bit o each lane keeps half of its values
// and swaps the other half with lane ^ o, so 32 slots cost 16 + 8 + 4 + 2 + 1
// exchanges instead of 5 per value; lane l ends with the warp total of slot
// l.  The maximum takes a plain butterfly.
template <class C, bool TRAILING_SYNC = true>
__device__ inline void block_sum_glcm(long long (&iv)[GN], double* scratch_d, long long* out) {
  long long* si = (long long*)scratch_d;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long mx = iv[11];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long y = __shfl_xor_sync(0xFFFFFFFFu, mx, o);
    mx = y > mx ? y : mx;
  }
  long long v[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = i < GN && i != 11 ? iv[i] : 0ll;
#pragma unroll
  for (int h = 16, o = 16; h > 0; h >>= 1, o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const long long send = up ? v[i] : v[i + h];
      const long long keep = up ? v[i + h] : v[i];
      v[i] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, o);
    }
  }
  // lane l holds slot l: at bit o the lane kept the half selected by its bit o
  if (lane < GN && lane != 11) si[warp * GN + lane] = v[0];
  if (lane == 0) si[warp * GN + 11] = mx;
  __syncthreads();
  const int t = threadIdx.x;
  if (t < GN) {
    long long r = si[t];
    for (int w = 1; w < C::NW; ++w) r = t == 11 ? (si[w * GN + t] > r ? si[w * GN + t] : r) : r + si[w * GN + t];
    out[t] = r;
  }
  if (TRAILING_SYNC) __syncthreads();
}

// ----------------------------------------------------------------------------
// NGTDM (Table S3 rows 246-250).  For a pixel of grey level L (1-based bin)
// whose Chebyshev-1 neighbourhood holds cnt > 0 ROI pixels with level sum
// `sum`, the term |L - sum / cnt| in units of 2^-32: the FP32 quotient of the
// two integers is correctly rounded and the power-of-two scaling exact, so
// the per-level sums do not depend on the order of the atomics.
__device__ inline unsigned long long ngtdm_term(int L, int sum, int cnt) {
  const int num = L * cnt - sum;
  const float q = (float)(num < 0 ? -num : num) / (float)cnt;
  return __float2ull_rn(q * 4294967296.f);
}

// The five NGTDM features from the per-level counts nL[0..ng) and sums
// S[0..ng) (2^-32 units) in shared memory; every thread of the block calls
// it, thread 0 writes the columns.  lst: shared scratch of ng words.  With
// p = n / N (N valid pixels), G levels present, mu = sum p L, m = mean of
// the present levels: coarseness 1 / sum p s; contrast
// 2 sum p (L - mu)^2 / (G (G - 1)) * sum s / N; busyness sum p s /
// sum_i sum_j |L_i p_i - L_j p_j|; complexity (1/N) sum_i sum_j |L_i - L_j|
// (p_i s_i + p_j s_j) / (p_i + p_j); strength 2 (G sum p (L - m)^2 +
// sum (L - m)^2) / sum s (the double sums over the present levels, written
// about the means so that they do not cancel).
template <class C, class A>
__device__ void ngtdm_features(const KParams& p, double* row, int ng, unsigned* nL, unsigned long long* S,
                               unsigned* lst, double* red, A* sc, long long* s64) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const A nan = anan<A>();
  const A fx = (A)(1.0 / 4294967296.0);
  if (warp == 0) {  // levels present, ascending
    int cnt = 0;
    for (int b = 0; b < ng; b += 32) {
      const bool v = b + lane < ng && nL[b + lane] > 0;
      const unsigned bal = __ballot_sync(0xFFFFFFFFu, v);
      if (v) lst[cnt + __popc(bal & lanemask_lt())] = (unsigned)(b + lane);
      cnt += __popc(bal);
    }
    if (lane == 0) s64[0] = cnt;
  }
  {
    long long t[1] = {0};
    for (int i = tid; i < ng; i += C::NT) t[0] += nL[i];
    block_sum_i64<C, 1>(t, red, s64 + 1);  // ends with a barrier: lst and s64[0] are visible
  }
  const int G = (int)s64[0];
  const long long Nv = s64[1];
  if (Nv == 0) {
    if (tid == 0)
      for (int q = 0; q < N_NGTDM; ++q) putA(p, row, Q_NGTDM + q, nan);
    return;
  }
  const A invN = (A)1 / (A)Nv;
  // FP32: p, p s and L p of the present levels, compacted in level order into
  // the storage of S (float2 per level) and nL, read by the pair sums below
  constexpr bool F32 = std::is_same<A, float>::value;
  float2* PA = (float2*)S;
  float* V = (float*)nL;
  if constexpr (F32) {
    constexpr int MAXK = 256 / C::NT + 1;
    float2 pa[MAXK];
    float vv[MAXK];
#pragma unroll
    for (int q = 0; q < MAXK; ++q) {
      const int k = tid + q * C::NT;
      if (k < G) {
        const int i = (int)lst[k];
        const float pi = (float)nL[i] * invN;
        pa[q] = make_float2(pi, pi * (ll2f((long long)S[i]) * fx));
        vv[q] = (float)(i + 1) * pi;
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < MAXK; ++q) {
      const int k = tid + q * C::NT;
      if (k < G) {
        PA[k] = pa[q];
        V[k] = vv[q];
      }
    }
    __syncthreads();
  }
  auto level = [&](int k, A& pi, A& ai, A& L) {  // p, p s, L of the k-th present level
    if constexpr (F32) {
      const float2 x = PA[k];
      pi = x.x;
      ai = x.y;
      L = (A)(lst[k] + 1);
    } else {
      const int i = (int)lst[k];
      pi = (A)nL[i] * invN;
      ai = pi * ((A)ll2f((long long)S[i]) * fx);
      L = (A)(i + 1);
    }
  };
  {  // ps = sum p s, ssum = sum s, mu = sum p L, T1 = sum L
    A v[4] = {0, 0, 0, 0};
    for (int k = tid; k < G; k += C::NT) {
      A pi, ai, L;
      level(k, pi, ai, L);
      v[0] += ai;
      v[1] += ai / pi;
      v[2] += pi * L;
      v[3] += L;
    }
    block_sum<C, A, 4>(v, red, sc);
  }
  const A ps = sc[0], ssum = sc[1], mu = sc[2], m = sc[3] / (A)G;
  {  // centred sums, then the pair sums over i < j (rows paired for balance)
    A v[5] = {0, 0, 0, 0, 0};
    for (int k = tid; k < G; k += C::NT) {
      A pi, ai, L;
      level(k, pi, ai, L);
      v[0] += pi * (L - mu) * (L - mu);
      v[1] += pi * (L - m) * (L - m);
      v[2] += (L - m) * (L - m);
    }
    for (int a = tid; a < (G + 1) / 2; a += C::NT) {
#pragma unroll 1
      for (int h = 0; h < 2; ++h) {
        const int r = h ? G - 1 - a : a;
        if (h && r == a) break;
        A pi, ai, Li;
        level(r, pi, ai, Li);
        const A vi = Li * pi;
        A b0 = 0, b1 = 0;
        for (int c = r + 1; c < G; ++c) {
          A pj, aj, Lj;
          if constexpr (F32) {
            const float2 x = PA[c];
            pj = x.x;
            aj = x.y;
            Lj = (A)(lst[c] + 1);
            const float dv = vi - V[c];
            b0 += fabsf(dv);
            b1 += __fdividef((Lj - Li) * (ai + aj), pi + pj);  // Lj > Li
          } else {
            level(c, pj, aj, Lj);
            const A dv = vi - Lj * pj;
            b0 += dv < 0 ? -dv : dv;
            b1 += (Lj - Li) * (ai + aj) / (pi + pj);
          }
        }
        v[3] += b0;
        v[4] += b1;
      }
    }
    block_sum<C, A, 5>(v, red, sc + 4);
  }
  if (tid == 0) {
    const A V1 = sc[4], V2 = sc[5], V3 = sc[6], bden = 2 * sc[7], cplx = 2 * sc[8];
    putA(p, row, Q_NGTDM + NT_COARSENESS, ps > 0 ? (A)1 / ps : nan);
    putA(p, row, Q_NGTDM + NT_CONTRAST, G > 1 ? (A)2 * V1 / ((A)G * (A)(G - 1)) * ssum * invN : (A)0);
    putA(p, row, Q_NGTDM + NT_BUSYNESS, bden > 0 ? ps / bden : (A)0);
    putA(p, row, Q_NGTDM + NT_COMPLEXITY, cplx * invN);
    putA(p, row, Q_NGTDM + NT_STRENGTH, ssum > 0 ? (A)2 * ((A)G * V2 + V3) / ssum : (A)0);
  }
  __syncthreads();
}

// 2^32 / j^2 rounded to nearest (j <= 27), exact in integers
__device__ inline unsigned long long inv_sq_fx(unsigned j) {
  const unsigned long long d = (unsigned long long)j * j;
  return ((1ull << 32) + d / 2) / d;
}

// GLDM (Table S3 rows 251-264) from per-level sums over the levels a < ng
// (grey level i = a + 1): lv(a, r, c2, cm) gives the level's pixel count r,
// sum_j P(i, j) j^2 (c2) and sum_j P(i, j) round(2^32 / j^2) (cm, 2^-32
// units); col[0..nj) counts the pixels of each dependence j = 1..nj; ent is
// this thread's share of sum over the cells of P log2 P (2^-24 units).  With
// N the ROI's pixel count: SDE sum P / j^2 / N, LDE sum P j^2 / N, GLN
// sum_i r_i^2 / N, DN sum_j col_j^2 / N, DNN DN / N, GLV and DV the
// variances of i and j under P / N, DE log2 N - sum P log2 P / N, and the
// grey-level emphases sum P i^{+-2} (j^{+-2}) / N.  Every thread of the block
// calls it; thread 0 writes the columns.
template <class C, class A, class LV>
__device__ void gldm_features(const KParams& p, double* row, int ng, int nj, LV lv, const unsigned* col, long long ent,
                              double* red, A* sc, long long* s64) {
  const int tid = threadIdx.x;
  {
    long long t[2] = {0, ent};
    for (int a = tid; a < ng; a += C::NT) {
      unsigned long long r, c2, cm;
      lv(a, r, c2, cm);
      t[0] += (long long)r;
    }
    block_sum_i64<C, 2>(t, red, s64);  // ends with a barrier
  }
  const long long N = s64[0], E = s64[1];
  if (N == 0) {
    if (tid == 0)
      for (int q = 0; q < N_GLDM; ++q) putA(p, row, Q_GLDM + q, anan<A>());
    __syncthreads();
    return;
  }
  const A invN = (A)1 / (A)N, Q = (A)(1.0 / 4294967296.0);
  {
    A v[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int a = tid; a < ng; a += C::NT) {
      unsigned long long r, c2, cm;
      lv(a, r, c2, cm);
      if (!r) continue;
      const A i = (A)(a + 1), i2 = i * i, ii2 = (A)1 / i2;
      const A ra = (A)r, c2a = (A)c2, cma = (A)cm * Q;
      v[0] += cma;
      v[1] += c2a;
      v[2] += ra * ra;
      v[3] += ra * i;
      v[4] += ra * i2;
      v[5] += ra * ii2;
      v[6] += cma * ii2;
      v[7] += cma * i2;
      v[8] += c2a * ii2;
      v[9] += c2a * i2;
    }
    block_sum<C, A, 10>(v, red, sc);
  }
  const A mui = sc[3] * invN;
  {
    A v[1] = {0};
    for (int a = tid; a < ng; a += C::NT) {
      unsigned long long r, c2, cm;
      lv(a, r, c2, cm);
      const A d = (A)(a + 1) - mui;
      v[0] += (A)r * d * d;
    }
    block_sum<C, A, 1>(v, red, sc + 10);
  }
  if (tid == 0) {
    A dn = 0, sj = 0;
    for (int j = 0; j < nj; ++j) {
      const A c = (A)col[j];
      dn += c * c;
      sj += c * (A)(j + 1);
    }
    const A muj = sj * invN;
    A dv = 0;
    for (int j = 0; j < nj; ++j) {
      const A d = (A)(j + 1) - muj;
      dv += (A)col[j] * d * d;
    }
    putA(p, row, Q_GLDM + GD_SDE, sc[0] * invN);
    putA(p, row, Q_GLDM + GD_LDE, sc[1] * invN);
    putA(p, row, Q_GLDM + GD_GLN, sc[2] * invN);
    putA(p, row, Q_GLDM + GD_DN, dn * invN);
    putA(p, row, Q_GLDM + GD_DNN, dn * invN * invN);
    putA(p, row, Q_GLDM + GD_GLV, sc[10] * invN);
    putA(p, row, Q_GLDM + GD_DV, dv * invN);
    // one thread per ROI: the difference of two terms near log2 N in FP64
    put(p, row, Q_GLDM + GD_DE, log2((double)N) - (double)E * (1.0 / 16777216.0) / (double)N);
    putA(p, row, Q_GLDM + GD_LGLE, sc[5] * invN);
    putA(p, row, Q_GLDM + GD_HGLE, sc[4] * invN);
    putA(p, row, Q_GLDM + GD_SDLGLE, sc[6] * invN);
    putA(p, row, Q_GLDM + GD_SDHGLE, sc[7] * invN);
    putA(p, row, Q_GLDM + GD_LDLGLE, sc[8] * invN);
    putA(p, row, Q_GLDM + GD_LDHGLE, sc[9] * invN);
  }
  __syncthreads();
}

// Per (ROI, offset) GLCM accumulator handed from the accumulation kernels to
// k_glcm_final: the GN integer sums.  An all-zero record (T = 0) marks an
// offset without pairs.
constexpr int GACC_BYTES = 8 * GN;
__device__ inline void store_gacc(const KParams& p, int64_t item, int oi, const long long* iv, bool empty) {
  long long* g = (long long*)(p.gacc + ((size_t)item * (p.n_dist * p.n_dirs) + oi) * GACC_BYTES);
  const int t = threadIdx.x;
  if (t < GN) g[t] = empty ? 0ll : iv[t];
}

// Per-ROI statistics and moment sums handed from the accumulation kernels to
// k_stats_final, in slots of type A: [0..7] centred power sums, [8..27]
// intensity moments, [28..47] binary moments, [48] mean, [49] sum I, [50]
// energy, [51..53] the centre of the intensity moment sums, [54..56] that of
// the binary ones (ROI-local); then, as FP64 at byte SACC_CD, the intensity
// and binary centroids (ROI-local).
constexpr int SACC_SLOTS = 64, SACC_BYTES = 8 * SACC_SLOTS, SACC_CD = 464;
template <class A>
__device__ inline void store_sacc(const KParams& p, int64_t item, int nm, const A* st, const A* mi, const A* mb,
                                  A mean, A sumI, A energy, A cx, A cy, A cz, A bx, A by, A bz, const double* cd) {
  A* g = (A*)(p.sacc + (size_t)item * SACC_BYTES);
  double* gd = (double*)(p.sacc + (size_t)item * SACC_BYTES + SACC_CD);
  for (int i = threadIdx.x; i < 6; i += blockDim.x) gd[i] = cd[i];
  for (int i = threadIdx.x; i < 57; i += blockDim.x) {
    A v;
    if (i < 8) v = st[i];
    else if (i < 28) v = i - 8 < nm ? mi[i - 8] : (A)0;
    else if (i < 48) v = i - 28 < nm ? mb[i - 28] : (A)0;
    else {
      const A sc[9] = {mean, sumI, energy, cx, cy, cz, bx, by, bz};
      v = sc[i - 48];
    }
    g[i] = v;
  }
}

// Percentiles by linear interpolation at h = (n-1) q on the sorted values,
// computed in FP64 with separately rounded operations like the definition,
// one lane per percentile.  Lane 0 also turns [P10, P90] into an inclusive
// range of encoded values (bnd[0], bnd[1]): a value lies in [P10, P90] exactly
// when its code lies in that range.  Writes median, P10, P90 to sc[] (FP64).
template <class T>
__device__ __noinline__ void finalize_percentiles(const KParams& p, double* row, const unsigned* v, int n, double* sc,
                                                  unsigned* bnd) {
  const int lane = threadIdx.x & 31;
  const double qs[7] = {0.01, 0.10, 0.25, 0.50, 0.75, 0.90, 0.99};
  const int qcol[7] = {S_P01, S_P10, S_P25, S_MEDIAN, S_P75, S_P90, S_P99};
  double pv_ = 0;
  if (lane < 7) {
    const double h = __dmul_rn((double)(n - 1), qs[lane]);
    const int lo = (int)floor(h);
    if (lo >= n - 1) {
      pv_ = Enc<T>::dec(v[n - 1]);
    } else {
      const double a = Enc<T>::dec(v[lo]), b = Enc<T>::dec(v[lo + 1]);
      pv_ = __dadd_rn(a, __dmul_rn(__dsub_rn(h, (double)lo), __dsub_rn(b, a)));
    }
    put(p, row, Q_STATS + qcol[lane], pv_);
  }
  const double p25 = __shfl_sync(0xFFFFFFFFu, pv_, 2), p75 = __shfl_sync(0xFFFFFFFFu, pv_, 4);
  const double p10 = __shfl_sync(0xFFFFFFFFu, pv_, 1), p90 = __shfl_sync(0xFFFFFFFFu, pv_, 5);
  const double med = __shfl_sync(0xFFFFFFFFu, pv_, 3);
  if (lane != 0) return;
  put(p, row, Q_STATS + S_IQR, __dsub_rn(p75, p25));
  {
    const float a = (float)p75, b = (float)p25;
    put(p, row, Q_STATS + S_QCOD, (a + b) != 0.f ? f2d((a - b) / (a + b)) : f2d(__int_as_float(0x7FC00000)));
  }
  sc[0] = med;
  sc[1] = p10;
  sc[2] = p90;
  if constexpr (Enc<T>::INTEGER) {
    // integer values: v >= P10 <=> v >= ceil(P10); v <= P90 <=> v <= floor(P90)
    const long long bias = std::is_same<T, int16_t>::value ? 32768 : 0;
    bnd[0] = (unsigned)((long long)ceil(p10) + bias);
    bnd[1] = (unsigned)((long long)floor(p90) + bias);
  } else {
    // float values: v >= P10 <=> v >= the smallest float not below P10, and
    // v <= P90 <=> v <= the largest float not above P90; a zero bound admits
    // both signed zeros, which compare equal to it
    float lo = (float)p10, hi = (float)p90;
    if ((double)lo < p10) lo = nextafterf(lo, INFINITY);
    if ((double)hi > p90) hi = nextafterf(hi, -INFINITY);
    if (lo == 0.f) lo = -0.f;
    if (hi == 0.f) hi = 0.f;
    bnd[0] = Enc<T>::enc(lo);
    bnd[1] = Enc<T>::enc(hi);
  }
}

// Rule a4 for float images: b = floor(n (x - min) / (max - min)) in FP64 with
// separately rounded operations.  An FP32 evaluation decides whenever it is
// farther than 1e-4 (relative) from a bin edge, which covers the FP32
// rounding with a wide margin; otherwise the FP64 expression is evaluated.
__device__ inline unsigned bin_float(float x, float mn, float mx, int nb) {
  const float q = (float)nb * (x - mn) / (mx - mn);
  const float fl = floorf(q);
  const float tol = 1e-4f * (1.f + q);
  unsigned b;
  if (q - fl > tol && fl + 1.f - q > tol) {
    b = (unsigned)fl;
  } else {
    const double dq = __ddiv_rn(__dmul_rn((double)nb, __dsub_rn((double)x, (double)mn)), __dsub_rn((double)mx, (double)mn));
    b = (unsigned)floor(dq);
  }
  return min(b, (unsigned)(nb - 1));
}

// Order statistics of Table S1 from the sorted encoded values v[0..n) (in
// shared or global memory): percentiles, mode (longest run, ties to the
// smallest value), robust mean and mean absolute deviation over [P10, P90],
// and the mean absolute deviation from the median.  Called by every thread of
// the block; uses s_sc[4..7] and s_sc[10..11].
template <class T, class C, class A>
__device__ inline void order_tail(const KParams& p, double* row, const unsigned* v, int n, double* red,
                                  double* s_sd, unsigned* s_bnd, A* s_sc) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const A nan = anan<A>();
  const int ibias = std::is_same<T, int16_t>::value ? 32768 : 0;
  if (warp == 0) finalize_percentiles<T>(p, row, v, n, s_sd, s_bnd);
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
    int* sc = (int*)red;
    sc[tid] = last_start;
    __syncthreads();
    if (warp == 0) {  // exclusive max-scan over the C::NT entries
      int carry = -1;
      for (int base = 0; base < C::NT; base += 32) {
        const int x = sc[base + lane];
        int incl = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
          if (lane >= o) incl = max(incl, y);
        }
        const int prev = __shfl_up_sync(0xFFFFFFFFu, incl, 1);  // every lane executes the shuffle
        const int excl = lane == 0 ? carry : max(carry, prev);
        sc[base + lane] = excl;
        carry = max(carry, __shfl_sync(0xFFFFFFFFu, incl, 31));
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
  // robust mean over [P10, P90], mean absolute deviation from the median
  const unsigned b10 = s_bnd[0], b90 = s_bnd[1];
  if (tid == 0) s_sc[10] = (A)s_sd[0];  // median in the accumulation type
  __syncthreads();
  const A medA = s_sc[10];
  A rv[3] = {0, 0, 0};  // sum over [P10, P90], sum |x - median|, count in [P10, P90] (exact)
  for (int i = tid; i < n; i += C::NT) {
    const unsigned e = v[i];
    const A x = decA<T, A>(e);
    if (e >= b10 && e <= b90) {
      rv[0] += x;
      rv[2] += (A)1;
    }
    rv[1] += x > medA ? x - medA : medA - x;
  }
  block_sum<C, A, 3>(rv, red, s_sc + 4);
  const int cntV = (int)s_sc[6];
  if (tid == 0) s_sc[11] = cntV > 0 ? s_sc[4] / (A)cntV : nan;
  __syncthreads();
  const A rmA = s_sc[11];
  A ra[1] = {0};
  for (int i = tid; i < n; i += C::NT) {
    const unsigned e = v[i];
    if (e >= b10 && e <= b90) {
      const A x = decA<T, A>(e);
      ra[0] += x > rmA ? x - rmA : rmA - x;
    }
  }
  block_sum<C, A, 1>(ra, red, s_sc + 7);
  if (tid == 0) {
    const unsigned mode_e = ~(unsigned)(best & 0xFFFFFFFFu);
    if (Enc<T>::INTEGER) put(p, row, Q_STATS + S_MODE, i2d((long long)mode_e - ibias));
    else put(p, row, Q_STATS + S_MODE, f2d(Enc<T>::decf(mode_e)));
    putA(p, row, Q_STATS + S_MODE_PROB, (A)(int)(best >> 32) / (A)n);
    putA(p, row, Q_STATS + S_RMEAN, rmA);
    putA(p, row, Q_STATS + S_RMAD, cntV > 0 ? s_sc[7] / (A)cntV : nan);
    putA(p, row, Q_STATS + S_MEDAD, s_sc[5] / (A)n);
  }
}

// ----------------------------------------------------------------------------
// the kernel

template <class T, int NDIM, class C, class A>
__global__ void __launch_bounds__(C::NT, C::MINB) k_roi(KParams p, int cls) {
  static_assert(C::CELLS <= 65536, "GLCM pixel words hold a 16-bit raster index");
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
  A* res = (A*)(smem + L.res);
  __shared__ RoiInfo s_r;
  __shared__ int s_item;
  __shared__ unsigned s_rowcnt[C::NW], s_rowbase[C::NW + 1];
  __shared__ FastDiv s_fd;
  __shared__ A s_sc[16];
  __shared__ A s_sl[8];     // low parts of the pass-1 float sums
  __shared__ double s_sd[4];
  __shared__ double s_cd[8];  // FP64 intensity and binary centroids (ROI-local)
  __shared__ long long s_i64[GN + 4];  // pass-1 sums, then the GLCM sums of an offset
  __shared__ unsigned s_bnd[4];
  __shared__ A s_pa[12];  // per-ROI scalars: mean (hi, lo), centroids, sums, edge mean
  __shared__ unsigned s_ncell, s_npair;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned* qlen = p.qlen + cls;
  const int* queue = p.queue + (int64_t)cls * p.max_rois;
  const int64_t per = p.nx * p.ny * p.nz;
  const bool need_glcm = (p.need & NEED_GLCM) != 0;
  const bool need_ngtdm = (p.need & NEED_NGTDM) != 0;
  const bool need_gldm = (p.need & NEED_GLDM) != 0;
  const bool need_levels = need_glcm || need_ngtdm || need_gldm;  // grey levels (GLCM bins) of the pixels
  const bool need_raster = need_levels || (p.need & NEED_EDGE) != 0;  // padded raster of the ROI's cells
  const int pad = need_raster ? p.pad : 0;
  const A nan = anan<A>();

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
    const unsigned need = p.need;

    // ---- stage the ROI: raster of bins, pixel list, value histogram -------
    for (int i = tid; i < cells; i += C::NT) raster[i] = 0xFFFF;
    for (int i = tid; i < p.hist_bins; i += C::NT) hist[i] = 0;
    if (tid == 0) s_rowbase[C::NW] = 0;
    __syncthreads();
    const int nrows = H * D;
    const T* img = (const T*)p.img;
    const float fmn = Enc<T>::decf(vmin), fmx = Enc<T>::decf(vmax);
    // Work items are (row, 32-column chunk) pairs in raster order.  Each warp
    // takes U consecutive items per iteration and issues all their loads
    // before using them (the bounding box is L2-resident, so latency, not
    // bandwidth, bounds this loop); pixel positions follow raster order via a
    // prefix over warps, which keeps the pixel list deterministic.
    constexpr int U = C::NW == 1 ? 8 : (C::NW <= 4 ? 4 : 2);
    const int nchk = (W + 31) >> 5;
    const int nitems = nrows * nchk;
    unsigned run = 0;  // pixels placed so far (single-warp blocks)
    for (int ib = 0; ib < nitems; ib += C::NW * U) {
      const int i0 = ib + warp * U;
      int rr = i0 / nchk, xc = i0 - rr * nchk;
      int ry = rr % H, rz = rr / H;
      unsigned bal[U];
      int64_t roff[U];
      int xs[U];
      unsigned wcnt = 0;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const bool have = i0 + u < nitems;
        xs[u] = xc * 32 + lane;
        roff[u] = origin + ((int64_t)rz * p.ny + ry) * p.nx;
        const bool in = have && xs[u] < W && __ldg(p.mask + roff[u] + xs[u]) == label;
        bal[u] = __ballot_sync(0xFFFFFFFFu, in);
        wcnt += __popc(bal[u]);
        if (++xc == nchk) {
          xc = 0;
          if (++ry == H) {
            ry = 0;
            ++rz;
          }
        }
      }
      unsigned base;
      if (C::NW == 1) {
        base = run;
        run += wcnt;
      } else {
        if (lane == 0) s_rowcnt[warp] = wcnt;
        __syncthreads();
        if (tid == 0) {
          unsigned acc = s_rowbase[C::NW];
          for (int w = 0; w < C::NW; ++w) {
            s_rowbase[w] = acc;
            acc += s_rowcnt[w];
          }
          s_rowbase[C::NW] = acc;
        }
        __syncthreads();
        base = s_rowbase[warp];
      }
      rr = i0 / nchk;
      xc = i0 - rr * nchk;
      ry = rr % H;
      rz = rr / H;
      T val[U];
#pragma unroll
      for (int u = 0; u < U; ++u)
        if ((bal[u] >> lane) & 1u) val[u] = __ldg(img + roff[u] + xs[u]);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if ((bal[u] >> lane) & 1u) {
          const int x = xs[u];
          const unsigned pos = base + __popc(bal[u] & lanemask_lt());
          const unsigned e = Enc<T>::enc(val[u]);
          if (pos < (unsigned)C::PIX) {
            pc[pos] = NDIM == 3 ? ((unsigned)x | ((unsigned)ry << 11) | ((unsigned)rz << 22))
                                : ((unsigned)x | ((unsigned)ry << 16));
            pv[pos] = e;
          }
          // GLCM bin and histogram bin (IBSI fixed bin number)
          unsigned gb = 0, hb = 0;
          if (vmax > vmin) {
            if (Enc<T>::INTEGER) {
              const unsigned dv = e - vmin;
              gb = min(s_fd.div((unsigned)p.ng * dv), (unsigned)(p.ng - 1));
              hb = min(s_fd.div((unsigned)p.hist_bins * dv), (unsigned)(p.hist_bins - 1));
            } else {
              const float xv = Enc<T>::decf(e);
              if (need_levels) gb = bin_float(xv, fmn, fmx, p.ng);
              if (need & NEED_HIST) hb = bin_float(xv, fmn, fmx, p.hist_bins);
            }
          }
          if (need_raster) {
            const int ri = ((NDIM == 3 ? rz + pad : 0) * Hp + (ry + pad)) * Wp + (x + pad);
            if (ri < cells) raster[ri] = (uint16_t)gb;
            else atomicOr(p.err, E_INTERNAL);
          }
          if (need & NEED_HIST) atomicAdd(&hist[hb], 1u);
        }
        base += __popc(bal[u]);
        if (++xc == nchk) {
          xc = 0;
          if (++ry == H) {
            ry = 0;
            ++rz;
          }
        }
      }
    }
    if (C::NW == 1 && lane == 0) s_rowbase[C::NW] = run;
    __syncthreads();
    if (tid == 0 && s_rowbase[C::NW] != (unsigned)n) atomicOr(p.err, E_INTERNAL);

    // ---- geometry and range columns (exact integers) -------------------------
    if (tid == 0) {
      put(p, row, Q_LABEL, i2d(label));
      put(p, row, Q_IMAGE, i2d(bimg));
      put(p, row, Q_AREA, i2d(n));
      put(p, row, Q_BB_X, i2d(r.x0));
      put(p, row, Q_BB_Y, i2d(r.y0));
      put(p, row, Q_BB_Z, i2d(r.z0));
      put(p, row, Q_BB_W, i2d(W));
      put(p, row, Q_BB_H, i2d(H));
      put(p, row, Q_BB_D, i2d(D));
      if (Enc<T>::INTEGER) {
        const long long bias = std::is_same<T, int16_t>::value ? 32768 : 0;
        put(p, row, Q_STATS + S_MIN, i2d((long long)vmin - bias));
        put(p, row, Q_STATS + S_MAX, i2d((long long)vmax - bias));
        put(p, row, Q_STATS + S_RANGE, i2d((long long)vmax - (long long)vmin));
      } else {
        put(p, row, Q_STATS + S_MIN, f2d(fmn));
        put(p, row, Q_STATS + S_MAX, f2d(fmx));
        put(p, row, Q_STATS + S_RANGE, __dsub_rn(f2d(fmx), f2d(fmn)));  // as the FP64 definition
      }
    }

    // ---- pass 1: exact sums (integers) --------------------------------------
    // Edge intensity statistics (Table S1 rows 3-7, Table S5) ride along: an
    // edge pixel has a face neighbour (4 in 2D, 6 in 3D) outside the ROI, and
    // in the padded raster every cell that is not one of the ROI's pixels
    // (another label, background, beyond the image) holds the sentinel.
    const int ibias = std::is_same<T, int16_t>::value ? 32768 : 0;
    const bool do_edge = (need & NEED_EDGE) != 0;
    const int plane = Wp * Hp;
    unsigned emn = 0xFFFFFFFFu, emx = 0;  // edge codes (block-reduced below)
    {
      // [0] sum I, [1] sum x I, [2] sum y I, [3] sum z I, [4] sum x, [5] sum y, [6] sum z, [7] sum I^2,
      // [8] edge count, [9] edge sum d, [10] edge sum d^2 with d = code - vmin (exact for integer images)
      long long s[11] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
      KSum<A> fs[6];  // float images: sum I, x I, y I, z I, I^2, edge sum (I - min), compensated
      for (int i = tid; i < n; i += C::NT) {
        const unsigned c = pc[i];
        const int x = NDIM == 3 ? (int)(c & 2047u) : (int)(c & 0xFFFFu);
        const int y = NDIM == 3 ? (int)((c >> 11) & 2047u) : (int)(c >> 16);
        const int z = NDIM == 3 ? (int)(c >> 22) : 0;
        s[4] += x;
        s[5] += y;
        s[6] += z;
        const bool edge = do_edge && edge_pixel<NDIM>(raster, c, pad, Wp, Hp, plane);
        if (edge) {
          s[8] += 1;
          emn = min(emn, pv[i]);
          emx = max(emx, pv[i]);
        }
        if (Enc<T>::INTEGER) {
          const int v = (int)pv[i] - ibias;
          s[0] += v;
          s[1] += (long long)x * v;
          s[2] += (long long)y * v;
          s[3] += (long long)z * v;
          s[7] += (long long)v * v;
          if (edge) {
            const long long d = (long long)(pv[i] - vmin);
            s[9] += d;
            s[10] += d * d;
          }
        } else {
          const A v = decA<T, A>(pv[i]);
          fs[0].add(v);
          fs[1].add((A)x * v);
          fs[2].add((A)y * v);
          fs[3].add((A)z * v);
          fs[4].add(v * v);
          if (edge) fs[5].add(v - (A)fmn);
        }
      }
      block_sum_i64<C, 11>(s, red, s_i64);
      if constexpr (!Enc<T>::INTEGER) {
        if constexpr (std::is_same<A, float>::value) {
          block_sum_pair<C, 6>(fs, red, s_sc, s_sl);  // (hi, lo) pairs
        } else {
          A f6[6];
#pragma unroll
          for (int k = 0; k < 6; ++k) f6[k] = fs[k].s - fs[k].c;
          block_sum<C, A, 6>(f6, red, s_sc);
          if (tid < 6) s_sl[tid] = 0;
          __syncthreads();
        }
      }
      if (do_edge) block_minmax_u32<C>(emn, emx, red);
    }
    // per-ROI scalars by one thread, broadcast through shared memory: mean
    // (as hi + lo so that I - mean keeps its accuracy in FP32), the centre of
    // the intensity-weighted sums (the exact centroid, or the binary centroid
    // when the weights sum to zero) and the binary centroid
    if (tid == 0) {
      const A nA = (A)n;
      A sI, en, mhi, mlo;
      // FP64 sums for the centroids and the mean: exact integers (16-bit
      // images) or the compensated float pairs
      double dI, dxI, dyI, dzI;
      if (Enc<T>::INTEGER) {
        const long long si = s_i64[0];
        sI = (A)si;
        en = (A)s_i64[7];
        dI = (double)si;
        dxI = (double)s_i64[1];
        dyI = (double)s_i64[2];
        dzI = (double)s_i64[3];
        if constexpr (std::is_same<A, float>::value) {
          const long long q = si / n, rm = si - q * n;  // mean = q + rm / n exactly
          mhi = (A)q;
          mlo = (A)rm / nA;
        } else {
          mhi = (A)si / nA;
          mlo = 0;
        }
        put(p, row, Q_STATS + S_II, i2d(si));
        put(p, row, Q_STATS + S_ENERGY, i2d(s_i64[7]));
      } else {
        if constexpr (std::is_same<A, float>::value) {
          dI = pair_d(s_sc[0], s_sl[0]);
          dxI = pair_d(s_sc[1], s_sl[1]);
          dyI = pair_d(s_sc[2], s_sl[2]);
          dzI = pair_d(s_sc[3], s_sl[3]);
          const double md = dI / (double)n;  // mean as an unevaluated float pair
          mhi = (A)md;
          mlo = (A)(md - (double)mhi);
        } else {
          dI = s_sc[0];
          dxI = s_sc[1];
          dyI = s_sc[2];
          dzI = s_sc[3];
          mhi = s_sc[0] / nA;
          mlo = 0;
        }
        sI = (A)dI;
        en = s_sc[4] + s_sl[4];
        put(p, row, Q_STATS + S_II, dI);
        putA(p, row, Q_STATS + S_ENERGY, en);
      }
      // centroids in FP64 (ROI-local): binary from the exact coordinate sums,
      // intensity-weighted from the sums above (binary when sum I = 0)
      const double bxd = (double)s_i64[4] / n, byd = (double)s_i64[5] / n, bzd = (double)s_i64[6] / n;
      const bool wv = dI != 0;
      s_cd[0] = wv ? dxI / dI : bxd;
      s_cd[1] = wv ? dyI / dI : byd;
      s_cd[2] = wv ? dzI / dI : bzd;
      s_cd[3] = bxd;
      s_cd[4] = byd;
      s_cd[5] = bzd;
      s_pa[0] = mhi;
      s_pa[1] = mlo;
      // centre of the intensity-weighted moment sums: the weighted centroid
      // if it lies in the bounding box, else the binary one
      const bool inbox = wv && s_cd[0] >= 0 && s_cd[0] <= W - 1 && s_cd[1] >= 0 && s_cd[1] <= H - 1 &&
                         (NDIM != 3 || (s_cd[2] >= 0 && s_cd[2] <= D - 1));
      s_pa[2] = (A)(inbox ? s_cd[0] : bxd);
      s_pa[3] = (A)(inbox ? s_cd[1] : byd);
      s_pa[4] = (A)(inbox ? s_cd[2] : bzd);
      s_pa[5] = (A)bxd;
      s_pa[6] = (A)byd;
      s_pa[7] = (A)bzd;
      s_pa[8] = sI;
      s_pa[9] = en;
      if (do_edge) {  // edge statistics (the float deviation follows in pass 2)
        const long long ne = s_i64[8];  // >= 1: a finite ROI has an edge pixel
        A emean, estd = 0;
        if (Enc<T>::INTEGER) {
          const long long bias = std::is_same<T, int16_t>::value ? 32768 : 0;
          const long long s1 = s_i64[9], sumx = s1 + ne * ((long long)vmin - bias);
          const __int128 num = (__int128)ne * s_i64[10] - (__int128)s1 * s1;  // n^2 var_biased, exact
          emean = (A)sumx / (A)ne;
          estd = ne > 1 ? asqrt(i128A<A>(num) / ((A)ne * (A)(ne - 1))) : (A)0;
          put(p, row, Q_EDGE + E_II, i2d(sumx));
          put(p, row, Q_EDGE + E_MAX, i2d((long long)emx - bias));
          put(p, row, Q_EDGE + E_MIN, i2d((long long)emn - bias));
          putA(p, row, Q_EDGE + E_STD, estd);
        } else {
          const A es5 = s_sc[5] + s_sl[5];
          emean = (A)fmn + es5 / (A)ne;
          putA(p, row, Q_EDGE + E_II, (A)fmn * (A)ne + es5);
          put(p, row, Q_EDGE + E_MAX, f2d(Enc<T>::decf(emx)));
          put(p, row, Q_EDGE + E_MIN, f2d(Enc<T>::decf(emn)));
        }
        putA(p, row, Q_EDGE + E_MEAN, emean);
        s_pa[10] = emean;
        if (need & NEED_SAVE) {
          double* sv = p.saved + (size_t)item * SV_WORDS;
          sv[SV_EMEAN] = to_d(emean);
          sv[SV_ESTD] = to_d(estd);
          sv[SV_ECNT] = i2d(ne);
        }
      }
    }
    __syncthreads();
    const A mu_hi = s_pa[0], mu_lo = s_pa[1];
    const A cx = s_pa[2], cy = s_pa[3], cz = s_pa[4], bx = s_pa[5], by = s_pa[6], bz = s_pa[7];
    const A sumI = s_pa[8], energy = s_pa[9];
    const bool wvalid = sumI != 0;

    // ---- pass 2: centred sums (one loop per feature group keeps the live
    // accumulators few) -------------------------------------------------------
    constexpr int NM = NDIM == 3 ? 20 : 10;
    A* res_st = res;            // [8]  statistics
    A* res_mi = res + 8;        // [NM] intensity-weighted moments
    A* res_mb = res + 8 + NM;   // [NM] binary moments
    // float images add the squared deviations of the edge pixels from their
    // mean as a ninth sum
    constexpr int NP2 = Enc<T>::INTEGER ? 8 : 9;
    const bool edge_p2 = !Enc<T>::INTEGER && do_edge;
    if ((need & (NEED_STATS | NEED_SAVE)) || edge_p2) {
      const A emean = s_pa[10];
      A acc[NP2];
#pragma unroll
      for (int i = 0; i < NP2; ++i) acc[i] = 0;
#pragma unroll 1
      for (int i = tid; i < n; i += C::NT) {
        const A v = Enc<T>::INTEGER ? (A)((int)pv[i] - ibias) : decA<T, A>(pv[i]);
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
        if constexpr (NP2 == 9)
          if (edge_p2 && edge_pixel<NDIM>(raster, pc[i], pad, Wp, Hp, plane)) acc[8] += (v - emean) * (v - emean);
      }
      if constexpr (NP2 == 8) {
        block_sum<C, A, 8>(acc, red, res_st);
      } else {
        block_sum<C, A, 9>(acc, red, s_sc + 4);  // s_sc[4..12]
        if (tid < 8) res_st[tid] = s_sc[4 + tid];
        if (edge_p2 && tid == 0) {
          const long long ne = s_i64[8];
          const A estd = ne > 1 ? asqrt(s_sc[12] / (A)(ne - 1)) : (A)0;
          putA(p, row, Q_EDGE + E_STD, estd);
          if (need & NEED_SAVE) p.saved[(size_t)item * SV_WORDS + SV_ESTD] = to_d(estd);
        }
        __syncthreads();
      }
    }
#pragma unroll 1
    for (int w = 0; w < 2; ++w) {
      if (!(need & (w ? NEED_MOM_BIN : (NEED_MOM_INT | NEED_SAVE)))) continue;
      A acc[NM];
#pragma unroll
      for (int i = 0; i < NM; ++i) acc[i] = 0;
      const A c0 = w ? bx : cx, c1 = w ? by : cy, c2 = w ? bz : cz;
#pragma unroll 1
      for (int i = tid; i < n; i += C::NT) {
        const unsigned c = pc[i];
        const A u0 = (A)(NDIM == 3 ? (int)(c & 2047u) : (int)(c & 0xFFFFu)) - c0;
        const A u1 = (A)(NDIM == 3 ? (int)((c >> 11) & 2047u) : (int)(c >> 16)) - c1;
        const A u2 = (A)(NDIM == 3 ? (int)(c >> 22) : 0) - c2;
        const A wt = w ? (A)1 : (Enc<T>::INTEGER ? (A)((int)pv[i] - ibias) : decA<T, A>(pv[i]));
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

    // ---- the sums go to k_stats_final (one warp per ROI), which derives the
    // statistics, moments and Hu invariants, so no block waits on that
    // serial arithmetic
    store_sacc<A>(p, item, NM, res_st, res_mi, res_mb, mu_hi + mu_lo, sumI, energy, cx, cy, cz, bx, by, bz, s_cd);
    (void)wvalid;

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
        putA(p, row, Q_STATS + S_ENTROPY, s_sc[8]);
        putA(p, row, Q_STATS + S_UNIFORMITY, s_sc[9]);
      }
    }

    // the pixel list's coordinates are not needed after the moments: keep
    // each pixel's padded raster index (low 16 bits; cells <= 16,384) and its
    // own bin (high 16 bits) there instead of decoding them per neighbour
    if (need_levels)
      for (int i = tid; i < n; i += C::NT) {
        const unsigned c = pc[i];
        const int x = NDIM == 3 ? (int)(c & 2047u) : (int)(c & 0xFFFFu);
        const int y = NDIM == 3 ? (int)((c >> 11) & 2047u) : (int)(c >> 16);
        const int z = NDIM == 3 ? (int)(c >> 22) : 0;
        const unsigned ci = (unsigned)(((NDIM == 3 ? z + pad : 0) * Hp + (y + pad)) * Wp + (x + pad));
        pc[i] = ci | ((unsigned)raster[ci] << 16);
      }

    // ---- NGTDM (Table S3 rows 246-250) and GLDM (rows 251-264) ----------------
    // One visit of each pixel's Chebyshev-1 neighbours (raster cells that are
    // not the sentinel) gives the NGTDM level sum and count and the GLDM
    // dependence (1 + the neighbours at the pixel's own level).  NGTDM: n_L
    // and the fixed-point s_L per level in shared memory.  GLDM: the
    // (level, dependence) cells counted in the shared hash table, with runs of
    // equal cells in consecutive lanes added once, then per-level sums.
    if (need_ngtdm || need_gldm) {
      const int ng = p.ng;
      unsigned long long* S = (unsigned long long*)marg;  // [ng] sums of |L - A|, 2^-32 units
      unsigned* nL = (unsigned*)(S + ng);                  // [ng] valid pixels per level
      unsigned* lst = nL + ng;                             // [ng] levels present
      uint16_t* cells = rank;                              // occupied slots of the GLDM table
      int cap = 64;
      while (cap < 2 * n && cap < C::TAB) cap <<= 1;
      if (need_ngtdm)
        for (int i = tid; i < ng; i += C::NT) {
          S[i] = 0;
          nL[i] = 0;
        }
      if (need_gldm) {
        for (int i = tid; i < cap; i += C::NT) tab[i] = 0;
        if (tid == 0) s_ncell = 0;
      }
      __syncthreads();
      for (int i0 = warp * 32; i0 < n; i0 += C::NT) {
        const int i = i0 + lane;
        unsigned key = 0xFFFFFFFFu;
        if (i < n) {
          const unsigned w = pc[i];
          const int ci = (int)(w & 0xFFFFu);
          const unsigned a = w >> 16;
          int sum = 0, cnt = 0, same = 0;
#pragma unroll
          for (int dz = (NDIM == 3 ? -1 : 0); dz <= (NDIM == 3 ? 1 : 0); ++dz)
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
              for (int dx = -1; dx <= 1; ++dx) {
                if (dx == 0 && dy == 0 && dz == 0) continue;
                const unsigned b = raster[ci + (dz * Hp + dy) * Wp + dx];
                if (b != 0xFFFFu) {
                  sum += (int)b + 1;
                  ++cnt;
                }
                same += b == a;
              }
          if (need_ngtdm && cnt) {
            atomicAdd(&nL[a], 1u);
            atomicAdd(&S[a], ngtdm_term((int)a + 1, sum, cnt));
          }
          key = (a << 5) | (unsigned)same;  // level, dependence - 1
        }
        if (need_gldm) {
          const unsigned add = run_leader(key, 0xFFFFFFFFu);
          if (add) tab_add(tab, cap, key, add, cells, &s_ncell);
        }
      }
      __syncthreads();
      if (need_ngtdm) ngtdm_features<C, A>(p, row, ng, nL, S, lst, red, s_sc, s_i64);  // ends with a barrier
      if (need_gldm) {
        unsigned long long* Cm = (unsigned long long*)marg;  // [ng] sum_j P round(2^32 / j^2)
        unsigned* R = (unsigned*)(Cm + ng);                   // [ng] pixels per level
        unsigned* C2 = R + ng;                                // [ng] sum_j P j^2
        unsigned* col = C2 + ng;                              // [27] pixels per dependence
        for (int i = tid; i < ng; i += C::NT) {
          Cm[i] = 0;
          R[i] = 0;
          C2[i] = 0;
        }
        if (tid < 27) col[tid] = 0;
        __syncthreads();
        const int ncell = (int)s_ncell;
        long long ent = 0;
        for (int k = tid; k < ncell; k += C::NT) {
          const unsigned wv = tab[cells[k]];
          const unsigned cnt = wv & 0xFFFFu, key = wv >> 16;
          const unsigned a = key >> 5, j = (key & 31u) + 1u;
          atomicAdd(&R[a], cnt);
          atomicAdd(&C2[a], cnt * j * j);
          atomicAdd(&Cm[a], (unsigned long long)cnt * inv_sq_fx(j));
          atomicAdd(&col[j - 1], cnt);
          ent += clog_fx<A>(p.clog, cnt);
        }
        __syncthreads();
        gldm_features<C, A>(
            p, row, ng, NDIM == 3 ? 27 : 9,
            [&](int a, unsigned long long& r, unsigned long long& c2, unsigned long long& cm) {
              r = R[a];
              c2 = C2[a];
              cm = Cm[a];
            },
            col, ent, red, s_sc, s_i64);
      }
    }

    // ---- GLCM ------------------------------------------------------------------
    // Per offset, three passes and one reduction:
    //   insert: warp-aggregated inserts of (min bin, max bin) into a shared
    //     hash table that records its occupied slots, and the row marginal
    //     p_x (one update per run of equal keys);
    //   cells: the sum / difference marginals p_{x+y}, p_{x-y}, the sums
    //     linear in the pairs (powers of i + j and |i - j|, sum i^2), sum C^2,
    //     sum C log2 C, max C and the mutual information (p_x is final);
    //   marginals: the entropies of p_x, p_{x+y}, p_{x-y} and the
    //     inverse-difference family over their nonzero entries, zeroing them
    //     as it goes, and the clean-up of the table;
    //   reduction: 19 int64 sums (one maximum) over the warps.
    // All sums are integers or fixed point, so nothing depends on the order
    // of the hash table or of the atomics.
    if (need_glcm) {
      const int ng = p.ng;
      unsigned* px = marg;
      unsigned* psum = marg + ng;      // index a + b, 0 .. 2ng-2
      unsigned* pdiff = marg + 3 * ng; // index |a - b|
      uint16_t* cells = rank;          // occupied slots of the table (rank is free until the sort)
      long long* s_cv = (long long*)red;  // [NW][19] per-warp sums
      int cap = 64;
      while (cap < 2 * n && cap < C::TAB) cap <<= 1;
      const bool dbg = p.dbg_roi == (int64_t)item;
      for (int i = tid; i < cap; i += C::NT) tab[i] = 0;
      for (int i = tid; i < 4 * ng; i += C::NT) marg[i] = 0;
      if (tid == 0) {
        s_ncell = 0;
        s_npair = 0;
      }
      for (int di = 0; di < p.n_dist; ++di) {
        for (int dir = 0; dir < p.n_dirs; ++dir) {
          const int oi = di * p.n_dirs + dir;
          const int dx = p.off[oi][0], dy = p.off[oi][1], dz = p.off[oi][2];
          const int olin = (dz * Hp + dy) * Wp + dx;
          __syncthreads();
          // accumulate pairs (q, q + o) inside the ROI
          unsigned npair = 0;  // this lane's pairs
          for (int i0 = warp * 32; i0 < n; i0 += C::NT) {
            const int i = i0 + lane;
            unsigned key = 0xFFFFFFFFu;
            if (i < n) {
              const unsigned w = pc[i];
              const unsigned a = w >> 16, b = raster[(w & 0xFFFFu) + olin];
              if (b != 0xFFFFu) key = a < b ? (a << 8) | b : (b << 8) | a;
            }
            // one insert per run of equal keys in consecutive lanes (noisy
            // images give runs of 1; smooth ones long runs that would
            // otherwise serialise on one address)
            npair += key != 0xFFFFFFFFu;
            const unsigned add = run_leader(key, 0xFFFFFFFFu);
            if (add) {
              tab_add(tab, cap, key, add, cells, &s_ncell);
              atomicAdd(&px[key >> 8], add);
              atomicAdd(&px[key & 255u], add);
            }
          }
          npair = __reduce_add_sync(0xFFFFFFFFu, npair);
          if (lane == 0 && npair) atomicAdd(&s_npair, npair);
          __syncthreads();
          const int ncell = (int)s_ncell;
          if (ncell == 0) {  // no pair for this offset (nothing was touched): every feature NaN
            long long z[GN];
            store_gacc(p, item, oi, z, true);
            continue;
          }
          const long long Tl = 2 * (long long)s_npair;  // total mass of the symmetric matrix
          // cell pass.  cv: [0..3] sum C k^m (k = i + j), [4..5] sum C d^m
          // (d = |i - j|), [6] sum C i^2, [7] sum C^2, [8] sum C log2 C (2^-24),
          // [9] mutual information (2^-32), [10] max C; C = the count of one
          // matrix cell, each off-diagonal cell standing for its mirror too
          long long cv[11];
#pragma unroll
          for (int k = 0; k < 11; ++k) cv[k] = 0;
          for (int sc = tid; sc < ncell; sc += C::NT) {
            const unsigned wv = tab[cells[sc]];
            const unsigned key = wv >> 16, cnt = wv & 0xFFFFu;
            const unsigned a = key >> 8, b = key & 255u;
            atomicAdd(&psum[a + b], 2 * cnt);
            atomicAdd(&pdiff[b - a], 2 * cnt);
            const long long Cm = 2 * (long long)cnt;  // mass of the cell pair (or of the doubled diagonal cell)
            const long long k = a + b + 2, d = b - a, k2 = k * k;
            cv[0] += Cm * k;
            cv[1] += Cm * k2;
            cv[2] += Cm * k2 * k;
            cv[3] += Cm * k2 * k2;
            cv[4] += Cm * d;
            cv[5] += Cm * d * d;
            cv[6] += (long long)cnt * ((long long)(a + 1) * (a + 1) + (long long)(b + 1) * (b + 1));
            const long long Cc = a == b ? Cm : (long long)cnt;
            const long long mult = a == b ? 1 : 2;
            cv[7] += mult * Cc * Cc;
            cv[8] += mult * clog_fx<A>(p.clog, (unsigned)Cc);
            cv[9] += mult * mi_fx<A>((unsigned)Cc, Tl, px[a], px[b]);
            cv[10] = Cc > cv[10] ? Cc : cv[10];
            if (dbg) {
              p.dbg_glcm[(int64_t)oi * ng * ng + a * ng + b] = (unsigned)Cc;
              p.dbg_glcm[(int64_t)oi * ng * ng + b * ng + a] = (unsigned)Cc;
            }
          }
          __syncthreads();  // the marginals are final, the table is read
          // marginal entropies (2^-24) and inverse differences (2^-32) over
          // the nonzero marginal entries, which are zeroed for the next
          // offset; the table slots this offset used are cleared
          long long mv[8];
#pragma unroll
          for (int k = 0; k < 8; ++k) mv[k] = 0;
          for (int i = tid; i < ng; i += C::NT) {
            const unsigned c = px[i];
            if (c) {
              mv[0] += clog_fx<A>(p.clog, c);
              px[i] = 0;
            }
          }
          for (int i = tid; i < 2 * ng - 1; i += C::NT) {
            const unsigned c = psum[i];
            if (c) {
              mv[1] += clog_fx<A>(p.clog, c);
              psum[i] = 0;
            }
          }
          for (int i = tid; i < ng; i += C::NT) {
            const unsigned c = pdiff[i];
            if (c) {
              mv[2] += clog_fx<A>(p.clog, c);
              long long w5[GN];
#pragma unroll
              for (int q = 15; q < 20; ++q) w5[q] = 0;
              invdiff_fx<A>(p, c, i, w5);
#pragma unroll
              for (int q = 0; q < 5; ++q) mv[3 + q] += w5[15 + q];
              pdiff[i] = 0;
            }
          }
          for (int sc = tid; sc < ncell; sc += C::NT) tab[cells[sc]] = 0;
          // per-warp sums (reduce-scatter), [warp][0..10] cell values (10: max),
          // [warp][11..18] marginal values
          {
            long long mx = cv[10];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
              const long long y = __shfl_xor_sync(0xFFFFFFFFu, mx, o);
              mx = y > mx ? y : mx;
            }
            long long v10[10];
#pragma unroll
            for (int k = 0; k < 10; ++k) v10[k] = cv[k];
            long long hi, lo;
            warp_rs<long long, 10>(v10, hi, lo);
            constexpr int SH = RsSlots<10>::SH;
            int slot = lane >> SH;
            if ((lane & ((1 << SH) - 1)) == 0 && slot < 10) s_cv[warp * 19 + slot] = hi;
            if (lane == 0) s_cv[warp * 19 + 10] = mx;
            warp_rs<long long, 8>(mv, hi, lo);
            (void)lo;
            constexpr int SH8 = RsSlots<8>::SH;
            slot = lane >> SH8;
            if ((lane & ((1 << SH8) - 1)) == 0) s_cv[warp * 19 + 11 + slot] = hi;
          }
          __syncthreads();
          if (tid < GN) {  // combine and hand the sums to k_glcm_final
            long long v;
            if (tid == 0) {
              v = Tl;
            } else {
              const int j = tid - 1;  // slot: 0..10 cell values, 11..18 marginal values
              v = s_cv[j];
              for (int w = 1; w < C::NW; ++w) {
                const long long y = s_cv[w * 19 + j];
                v = j == 10 ? (y > v ? y : v) : v + y;
              }
            }
            long long* g = (long long*)(p.gacc + ((size_t)item * (p.n_dist * p.n_dirs) + oi) * GACC_BYTES);
            g[tid] = gacc_value(tid, v, tid == 9 || tid >= 12 ? tlog_fx(p.clog, Tl) : 0);
          }
          if (tid == 0) {
            s_ncell = 0;
            s_npair = 0;
          }
        }
      }
      __syncthreads();
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
          const unsigned dg = act ? (src[i] >> shift) & 255u : 0u;
          // lanes holding the same digit, from 8 ballots (constant cost, unlike
          // a match over up to 32 distinct values)
          unsigned peers = __ballot_sync(0xFFFFFFFFu, act);
#pragma unroll
          for (int bit = 0; bit < 8; ++bit) {
            const unsigned bb = __ballot_sync(0xFFFFFFFFu, (dg >> bit) & 1u);
            peers &= ((dg >> bit) & 1u) ? bb : ~bb;
          }
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
      order_tail<T, C, A>(p, row, v, n, red, s_sd, s_bnd, s_sc);
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

// First-order statistics (Table S1/S5), moments and Hu invariants (Table S2,
// S5) of every ROI from the sums its accumulation kernel left in sacc: one
// warp per ROI (the statistics one column per lane, lanes 0..NM-1 the
// moments).
template <class T, int NDIM, class A>
__global__ void __launch_bounds__(256) k_stats_final(KParams p) {
  const int64_t nroi = min((int64_t)*p.n_roi, p.cap_roi);
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t item = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); item < nroi; item += nw) {
    const A* g = (const A*)(p.sacc + (size_t)item * SACC_BYTES);
    const RoiInfo r = p.rois[item];
    double* row = p.table + item * p.n_col;
    double* save = (p.need & NEED_SAVE) ? p.saved + item * SV_WORDS : nullptr;
    const bool wvalid = g[49] != (A)0;
    const double* cd = (const double*)(p.sacc + (size_t)item * SACC_BYTES + SACC_CD);
    finalize_stats<T, NDIM, A>(p, row, g, (int)r.n, g[48], g[49], g[50], r.vmin, r.vmax, (int64_t)(r.key >> 32),
                               r.x0, r.y0, r.z0, cd, wvalid, save);
    const bool need_int = (p.need & (NEED_MOM_INT | NEED_SAVE)) != 0, need_bin = (p.need & NEED_MOM_BIN) != 0;
    if (NDIM == 2) {  // both weightings at once: intensity on lanes 0..15, binary on lanes 16..31
      const bool hb = (threadIdx.x & 16) != 0;
      if (need_int || need_bin)
        finalize_moments_warp<NDIM, A>(p, row, hb ? 5 : 0, g + (hb ? 28 : 8), hb ? g[54] : g[51], hb ? g[55] : g[52],
                                       hb ? g[56] : g[53], hb ? cd + 3 : cd, hb ? (double)r.n : to_d(g[49]),
                                       hb || wvalid, hb || !save ? nullptr : save + SV_MU, hb ? need_bin : need_int,
                                       hb ? 16 : 0);
    } else {
      if (need_int)
        finalize_moments_warp<NDIM, A>(p, row, 0, g + 8, g[51], g[52], g[53], cd, to_d(g[49]), wvalid,
                                       save ? save + SV_MU : nullptr);
      if (need_bin)
        finalize_moments_warp<NDIM, A>(p, row, 5, g + 28, g[54], g[55], g[56], cd + 3, (double)r.n, true, nullptr);
    }
  }
}

template <class T, int NDIM, class A>
cudaError_t launch_stats_final(const KParams& p, int nsm, cudaStream_t st) {
  const int64_t rows = p.cap_roi < p.max_rois ? p.cap_roi : p.max_rois;
  int64_t nb = (rows + 7) / 8;
  if (nb > 16ll * nsm) nb = 16ll * nsm;
  if (nb < 1) nb = 1;
  k_stats_final<T, NDIM, A><<<(int)nb, 256, 0, st>>>(p);
  return cudaGetLastError();
}

template <class T, class C>
cudaError_t launch_roi_c(const KParams& p, int cls, int fp64, int nsm, cudaStream_t st) {
  if (p.ndim == 3)
    return fp64 ? launch_roi_one<T, 3, C, double>(p, cls, nsm, st) : launch_roi_one<T, 3, C, float>(p, cls, nsm, st);
  return fp64 ? launch_roi_one<T, 2, C, double>(p, cls, nsm, st) : launch_roi_one<T, 2, C, float>(p, cls, nsm, st);
}

// cls 0..N_BLOCK_CLASSES-1: the block classes; cls N_BLOCK_CLASSES:
// k_stats_final over all ROIs
template <class T>
cudaError_t launch_roi_t(const KParams& p, int cls, int fp64, int nsm, cudaStream_t st) {
  static_assert(N_BLOCK_CLASSES == 4, "one case per block class");
  switch (cls) {
    case 0: return launch_roi_c<T, ClassW>(p, cls, fp64, nsm, st);
    case 1: return launch_roi_c<T, ClassS>(p, cls, fp64, nsm, st);
    case 2: return launch_roi_c<T, ClassM>(p, cls, fp64, nsm, st);
    case 3: return launch_roi_c<T, ClassL>(p, cls, fp64, nsm, st);
    default:
      if (p.ndim == 3)
        return fp64 ? launch_stats_final<T, 3, double>(p, nsm, st) : launch_stats_final<T, 3, float>(p, nsm, st);
      return fp64 ? launch_stats_final<T, 2, double>(p, nsm, st) : launch_stats_final<T, 2, float>(p, nsm, st);
  }
}

}  // namespace nyx
