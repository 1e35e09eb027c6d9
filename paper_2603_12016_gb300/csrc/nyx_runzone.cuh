// nyx_runzone.cuh -- grey-level run-length (GLRLM, Table S3 rows from 193)
// and size-zone (GLSZM, Table S3 rows 228-245) features on the GLCM grey
// levels.  Included by nyx_rz_<dtype>.cu.
//
// Both families count items by (grey level i, size s):
//   GLRLM, per unit direction v (the GLCM's 4 directions in 2D, 13 in 3D):
//     a run is a maximal chain p, p + v, p + 2v, ... of ROI pixels of one
//     level; its size is its length.  A pixel starts a run when the pixel
//     at p - v is not an ROI pixel of its level, so every run is found once
//     by walking from its start.  Features are taken per direction, then
//     averaged over the directions.
//   GLSZM: a zone is a maximal set of one level's ROI pixels connected
//     through their 8 (2D) / 26 (3D) neighbours; its size is its area.
//     Zones are the sets of a union-find over the links p -- p + v between
//     pixels of one level, v over the same 4 / 13 forward directions (each
//     neighbour pair is one forward link).
//
// From the item counts c(i, s) of one set (a direction, or the zones), with
// M items over the ROI's Np pixels, n_i = sum_s c(i, s), n_s = sum_i c(i, s):
//   [0] sum 1/s^2 / M        [1] sum s^2 / M       [2] sum n_i^2 / M  [3] / M^2
//   [4] sum n_s^2 / M        [5] / M^2             [6] M / Np
//   [7] grey-level variance  [8] size variance     [9] entropy of c / M (log2)
//   [10] sum 1/i^2 / M       [11] sum i^2 / M      [12] sum 1/(i^2 s^2) / M
//   [13] sum i^2/s^2 / M     [14] sum s^2/i^2 / M  [15] sum i^2 s^2 / M
//   [16] mean level          [17] mean size        (GLSZM only)
// Every sum is an integer or a 2^-63 / 2^-47 fixed-point integer summed in
// 128 bits (the reciprocals of the emphases), and the entropy is
// log2 M - sum c log2 c / M with c log2 c in 2^-24 units, so no result
// depends on the order of atomics, hash slots or reductions: tables are
// bit-identical from run to run.
//
// Paths:
//   k_rz<T, NDIM, Tier>  ROIs of the block classes, one block per ROI: the
//       level raster (one sentinel cell around the bounding box) in shared
//       memory; runs walk the raster, zones are a union-find on 16-bit
//       parent indices in shared memory; (i, s) counts in a shared hash.
//       Tier k drains the queue of size class k: one warp for the warp
//       class (<= 1,024 padded cells), blocks for the small (<= 4,096),
//       medium (<= 8,192) and large (<= 16,384) classes.
//   multi-block ROIs, units (ROI, chunk of BIG_CHUNK cells), zone parents
//   and areas one 32-bit word each per image pixel, cleared by one memset:
//       k_rzb_items  runs, walking through global memory (a run may cross
//                    chunks: only its start pixel reports it), and the union
//                    of each pixel with its forward neighbours of the same
//                    level (global atomicCAS)
//       k_rzb_count  zone areas at the roots, parents compressed
//       k_rzb_zones  one item per zone, from its root
//     the items of a unit meet in a shared hash, which flushes into the
//     ROI's global per-set tables in its arena region; k_rzb_final reduces
//     each (ROI, set) table on its own block, and the last of an ROI's sets
//     to finish computes the features.
#pragma once

#include "nyx_roi_big.cuh"

namespace nyx {

typedef unsigned long long rz_u64;
typedef unsigned __int128 rz_u128;

// Tier geometry of the block path: threads, max padded cells, max pixels,
// joint-hash slots, size-marginal slots (twice the threads of the matching
// k_roi class measured faster: the sets are short phases between barriers).  The hash sizes follow from the
// number of distinct (i, s) keys of a set: their sizes sum to at most the
// ROI's pixel count N, so there are at most sqrt(2 N Ng) of them (<= 724
// for N = 1,024, <= 2,048 for N = 8,192 at Ng = 256), and at most sqrt(2 N)
// distinct sizes.
template <int NT_, int CELLS_, int PIX_, int HC_, int HS_>
struct RzTier {
  static constexpr int NT = NT_, NW = NT_ / 32, CELLS = CELLS_, PIX = PIX_, HC = HC_, HS = HS_;
};
using RzT0 = RzTier<32, 1024, 256, 512, 64>;
using RzT1 = RzTier<256, 4096, 1024, 2048, 128>;
using RzT2 = RzTier<512, 8192, 4096, 4096, 256>;
using RzT3 = RzTier<512, 16384, 8192, 4096, 256>;
constexpr int RZ_NV = 26;          // reduced values per set
constexpr int RZ_BIG_HS = 8192;    // size-marginal slots of k_rzb_final
constexpr int RZ_BIG_SH = 4096;    // shared item slots per unit of the multi-block kernels
constexpr int RZ_SPIN = 1 << 20;   // iteration limit of every retry loop

// unit direction k of the GLCM (2D: 0, 45, 90, 135 degrees with rows growing
// downward; 3D: the 13 vectors of {-1,0,1}^3 whose first nonzero component
// in (z, y, x) order is positive, z outermost, x fastest)
__host__ __device__ inline void rz_dir(int ndim, int k, int& dx, int& dy, int& dz) {
  if (ndim != 3) {
    const int tx[4] = {1, 1, 0, -1}, ty[4] = {0, -1, -1, -1};
    dx = tx[k];
    dy = ty[k];
    dz = 0;
    return;
  }
  int idx = 0;
  for (int z = -1; z <= 1; ++z)
    for (int y = -1; y <= 1; ++y)
      for (int x = -1; x <= 1; ++x) {
        const int first = z != 0 ? z : (y != 0 ? y : x);
        if (first <= 0) continue;
        if (idx++ == k) {
          dx = x;
          dy = y;
          dz = z;
          return;
        }
      }
  dx = dy = dz = 0;
}

// Zone links that can be skipped: a cell p links to each forward neighbour
// n = p + d of its level, unless an earlier direction d' (in rz_dir order)
// gave a neighbour m = p + d' of its level adjacent to n (Chebyshev distance
// 1).  Then p -- m and m -- n are links too (n is another of m's 26
// neighbours), both from a source later in the (raster index, reversed
// direction order) order than p -- n (m and n come after p in raster order;
// p -- m has an earlier direction), so by induction from the last links p
// and n end in one zone.  In a uniform region one link per cell remains.
// adj_mask(d): the directions d' < d whose neighbours are adjacent to p + d.
__host__ __device__ inline unsigned rz_adj_mask(int ndim, int d) {
  int ax, ay, az;
  rz_dir(ndim, d, ax, ay, az);
  unsigned m = 0;
  for (int e = 0; e < d; ++e) {
    int bx, by, bz;
    rz_dir(ndim, e, bx, by, bz);
    const int cx = ax - bx, cy = ay - by, cz = az - bz;
    if (cx >= -1 && cx <= 1 && cy >= -1 && cy <= 1 && cz >= -1 && cz <= 1) m |= 1u << e;
  }
  return m;
}

// ---- fixed-point terms -----------------------------------------------------
// round(2^63 / d) for 1 <= d < 2^62
__device__ inline rz_u64 rz_q63(rz_u64 d) {
  return d == 1 ? (1ull << 63) : ((1ull << 63) + (d >> 1)) / d;
}
// q(i) = round(2^63 / i^2) and q(s) = round(2^63 / s^2) come from the plan's
// tables (levels up to 256, sizes up to RZ_STAB, computed once on the host
// in integer arithmetic); larger sizes take the division
__device__ inline rz_u64 rz_qs(const KParams& p, rz_u64 s) {
  return s <= (rz_u64)RZ_STAB ? __ldg(p.rz_qs + s) : rz_q63(s * s);
}
// round(2^63 / (i^2 s^2)) ~ q(i) q(s) / 2^63, rounded (relative error below
// (i^2 + s^2) 2^-64: a fixed, order-free function of (i, s))
__device__ inline rz_u64 rz_inv63(rz_u64 qi, rz_u64 qs) {
  return (rz_u64)(((rz_u128)qi * qs + ((rz_u128)1 << 62)) >> 63);
}
// round(2^47 i^2 / s^2) ~ i^2 q(s) / 2^16, rounded (i^2 <= 2^16)
__device__ inline rz_u64 rz_r47(rz_u64 i2, rz_u64 qs) {
  return (rz_u64)(((rz_u128)i2 * qs + (1u << 15)) >> 16);
}
// 128-bit sums travel through the block reduction as three 43-bit limbs,
// whose sums over a block stay below 2^52
constexpr rz_u64 RZ_LIMB = (1ull << 43) - 1;
__device__ inline void rz_limbs(rz_u128 x, rz_u64* o) {
  o[0] = (rz_u64)x & RZ_LIMB;
  o[1] = (rz_u64)(x >> 43) & RZ_LIMB;
  o[2] = (rz_u64)(x >> 86);
}
__device__ inline rz_u128 rz_unlimb(const rz_u64* s) {
  return (rz_u128)s[0] + ((rz_u128)s[1] << 43) + ((rz_u128)s[2] << 86);
}
__device__ inline double rz_u128d(rz_u128 x) {
  return (double)(rz_u64)(x >> 64) * 18446744073709551616.0 + (double)(rz_u64)x;
}
__device__ inline double rz_i128d(__int128 x) {
  return x < 0 ? -rz_u128d((rz_u128)(-x)) : rz_u128d((rz_u128)x);
}

// add NV 64-bit values of every thread into out[] (shared): warp sums of
// 24-bit limbs (single-instruction reductions that cannot overflow), then
// one atomic per warp and value (integers, so the order does not matter)
template <int NV>
__device__ inline void rz_warp_add(rz_u64 (&v)[NV], rz_u64* out) {
  const int lane = threadIdx.x & 31;
  bool any = false;
#pragma unroll
  for (int i = 0; i < NV; ++i) any |= v[i] != 0;
  if (!__any_sync(0xFFFFFFFFu, any)) return;  // a warp without cells adds nothing
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    const rz_u64 x = v[i];
    const unsigned l0 = __reduce_add_sync(0xFFFFFFFFu, (unsigned)(x & 0xFFFFFFu));
    const unsigned l1 = __reduce_add_sync(0xFFFFFFFFu, (unsigned)((x >> 24) & 0xFFFFFFu));
    const unsigned l2 = __reduce_add_sync(0xFFFFFFFFu, (unsigned)(x >> 48));
    const rz_u64 t = (rz_u64)l0 + ((rz_u64)l1 << 24) + ((rz_u64)l2 << 48);
    if (lane == 0 && t) atomicAdd(out + i, t);
  }
}

// indices of the reduced values of one set
enum : int {
  RZ_M = 0, RZ_SI, RZ_SI2, RZ_QI, RZ_SS, RZ_SS2, RZ_QS, RZ_E,
  RZ_RI = 8,       // sum n_i round(2^63 / i^2)                (3 limbs)
  RZ_RS2I = 11,    // sum_i (sum_s c s^2) round(2^63 / i^2)    (3 limbs)
  RZ_RS = 14,      // sum n_s round(2^63 / s^2)                (3 limbs)
  RZ_RIS = 17,     // sum c round(2^63 / (i^2 s^2))            (3 limbs)
  RZ_RI2S = 20,    // sum c round(2^47 i^2 / s^2)              (3 limbs)
  RZ_SI2S2 = 23,   // sum c i^2 s^2                            (3 limbs)
};

// The features of one set from its reduced values (FP64, one thread).
// add = true adds them to f (the direction mean of the GLRLM), else stores.
__device__ inline void rz_features(const rz_u64* s, rz_u64 Np, int nf, double* f, bool add) {
  const rz_u64 M = s[RZ_M];
  const double Md = (double)M, iM = 1.0 / Md, M2 = Md * Md;
  const double P63 = 1.0842021724855044e-19, P47 = 7.105427357601002e-15, P24 = 5.9604644775390625e-08;
  double v[18];
  v[0] = rz_u128d(rz_unlimb(s + RZ_RS)) * P63 * iM;
  v[1] = (double)s[RZ_SS2] * iM;
  v[2] = (double)s[RZ_QI] * iM;
  v[3] = (double)s[RZ_QI] / M2;
  v[4] = (double)s[RZ_QS] * iM;
  v[5] = (double)s[RZ_QS] / M2;
  v[6] = Md / (double)Np;
  v[7] = rz_i128d((__int128)M * s[RZ_SI2] - (__int128)s[RZ_SI] * s[RZ_SI]) / M2;
  v[8] = rz_i128d((__int128)M * s[RZ_SS2] - (__int128)s[RZ_SS] * s[RZ_SS]) / M2;
  v[9] = log2(Md) - (double)(long long)s[RZ_E] * P24 * iM;
  v[10] = rz_u128d(rz_unlimb(s + RZ_RI)) * P63 * iM;
  v[11] = (double)s[RZ_SI2] * iM;
  v[12] = rz_u128d(rz_unlimb(s + RZ_RIS)) * P63 * iM;
  v[13] = rz_u128d(rz_unlimb(s + RZ_RI2S)) * P47 * iM;
  v[14] = rz_u128d(rz_unlimb(s + RZ_RS2I)) * P63 * iM;
  v[15] = rz_u128d(rz_unlimb(s + RZ_SI2S2)) * iM;
  v[16] = (double)s[RZ_SI] * iM;
  v[17] = (double)s[RZ_SS] * iM;
  for (int q = 0; q < nf; ++q) f[q] = add ? f[q] + v[q] : v[q];
}

// size-marginal hash in shared memory: key s (>= 1; 0 = empty), count
__device__ inline void rz_hs_add(unsigned* key, unsigned* cnt, int cap, unsigned s, unsigned c, unsigned* err) {
  unsigned h = (s * 2654435761u) & (unsigned)(cap - 1);
  for (int probe = 0; probe < cap; ++probe) {
    unsigned k = ((volatile unsigned*)key)[h];
    if (k == 0) {
      k = atomicCAS(key + h, 0u, s);
      if (k == 0) k = s;
    }
    if (k == s) {
      atomicAdd(cnt + h, c);
      return;
    }
    h = (h + 1) & (unsigned)(cap - 1);
  }
  atomicOr(err, E_INTERNAL);
}

// The reduced values of one set, in two phases separated by a barrier.
// Phase 1 (rz_joint_pass): joint(f) calls f(i, s, c) for the (level, size,
// count) cells this thread owns (and clears them); the cells feed the
// per-level arrays lvl_n / lvl_a (item count and sum c s^2 per level) and the
// size hash, and this thread's joint sums v[RZ_SI2S2, RZ_RIS, RZ_RI2S, RZ_E].
// Phase 2 (rz_marg_pass): the per-level and per-size sums, clearing lvl_n,
// lvl_a and the size hash for the next set, then every value is added into
// out[RZ_NV] (zeroed beforehand).
template <class Joint>
__device__ inline void rz_joint_pass(Joint joint, const KParams& p, unsigned* lvl_n, rz_u64* lvl_a,
                                     unsigned* hs_key, unsigned* hs_cnt, int hs_cap, rz_u128 (&jv)[3],
                                     rz_u64& ent) {
  jv[0] = jv[1] = jv[2] = 0;
  ent = 0;
  joint([&](unsigned i, rz_u64 s, unsigned c) {
    const rz_u64 i2 = (rz_u64)i * i, qs = rz_qs(p, s);
    atomicAdd(lvl_n + (i - 1), c);
    atomicAdd(lvl_a + (i - 1), (rz_u64)c * s * s);
    rz_hs_add(hs_key, hs_cnt, hs_cap, (unsigned)s, c, p.err);
    jv[0] += (rz_u128)c * i2 * s * s;
    jv[1] += (rz_u128)c * rz_inv63(__ldg(p.rz_qi + i), qs);
    jv[2] += (rz_u128)c * rz_r47(i2, qs);
    ent += (rz_u64)tlog_fx(p.clog, (long long)c);
  });
}

template <int NT>
__device__ inline void rz_marg_pass(const KParams& p, unsigned* lvl_n, rz_u64* lvl_a, unsigned* hs_key,
                                    unsigned* hs_cnt, int hs_cap, const rz_u128 (&jv)[3], rz_u64 ent,
                                    rz_u64* out) {
  const int tid = threadIdx.x;
  rz_u64 M = 0, si = 0, si2 = 0, qi = 0, ss = 0, ss2 = 0, qs = 0;
  rz_u128 ri = 0, rs2i = 0, rs = 0;
  for (int a = tid; a < p.ng; a += NT) {
    const unsigned n = lvl_n[a];
    if (!n) continue;
    const rz_u64 i = (rz_u64)a + 1, q = __ldg(p.rz_qi + i);
    M += n;
    si += n * i;
    si2 += n * i * i;
    qi += (rz_u64)n * n;
    ri += (rz_u128)n * q;
    rs2i += (rz_u128)lvl_a[a] * q;
    lvl_n[a] = 0;
    lvl_a[a] = 0;
  }
  for (int h = tid; h < hs_cap; h += NT) {
    const unsigned sz = hs_key[h];
    if (!sz) continue;
    const rz_u64 n = hs_cnt[h], s2 = (rz_u64)sz * sz;
    ss += n * sz;
    ss2 += n * s2;
    qs += n * n;
    rs += (rz_u128)n * rz_qs(p, sz);
    hs_key[h] = 0;
    hs_cnt[h] = 0;
  }
  rz_u64 v[RZ_NV];
  v[RZ_M] = M;
  v[RZ_SI] = si;
  v[RZ_SI2] = si2;
  v[RZ_QI] = qi;
  v[RZ_SS] = ss;
  v[RZ_SS2] = ss2;
  v[RZ_QS] = qs;
  v[RZ_E] = ent;
  rz_limbs(ri, v + RZ_RI);
  rz_limbs(rs2i, v + RZ_RS2I);
  rz_limbs(rs, v + RZ_RS);
  rz_limbs(jv[1], v + RZ_RIS);
  rz_limbs(jv[2], v + RZ_RI2S);
  rz_limbs(jv[0], v + RZ_SI2S2);
  rz_warp_add<RZ_NV>(v, out);
}

// write one family's features (nf of them, starting at quantity q0) into the
// ROI's table row
__device__ inline void rz_write(const KParams& p, int64_t item, int q0, int nf, const double* f, double scale) {
  double* row = p.table + item * p.n_col;
  for (int q = threadIdx.x; q < nf; q += blockDim.x) {
    const int col = p.col_map[q0 + q];
    if (col >= 0) row[col] = f[q] * scale;
  }
}

// level (1..Ng) of encoded value e of an ROI with encoded range [vmin, vmax]:
// the GLCM bin + 1 (IBSI fixed bin number)
template <class T>
struct RzLevel {
  unsigned vmin, vmax;
  int ng;
  float fmn, fmx;
  FastDiv fd;
  __device__ void init(const RoiInfo& r, int ng_) {
    vmin = r.vmin;
    vmax = r.vmax;
    ng = ng_;
    fmn = Enc<T>::decf(vmin);
    fmx = Enc<T>::decf(vmax);
    fd.init(vmax > vmin ? vmax - vmin : 1u);
  }
  __device__ unsigned operator()(unsigned e) const {
    if (vmax <= vmin) return 1u;
    if constexpr (Enc<T>::INTEGER) return min(fd.div((unsigned)ng * (e - vmin)), (unsigned)(ng - 1)) + 1u;
    else return bin_float(Enc<T>::decf(e), fmn, fmx, ng) + 1u;
  }
};

// ---- hash tables of items ---------------------------------------------------
// block path: key (i << 16 | s) (i >= 1, so 0 = empty), n items added
// Insert-or-add into a block's joint hash; the thread that claims an empty
// slot appends its index to the occupied list lst (length *nl, room for
// lcap), so that the set's per-cell pass visits occupied slots only.
__device__ inline void rz_insert(unsigned* key, unsigned* cnt, int cap, unsigned k, unsigned n, uint16_t* lst,
                                 unsigned* nl, unsigned lcap, unsigned* err) {
  unsigned h = ((k * 2654435761u) >> 16) & (unsigned)(cap - 1);
  for (int probe = 0; probe < cap; ++probe) {
    unsigned cur = ((volatile unsigned*)key)[h];
    if (cur == 0) {
      cur = atomicCAS(key + h, 0u, k);
      if (cur == 0) {
        const unsigned at = atomicAdd(nl, 1u);
        if (at < lcap) lst[at] = (uint16_t)h;
        else atomicOr(err, E_INTERNAL);
        cur = k;
      }
    }
    if (cur == k) {
      atomicAdd(cnt + h, n);
      return;
    }
    h = (h + 1) & (unsigned)(cap - 1);
  }
  atomicOr(err, E_INTERNAL);
}

// multi-block path: an ROI's item tables in its arena region, one per set
// (GLRLM directions, then the zones), each `cap` slots of u64 keys
// (set << 48 | i << 32 | s; 0 = empty) with u32 counts, then each set's
// reduced values
struct RzTab {
  rz_u64* key;
  unsigned* cnt;
  rz_u64* red;
  unsigned* ctr;  // arrivals of k_rzb_final's (ROI, set) units
  rz_u64 cap;
  int nsets;
  __device__ void init(unsigned* base, rz_u64 cap_, int nsets_) {
    cap = cap_;
    nsets = nsets_;
    key = (rz_u64*)base;
    cnt = (unsigned*)(key + cap * nsets);
    red = (rz_u64*)(cnt + cap * nsets);
    ctr = (unsigned*)(red + (rz_u64)RZ_NV * nsets);
  }
  // table of a key's set (the zones are the last table)
  __device__ int tix(rz_u64 k) const { return min((int)(k >> 48), nsets - 1); }
  __device__ void add(rz_u64 k, unsigned c, unsigned* err) const {
    const rz_u64 off = (rz_u64)tix(k) * cap;
    rz_u64* kk = key + off;
    unsigned* cc = cnt + off;
    rz_u64 h = ((k * 0x9E3779B97F4A7C15ull) >> 20) & (cap - 1);
    for (rz_u64 probe = 0; probe < cap; ++probe) {
      rz_u64 cur = __ldcg(kk + h);
      if (cur == 0) {
        cur = atomicCAS(kk + h, 0ull, k);
        if (cur == 0) cur = k;
      }
      if (cur == k) {
        atomicAdd(cc + h, c);
        return;
      }
      h = (h + 1) & (cap - 1);
    }
    atomicOr(err, E_TOO_LARGE);
  }
};

// one item into the unit's shared table (a few probes), else straight into
// the ROI's global one
__device__ inline void rz_item(rz_u64* skey, unsigned* scnt, const RzTab& g, rz_u64 k, unsigned n, unsigned* err) {
  unsigned h = (unsigned)((k * 0x9E3779B97F4A7C15ull) >> 40) & (unsigned)(RZ_BIG_SH - 1);
  for (int probe = 0; probe < 32; ++probe) {
    rz_u64 cur = ((volatile rz_u64*)skey)[h];
    if (cur == 0) {
      cur = atomicCAS(skey + h, 0ull, k);
      if (cur == 0) cur = k;
    }
    if (cur == k) {
      atomicAdd(scnt + h, n);
      return;
    }
    h = (h + 1) & (unsigned)(RZ_BIG_SH - 1);
  }
  g.add(k, n, err);
}

// warp-aggregated version: every lane of the warp calls it with its key (0:
// none), and lanes with equal keys add their items once, through the lowest
// of them (in smooth images many runs share a key and would serialise on one
// shared-memory counter)
__device__ inline void rz_item_warp(rz_u64* skey, unsigned* scnt, const RzTab& g, rz_u64 k, unsigned* err) {
  if (!__any_sync(0xFFFFFFFFu, k != 0)) return;
  const unsigned peers = __match_any_sync(0xFFFFFFFFu, k);
  if (k && (peers & lanemask_lt()) == 0) rz_item(skey, scnt, g, k, (unsigned)__popc(peers), err);
}

// ---- union-find ---------------------------------------------------------------
// Links always go from the larger root index to the smaller, so parents only
// decrease along a path and every path ends.  Path halving stores an
// ancestor over a non-root's parent; a root changes only by compare-and-swap.

// 16-bit compare-and-swap through the aligned 32-bit word that holds it
__device__ inline bool rz_cas16(uint16_t* a16, unsigned expect, unsigned val) {
  unsigned* w = (unsigned*)((uintptr_t)a16 & ~(uintptr_t)3);
  const int sh = ((uintptr_t)a16 & 2) ? 16 : 0;
  unsigned old = *(volatile unsigned*)w;
  for (int it = 0; it < RZ_SPIN; ++it) {
    if (((old >> sh) & 0xFFFFu) != expect) return false;
    const unsigned nw = (old & ~(0xFFFFu << sh)) | (val << sh);
    const unsigned got = atomicCAS(w, old, nw);
    if (got == old) return true;
    old = got;
  }
  return false;
}

__device__ inline int rz_find(uint16_t* par, int x) {
  volatile uint16_t* vp = par;
  for (int it = 0; it < RZ_SPIN; ++it) {
    const int px = vp[x];
    if (px == x) return x;
    const int g = vp[px];
    if (g != px) vp[x] = (uint16_t)g;
    x = g;
  }
  return x;
}

__device__ inline void rz_union(uint16_t* par, int a, int b, unsigned* err) {
  for (int it = 0; it < RZ_SPIN; ++it) {
    a = rz_find(par, a);
    b = rz_find(par, b);
    if (a == b) return;
    if (a < b) {
      const int t = a;
      a = b;
      b = t;
    }
    if (rz_cas16(par + a, (unsigned)a, (unsigned)b)) return;
  }
  atomicOr(err, E_TIMEOUT);
}

// global version on 32-bit parents indexed by image pixel, stored as
// parent + 1 with 0 for a root, so that a memset starts every pixel as its
// own zone
__device__ inline unsigned rzg_find(unsigned* par, unsigned x, unsigned* err) {
  for (int it = 0; it < RZ_SPIN; ++it) {
    const unsigned v = __ldcg(par + x);
    if (v == 0) return x;
    const unsigned px = v - 1, g = __ldcg(par + px);
    if (g != 0) __stcg(par + x, g);  // halving; a root's slot is written only by the compare-and-swap
    x = px;
  }
  atomicOr(err, E_TIMEOUT);
  return x;
}

__device__ inline void rzg_union(unsigned* par, unsigned a, unsigned b, unsigned* err) {
  for (int it = 0; it < RZ_SPIN; ++it) {
    a = rzg_find(par, a, err);
    b = rzg_find(par, b, err);
    if (a == b) return;
    if (a < b) {
      const unsigned t = a;
      a = b;
      b = t;
    }
    if (atomicCAS(par + a, 0u, b + 1u) == 0u) return;
  }
  atomicOr(err, E_TIMEOUT);
}

// ---- block path ------------------------------------------------------------
// Dynamic shared memory: level raster (u16, CELLS), union-find parents (u16,
// CELLS), the joint hash (HC keys, HC counts), whose words hold the zone
// areas (two 16-bit counters a word) while the zones are counted, then the
// list of occupied hash slots (u16, HC / 2).
template <class Z>
constexpr int rz_smem_bytes() {
  return 4 * Z::CELLS + 8 * Z::HC + 2 * (Z::HC / 2);
}

// Set k's reduced values land in red[k] (GLRLM directions 0..ND-1, zones
// ND); once every set is reduced, threads 0..ND take one set's features
// each, and the GLRLM columns are the means over the directions, summed in
// direction order.
template <class T, int NDIM, class Z>
__global__ void __launch_bounds__(Z::NT) k_rz(KParams p, int tier) {
  static_assert(Z::CELLS <= 65536, "16-bit raster indices");
  static_assert(8 * Z::HC >= 2 * Z::CELLS, "zone areas (16 bits a cell) fit in the joint hash words");
  constexpr int ND = NDIM == 3 ? 13 : 4;
  extern __shared__ __align__(16) unsigned char rz_smem[];
  uint16_t* rast = (uint16_t*)rz_smem;
  uint16_t* par = rast + Z::CELLS;
  unsigned* hkey = (unsigned*)(par + Z::CELLS);
  unsigned* hcnt = hkey + Z::HC;
  unsigned* zw = hkey;
  uint16_t* slst = (uint16_t*)(hcnt + Z::HC);  // occupied joint-hash slots of the current set
  __shared__ unsigned lvl_n[256];
  __shared__ rz_u64 lvl_a[256];
  __shared__ unsigned hs_key[Z::HS], hs_cnt[Z::HS];
  __shared__ rz_u64 red[ND + 1][RZ_NV];
  __shared__ double sf[ND + 1][18];
  __shared__ int s_dv[13];
  __shared__ unsigned s_adj[13];
  __shared__ int s_item;
  __shared__ RoiInfo s_r;
  const int tid = threadIdx.x;
  const bool do_rl = (p.need & NEED_GLRLM) != 0, do_sz = (p.need & NEED_GLSZM) != 0;
  const int cl = tier;  // the size class whose queue this tier drains
  const T* img = (const T*)p.img;
  if (tid < ND) s_adj[tid] = rz_adj_mask(NDIM, tid);
  for (int i = tid; i < 256; i += Z::NT) {
    lvl_n[i] = 0;
    lvl_a[i] = 0;
  }
  for (int i = tid; i < Z::HS; i += Z::NT) {
    hs_key[i] = 0;
    hs_cnt[i] = 0;
  }
  for (int i = tid; i < Z::HC; i += Z::NT) {
    hkey[i] = 0;
    hcnt[i] = 0;
  }
  // the occupied cells of the joint hash, from the list of slots their
  // inserts claimed (a set has at most HC / 2 distinct keys, the hashes'
  // load bound): each is cleared and handed to f
  __shared__ unsigned s_nl;  // list length; 0 whenever a set starts (reset once every thread has read it)
  if (tid == 0) s_nl = 0;
  int hc = Z::HC;  // hash slots this ROI uses (set per ROI)
  auto joint = [&](auto f) {
    const unsigned nl = min(s_nl, (unsigned)(Z::HC / 2));
    for (unsigned i = tid; i < nl; i += Z::NT) {
      const unsigned h = slst[i];
      const unsigned k = hkey[h], c = hcnt[h];
      hkey[h] = 0;
      hcnt[h] = 0;
      f(k >> 16, (rz_u64)(k & 0xFFFFu), c);
    }
  };
  for (;;) {
    if (tid == 0) {
      const unsigned w = atomicAdd(p.rz_head + tier, 1u);
      const int it = w < p.qlen[cl] ? p.queue[(int64_t)cl * p.max_rois + w] : -1;
      s_item = it;
      if (it >= 0) s_r = p.rois[it];
    }
    for (int i = tid; i < (ND + 1) * RZ_NV; i += Z::NT) (&red[0][0])[i] = 0;
    __syncthreads();
    const int item = s_item;
    if (item < 0) break;
    const RoiInfo r = s_r;
    const int W = r.w, H = r.h, D = NDIM == 3 ? r.d : 1;
    const int Wp = W + 2, Hp = H + 2, Dp = NDIM == 3 ? D + 2 : 1;
    const int cells = Wp * Hp * Dp;
    if (cells > Z::CELLS || (int)r.n > Z::PIX) {  // excluded by the class limits
      if (tid == 0) atomicOr(p.err, E_INTERNAL);
      __syncthreads();
      continue;
    }
    if (tid < ND) {
      int dx, dy, dz;
      rz_dir(NDIM, tid, dx, dy, dz);
      s_dv[tid] = (dz * Hp + dy) * Wp + dx;
    }
    {  // hash slots: a power of two of at least twice the distinct keys a set
       // can have, min(n, sqrt(2 n Ng)), so small ROIs scan small tables
      const float kb = fminf((float)r.n, sqrtf(2.f * (float)r.n * (float)p.ng) + 1.f);
      hc = 64;
      while (hc < Z::HC && (float)hc < 2.f * kb) hc <<= 1;
    }
    RzLevel<T> lev;
    lev.init(r, p.ng);
    const int64_t per = p.nx * p.ny * p.nz;
    const int64_t org = (int64_t)(r.key >> 32) * per + ((int64_t)r.z0 * p.ny + r.y0) * p.nx + r.x0;
    const int label = (int)(r.key & 0xFFFFFFFFu);
    // level raster: 1..Ng on the ROI's cells, 0 elsewhere and on the border;
    // the loads of four cells are in flight together (every box cell is
    // inside the image)
    FastDiv fwp, fhp;
    fwp.init((unsigned)Wp);
    fhp.init((unsigned)Hp);
    for (int c0 = 0; c0 < cells; c0 += 4 * Z::NT) {
      int lab[4];
      T val[4];
      bool in[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int c = c0 + u * Z::NT + tid;
        const int yz = (int)fwp.div((unsigned)c), zq = (int)fhp.div((unsigned)yz);
        const int x = c - yz * Wp - 1, y = yz - zq * Hp - 1, z = NDIM == 3 ? zq - 1 : 0;
        in[u] = c < cells && x >= 0 && y >= 0 && z >= 0 && x < W && y < H && z < D;
        lab[u] = 0;
        if (in[u]) {
          const int64_t off = org + ((int64_t)z * p.ny + y) * p.nx + x;
          lab[u] = __ldg(p.mask + off);
          val[u] = __ldg(img + off);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int c = c0 + u * Z::NT + tid;
        if (c < cells) rast[c] = (uint16_t)(in[u] && lab[u] == label ? lev(Enc<T>::enc(val[u])) : 0u);
      }
    }
    __syncthreads();
    // one set: its items are in the joint hash; two barriers
    auto reduce_set = [&](int set) {
      rz_u128 jv[3];
      rz_u64 ent;
      rz_joint_pass(joint, p, lvl_n, lvl_a, hs_key, hs_cnt, Z::HS, jv, ent);
      __syncthreads();
      if (tid == 0) s_nl = 0;  // every thread has read the list length
      rz_marg_pass<Z::NT>(p, lvl_n, lvl_a, hs_key, hs_cnt, Z::HS, jv, ent, red[set]);
    };
    if (do_rl) {
      for (int k = 0; k < ND; ++k) {
        const int dv = s_dv[k];
        for (int c = tid; c < cells; c += Z::NT) {
          const unsigned L = rast[c];
          if (!L || rast[c - dv] == L) continue;  // not a run start (the border stops every walk)
          unsigned len = 1;
          for (int q = c + dv; rast[q] == L; q += dv) ++len;
          rz_insert(hkey, hcnt, hc, (L << 16) | len, 1u, slst, &s_nl, Z::HC / 2, p.err);
        }
        __syncthreads();  // also: the previous set's marginal pass is done with lvl / hs
        reduce_set(k);
      }
    }
    if (do_sz) {
      __syncthreads();  // the last direction's marginal pass is done with the hash words
      for (int c = tid; c < cells; c += Z::NT) par[c] = (uint16_t)c;
      for (int i = tid; i < (cells + 1) / 2; i += Z::NT) zw[i] = 0;
      __syncthreads();
      for (int c = tid; c < cells; c += Z::NT) {
        const unsigned L = rast[c];
        if (!L) continue;
        unsigned same = 0;  // directions whose neighbour has this level
#pragma unroll 1
        for (int k = 0; k < ND; ++k) {
          const int n = c + s_dv[k];
          if (rast[n] != L) continue;
          if (!(s_adj[k] & same)) rz_union(par, c, n, p.err);  // else already joined through an adjacent one
          same |= 1u << k;
        }
      }
      __syncthreads();
      // each cell's root from a find (not from its parent slot: a concurrent
      // path-halving store may leave an intermediate ancestor there; roots
      // themselves are never overwritten)
      for (int c = tid; c < cells; c += Z::NT)
        if (rast[c]) {
          const unsigned rt = (unsigned)rz_find(par, c);
          atomicAdd(zw + (rt >> 1), 1u << (16 * (rt & 1)));  // areas <= 8,192: no carry between halves
        }
      __syncthreads();
      // mark the roots (levels take 9 bits) and park each root's area in its
      // parent slot (only a cell's own thread reads or writes its slot here)
      for (int c = tid; c < cells; c += Z::NT)
        if (rast[c] && par[c] == c) {
          rast[c] |= 0x8000;
          par[c] = (uint16_t)((zw[c >> 1] >> (16 * (c & 1))) & 0xFFFFu);
        }
      __syncthreads();
      for (int i = tid; i < Z::HC; i += Z::NT) {
        hkey[i] = 0;
        hcnt[i] = 0;
      }
      __syncthreads();
      for (int c = tid; c < cells; c += Z::NT)
        if (rast[c] & 0x8000)
          rz_insert(hkey, hcnt, hc, ((unsigned)(rast[c] & 0x1FF) << 16) | par[c], 1u, slst, &s_nl, Z::HC / 2,
                    p.err);
      __syncthreads();
      reduce_set(ND);
    }
    __syncthreads();  // every set reduced
    if (tid <= ND && ((tid < ND && do_rl) || (tid == ND && do_sz)))
      rz_features(red[tid], r.n, tid < ND ? 16 : 18, sf[tid], false);
    __syncthreads();
    for (int q = tid; q < 34; q += Z::NT) {  // 16 GLRLM columns, then 18 GLSZM
      double v;
      int col;
      if (q < 16) {
        if (!do_rl) continue;
        v = 0;
        for (int k = 0; k < ND; ++k) v += sf[k][q];
        v *= 1.0 / ND;
        col = p.col_map[Q_GLRLM + q];
      } else {
        if (!do_sz) continue;
        v = sf[ND][q - 16];
        col = p.col_map[Q_GLSZM + q - 16];
      }
      if (col >= 0) p.table[(int64_t)item * p.n_col + col] = v;
    }
    __syncthreads();  // every thread is done with s_item / s_r / red / sf
  }
}

// ---- multi-block path -------------------------------------------------------
// One pass unit (ROI, chunk) at a time per block; `visit(x, y, z, off, level)`
// for the chunk's ROI cells.  RzBig holds what the unit's kernels share.
template <class T, int NDIM>
struct RzBig {
  BigBox bx;
  RzLevel<T> lev;
  RzTab tab;
  unsigned c0, c1;
  int item;
  unsigned n, tag0;  // tag0: (multi-block ROI index + 1) << 9
  __device__ void init(const KParams& p, int b, int chunk) {
    tag0 = (unsigned)(b + 1) << 9;
    const BigRoi br = p.big[b];
    const RoiInfo r = p.rois[br.item];
    bx.init(p, r, NDIM);
    lev.init(r, p.ng);
    const BigLayout L = big_layout(p, br.nch, br.nsp, br.range, r.n);
    tab.init(p.arena + br.arena + L.rzh, rz_hcap(p, r.n), rz_sets(p));
    c0 = (unsigned)chunk * BIG_CHUNK;
    c1 = min(bx.cells, c0 + (unsigned)BIG_CHUNK);
    item = br.item;
    n = r.n;
  }
  // tag (ROI + 1) << 9 | level of box cell (x, y, z) from the tag array, 0
  // off every multi-block ROI (or off the box)
  __device__ unsigned tag_at(const KParams& p, int x, int y, int z) const {
    if (x < 0 || y < 0 || z < 0 || x >= bx.W || y >= bx.H || z >= bx.D) return 0u;
    return __ldg(p.ztag + bx.origin + ((int64_t)z * p.ny + y) * p.nx + x);
  }
  // level of box cell (x, y, z), 0 off the ROI (or off the box)
  __device__ unsigned level_at(const KParams& p, const T* img, int x, int y, int z) const {
    if (x < 0 || y < 0 || z < 0 || x >= bx.W || y >= bx.H || z >= bx.D) return 0u;
    const int64_t o = bx.origin + ((int64_t)z * p.ny + y) * p.nx + x;
    return __ldg(p.mask + o) == bx.label ? lev(Enc<T>::enc(__ldg(img + o))) : 0u;
  }
};

template <class T, int NDIM, class F>
__device__ inline void rz_units(const KParams& p, F unit) {
  const unsigned long long ctr = *p.big_ctr;
  const int n_big = big_count(ctr);
  const unsigned n_units = big_units1(ctr);
  for (unsigned u = blockIdx.x; u < n_units; u += gridDim.x) {
    const int b = big_of_unit(p, n_big, u);
    RzBig<T, NDIM> g;
    g.init(p, b, (int)(u - p.big[b].u1));
    unit(g);
  }
}

// the unit's shared items into the ROI's global table; leaves the shared one empty
__device__ inline void rz_flush(rz_u64* skey, unsigned* scnt, const RzTab& g, unsigned* err) {
  __syncthreads();
  for (int i = threadIdx.x; i < RZ_BIG_SH; i += BIG_NT) {
    const rz_u64 k = skey[i];
    if (!k) continue;
    g.add(k, scnt[i], err);
    skey[i] = 0;
    scnt[i] = 0;
  }
  __syncthreads();
}

// the tag array: (multi-block ROI index + 1) << 9 | level of every pixel of
// a multi-block ROI (the array is cleared before), so that the items kernel
// compares one word per neighbour
template <class T, int NDIM>
__global__ void __launch_bounds__(BIG_NT) k_rzb_tags(KParams p) {
  const int tid = threadIdx.x;
  const T* img = (const T*)p.img;
  rz_units<T, NDIM>(p, [&](const RzBig<T, NDIM>& g) {
    if (g.c0 == 0) {  // the ROI's first unit clears its item tables, values and counter
      uint4* zr = (uint4*)g.tab.key;
      const unsigned long long n4 = rz_words(p, g.n) / 4;
      for (unsigned long long i = tid; i < n4; i += BIG_NT) zr[i] = make_uint4(0, 0, 0, 0);
    }
    for (unsigned c = g.c0 + tid; c < g.c1; c += BIG_NT) {
      int x, y, z;
      const int64_t off = g.bx.offset(c, x, y, z, p);
      if (__ldg(p.mask + off) == g.bx.label) p.ztag[off] = g.tag0 | g.lev(Enc<T>::enc(__ldg(img + off)));
    }
  });
}

// runs (GLRLM) and zone links (GLSZM) of the unit's cells: a run starts where
// the predecessor along its direction is not of its level and is walked to its
// end; a cell is linked to every forward neighbour of its level (the walk's
// first step reads the same neighbour).  Every lookup reads the image and the
// mask (L2-resident for all but the largest inputs).
template <class T, int NDIM>
__global__ void __launch_bounds__(BIG_NT) k_rzb_items(KParams p) {
  extern __shared__ __align__(16) unsigned char rz_smem[];
  rz_u64* skey = (rz_u64*)rz_smem;
  unsigned* scnt = (unsigned*)(skey + RZ_BIG_SH);
  __shared__ int s_d[13][3];
  __shared__ unsigned s_adj[13];
  constexpr int ND = NDIM == 3 ? 13 : 4;
  const int tid = threadIdx.x;
  const bool do_rl = (p.need & NEED_GLRLM) != 0, do_sz = (p.need & NEED_GLSZM) != 0;
  if (tid < ND) {
    rz_dir(NDIM, tid, s_d[tid][0], s_d[tid][1], s_d[tid][2]);
    s_adj[tid] = rz_adj_mask(NDIM, tid);
  }
  for (int i = tid; i < RZ_BIG_SH; i += BIG_NT) {
    skey[i] = 0;
    scnt[i] = 0;
  }
  __syncthreads();
  rz_units<T, NDIM>(p, [&](const RzBig<T, NDIM>& g) {
    for (unsigned cb = g.c0; cb < g.c1; cb += BIG_NT) {  // whole warps, for the aggregated inserts
      const unsigned c = cb + tid;
      int x = 0, y = 0, z = 0;
      int64_t off = 0;
      unsigned tg = 0;
      if (c < g.c1) {
        off = g.bx.offset(c, x, y, z, p);
        tg = __ldg(p.ztag + off);
        if ((tg & ~511u) != g.tag0) tg = 0;  // not this ROI's pixel
      }
      const unsigned L = tg & 511u;
      unsigned same = 0;  // directions whose neighbour has this level
#pragma unroll 1
      for (int k = 0; k < ND; ++k) {
        const int dx = s_d[k][0], dy = s_d[k][1], dz = s_d[k][2];
        rz_u64 key = 0;
        if (tg) {
          const bool next = g.tag_at(p, x + dx, y + dy, z + dz) == tg;
          if (do_sz && next && !(s_adj[k] & same))  // else already joined through an adjacent neighbour
            rzg_union(p.zpar, (unsigned)off, (unsigned)(off + ((int64_t)dz * p.ny + dy) * p.nx + dx), p.err);
          if (next) same |= 1u << k;
          if (do_rl && g.tag_at(p, x - dx, y - dy, z - dz) != tg) {  // a run start
            unsigned len = 1;
            if (next) {
              len = 2;
              while (g.tag_at(p, x + (int)len * dx, y + (int)len * dy, z + (int)len * dz) == tg) ++len;
            }
            key = ((rz_u64)k << 48) | ((rz_u64)L << 32) | len;
          }
        }
        rz_item_warp(skey, scnt, g.tab, key, p.err);
      }
    }
    rz_flush(skey, scnt, g.tab, p.err);
  });
}

// zone areas counted at the roots, every pixel's parent compressed to its root
template <class T, int NDIM>
__global__ void __launch_bounds__(BIG_NT) k_rzb_count(KParams p) {
  const int tid = threadIdx.x;
  rz_units<T, NDIM>(p, [&](const RzBig<T, NDIM>& g) {
    for (unsigned c = g.c0 + tid; c < g.c1; c += BIG_NT) {
      int x, y, z;
      const int64_t off = g.bx.offset(c, x, y, z, p);
      if (__ldg(p.mask + off) != g.bx.label) continue;
      const unsigned rt = rzg_find(p.zpar, (unsigned)off, p.err);
      if (rt != (unsigned)off) __stcg(p.zpar + off, rt + 1u);
      atomicAdd(p.zcnt + rt, 1u);
    }
  });
}

// one item (level, area) per zone, reported by its root
template <class T, int NDIM>
__global__ void __launch_bounds__(BIG_NT) k_rzb_zones(KParams p) {
  extern __shared__ __align__(16) unsigned char rz_smem[];
  rz_u64* skey = (rz_u64*)rz_smem;
  unsigned* scnt = (unsigned*)(skey + RZ_BIG_SH);
  constexpr int ND = NDIM == 3 ? 13 : 4;
  const int tid = threadIdx.x;
  for (int i = tid; i < RZ_BIG_SH; i += BIG_NT) {
    skey[i] = 0;
    scnt[i] = 0;
  }
  __syncthreads();
  rz_units<T, NDIM>(p, [&](const RzBig<T, NDIM>& g) {
    for (unsigned cb = g.c0; cb < g.c1; cb += BIG_NT) {
      const unsigned c = cb + tid;
      rz_u64 key = 0;
      if (c < g.c1) {
        int x, y, z;
        const int64_t off = g.bx.offset(c, x, y, z, p);
        const unsigned tg = __ldg(p.ztag + off);
        if ((tg & ~511u) == g.tag0 && __ldcg(p.zpar + off) == 0u)  // a root of this ROI
          key = ((rz_u64)ND << 48) | ((rz_u64)(tg & 511u) << 32) | __ldcg(p.zcnt + off);
      }
      rz_item_warp(skey, scnt, g.tab, key, p.err);
    }
    rz_flush(skey, scnt, g.tab, p.err);
  });
}

// units (multi-block ROI, set): each set's table reduced to its RZ_NV values
// (kept in the ROI's arena region); the last unit of an ROI to finish
// computes every set's features and writes the columns
template <class T, int NDIM>
__global__ void __launch_bounds__(BIG_NT) k_rzb_final(KParams p) {
  extern __shared__ __align__(16) unsigned char rz_smem[];
  unsigned* hs_key = (unsigned*)rz_smem;
  unsigned* hs_cnt = hs_key + RZ_BIG_HS;
  __shared__ unsigned lvl_n[256];
  __shared__ rz_u64 lvl_a[256];
  __shared__ rz_u64 red[RZ_NV];
  __shared__ double sf[14][18];
  __shared__ int s_flag;
  constexpr int ND = NDIM == 3 ? 13 : 4;
  const int tid = threadIdx.x;
  const bool do_rl = (p.need & NEED_GLRLM) != 0, do_sz = (p.need & NEED_GLSZM) != 0;
  const int nsets = rz_sets(p);
  for (int i = tid; i < 256; i += BIG_NT) {
    lvl_n[i] = 0;
    lvl_a[i] = 0;
  }
  for (int i = tid; i < RZ_BIG_HS; i += BIG_NT) {
    hs_key[i] = 0;
    hs_cnt[i] = 0;
  }
  const int n_big = big_count(*p.big_ctr);
  for (int u = blockIdx.x; u < n_big * nsets; u += gridDim.x) {
    const int b = u / nsets, t = u - b * nsets;  // t: table index (directions, then the zones)
    const BigRoi br = p.big[b];
    const RoiInfo r = p.rois[br.item];
    const BigLayout L = big_layout(p, br.nch, br.nsp, br.range, r.n);
    unsigned* reg = p.arena + br.arena;
    RzTab tab;
    tab.init(reg + L.rzh, rz_hcap(p, r.n), nsets);
    const rz_u64* kk = tab.key + (rz_u64)t * tab.cap;
    const unsigned* cc = tab.cnt + (rz_u64)t * tab.cap;
    if (tid < RZ_NV) red[tid] = 0;
    __syncthreads();
    auto joint = [&](auto f) {
      for (rz_u64 h = tid; h < tab.cap; h += BIG_NT) {
        const rz_u64 k = __ldcg(kk + h);
        if (k) f((unsigned)((k >> 32) & 0xFFFFu), k & 0xFFFFFFFFull, __ldcg(cc + h));
      }
    };
    rz_u128 jv[3];
    rz_u64 ent;
    rz_joint_pass(joint, p, lvl_n, lvl_a, hs_key, hs_cnt, RZ_BIG_HS, jv, ent);
    __syncthreads();
    rz_marg_pass<BIG_NT>(p, lvl_n, lvl_a, hs_key, hs_cnt, RZ_BIG_HS, jv, ent, red);
    __syncthreads();
    if (tid < RZ_NV) __stcg(tab.red + (rz_u64)t * RZ_NV + tid, red[tid]);
    if (!last_arrival(tab.ctr, (unsigned)nsets, &s_flag)) continue;
    // every set of this ROI is reduced: features, one thread per set
    if (tid < nsets) {
      rz_u64 v[RZ_NV];
      for (int i = 0; i < RZ_NV; ++i) v[i] = __ldcg(tab.red + (rz_u64)tid * RZ_NV + i);
      const bool zone = do_sz && tid == nsets - 1;
      rz_features(v, r.n, zone ? 18 : 16, sf[tid], false);
    }
    __syncthreads();
    double* row = p.table + (int64_t)br.item * p.n_col;
    if (do_rl && tid < 16) {
      double m = 0;
      for (int k = 0; k < ND; ++k) m += sf[k][tid];
      const int col = p.col_map[Q_GLRLM + tid];
      if (col >= 0) row[col] = m * (1.0 / ND);
    }
    if (do_sz && tid >= 32 && tid < 32 + 18) {
      const int col = p.col_map[Q_GLSZM + tid - 32];
      if (col >= 0) row[col] = sf[nsets - 1][tid - 32];
    }
    __syncthreads();
  }
}

// ---- launchers ---------------------------------------------------------------
template <auto K>
static cudaError_t rz_launch(int nt, int smem, int nsm, const KParams& p, cudaStream_t st, int arg = -1) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  static int configured[64] = {0};
  if (smem > 0 && (dev >= 64 || configured[dev] < smem)) {  // dynamic + static above 48 KB needs the opt-in
    e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    if (dev < 64) configured[dev] = smem;
  }
  int nb = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, K, nt, smem);
  if (e != cudaSuccess) return e;
  if (nb < 1) return cudaErrorInvalidConfiguration;
  if constexpr (std::is_invocable_v<decltype(K), KParams, int>) K<<<nb * nsm, nt, smem, st>>>(p, arg);
  else K<<<nb * nsm, nt, smem, st>>>(p);
  return cudaGetLastError();
}

// block path: both tiers, on one stream
template <class T, int NDIM>
cudaError_t launch_rz_blocks_one(const KParams& p, int nsm, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  if (p.lim_pix[0] > 0 && (e = rz_launch<k_rz<T, NDIM, RzT0>>(RzT0::NT, rz_smem_bytes<RzT0>(), nsm, p, st, 0)))
    return e;
  if (p.lim_pix[1] > 0 && (e = rz_launch<k_rz<T, NDIM, RzT1>>(RzT1::NT, rz_smem_bytes<RzT1>(), nsm, p, st, 1)))
    return e;
  if (p.lim_pix[2] > 0 && (e = rz_launch<k_rz<T, NDIM, RzT2>>(RzT2::NT, rz_smem_bytes<RzT2>(), nsm, p, st, 2)))
    return e;
  if (p.lim_pix[3] > 0) e = rz_launch<k_rz<T, NDIM, RzT3>>(RzT3::NT, rz_smem_bytes<RzT3>(), nsm, p, st, 3);
  return e;
}

// multi-block path (self-contained: it clears its own arena regions, so it
// runs beside the multi-block feature kernels)
template <class T, int NDIM>
cudaError_t launch_rz_big_one(const KParams& p, int nsm, cudaStream_t st) {
  const int sh = RZ_BIG_SH * 12;
  cudaError_t e = cudaSuccess;
  {  // tags 0, every pixel its own zone (parent 0), areas 0: one clear
    const unsigned long long px = (unsigned long long)p.batch * p.nx * p.ny * p.nz;
    if ((e = cudaMemsetAsync(p.ztag, 0, ((p.need & NEED_GLSZM) ? 12ull : 4ull) * px, st)) != cudaSuccess) return e;
  }
  if ((e = rz_launch<k_rzb_tags<T, NDIM>>(BIG_NT, 0, nsm, p, st)) != cudaSuccess) return e;
  if ((e = rz_launch<k_rzb_items<T, NDIM>>(BIG_NT, sh, nsm, p, st)) != cudaSuccess) return e;
  if (p.need & NEED_GLSZM) {
    if ((e = rz_launch<k_rzb_count<T, NDIM>>(BIG_NT, 0, nsm, p, st)) != cudaSuccess) return e;
    if ((e = rz_launch<k_rzb_zones<T, NDIM>>(BIG_NT, sh, nsm, p, st)) != cudaSuccess) return e;
  }
  return rz_launch<k_rzb_final<T, NDIM>>(BIG_NT, RZ_BIG_HS * 8, nsm, p, st);
}

template <class T>
cudaError_t launch_rz_t(const KParams& p, int big, int nsm, cudaStream_t st) {
  if (!(p.need & (NEED_GLRLM | NEED_GLSZM))) return cudaSuccess;
  if (p.ndim == 3) return big ? launch_rz_big_one<T, 3>(p, nsm, st) : launch_rz_blocks_one<T, 3>(p, nsm, st);
  return big ? launch_rz_big_one<T, 2>(p, nsm, st) : launch_rz_blocks_one<T, 2>(p, nsm, st);
}

}  // namespace nyx
