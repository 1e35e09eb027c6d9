// nyx_scan.cu -- label scan: ROI separation of the image + label mask.
//
// Paper: "Nyxus architecture" -- features are computed on an internal ROI
// layout (per-ROI pixel sets) separated from the image and mask; Table S2
// rows 41, 44-49 (area, bounding box, centroid) fall out of the separation.
//
// One streaming pass over image and mask (each byte read once) finds every
// distinct (image, label > 0) pair and accumulates its pixel count, bounding
// box and intensity range, plus the intensity range of every image.
// Aggregation is hierarchical so that few atomics reach global memory:
//   lane    : a register accumulator for the open label of its 4-column
//             strip, carried down the warp's rows
//   warp    : lanes holding the same label merge with match/reduce intrinsics
//   block   : a shared-memory hash table per 32 x 128 tile
//   global  : one insert + field atomics per (tile, label)
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdio>
#include <cstring>

#include "nyx_internal.cuh"

namespace nyx {

namespace {

constexpr int TX = 128;   // tile columns (32 lanes x 4 pixels)
constexpr int SCAN_RPT = 32; // tallest tile: rows per warp
// resident blocks per SM the register budget is set for (4-byte pixels need
// more registers for the rows in flight)
template <class T> constexpr int scan_minb() { return sizeof(T) == 4 ? 3 : 4; }
constexpr int SCAP = 256; // shared table capacity (labels per tile)
constexpr int SCAN_NT = 256;

__device__ inline void acc_identity(SlotAcc& a) {
  a.count = 0;
  a.vmin = 0xFFFFFFFFu;
  a.vmax = 0;
  a.xmin = a.ymin = a.zmin = 0x7FFFFFFF;
  a.xmax = a.ymax = a.zmax = (int)0x80000000;
}

// Insert-or-find in the global label table; records new slots in slot_list.
// Every table holds at least twice the labels its caller accepts, so once
// more than half of the slots are taken the call ends in a capacity error
// whatever happens next: give up at once instead of probing a nearly full
// table slot by slot.
__device__ int g_find_insert(const KParams& p, unsigned long long key) {
  if (*(volatile unsigned*)p.n_used > (p.hmask >> 1) + 1u) return -1;
  unsigned h = (unsigned)mix64(key) & p.hmask;
  for (unsigned i = 0; i <= p.hmask; ++i) {
    unsigned long long k = p.keys[h];
    if (k == key) return (int)h;
    if (k == EMPTY_KEY) {
      unsigned long long old = atomicCAS(&p.keys[h], EMPTY_KEY, key);
      if (old == EMPTY_KEY) {
        unsigned pos = atomicAdd(p.n_used, 1u);
        p.slot_list[pos] = (int)h;
        return (int)h;
      }
      if (old == key) return (int)h;
    }
    h = (h + 1) & p.hmask;
  }
  return -1;
}

__device__ int s_find_insert(unsigned long long* s_key, unsigned long long key) {
  unsigned h = (unsigned)mix64(key) & (SCAP - 1);
  for (int i = 0; i < SCAP; ++i) {
    unsigned long long k = *(volatile unsigned long long*)&s_key[h];
    if (k == key) return (int)h;
    if (k == EMPTY_KEY) {
      unsigned long long old = atomicCAS(&s_key[h], EMPTY_KEY, key);
      if (old == EMPTY_KEY || old == key) return (int)h;
    }
    h = (h + 1) & (SCAP - 1);
  }
  return -1;
}

// Merge a tile-table accumulator into a global one.
__device__ inline void acc_merge_acc(SlotAcc* a, const SlotAcc& s) {
  atomicAdd(&a->count, s.count);
  atomicMin(&a->vmin, s.vmin);
  atomicMax(&a->vmax, s.vmax);
  atomicMin(&a->xmin, s.xmin);
  atomicMax(&a->xmax, s.xmax);
  atomicMin(&a->ymin, s.ymin);
  atomicMax(&a->ymax, s.ymax);
  atomicMin(&a->zmin, s.zmin);
  atomicMax(&a->zmax, s.zmax);
}

template <class T> struct Vec4;
template <> struct Vec4<uint16_t> { using V = uint2; };
template <> struct Vec4<int16_t> { using V = uint2; };
template <> struct Vec4<float> { using V = uint4; };

template <class T> __device__ inline void unpack4(uint2 v, unsigned ev[4]) {
  ev[0] = Enc<T>::enc((T)(v.x & 0xFFFFu));
  ev[1] = Enc<T>::enc((T)(v.x >> 16));
  ev[2] = Enc<T>::enc((T)(v.y & 0xFFFFu));
  ev[3] = Enc<T>::enc((T)(v.y >> 16));
}
template <class T> __device__ inline void unpack4(uint4 v, unsigned ev[4]) {
  ev[0] = Enc<T>::enc(__uint_as_float(v.x));
  ev[1] = Enc<T>::enc(__uint_as_float(v.y));
  ev[2] = Enc<T>::enc(__uint_as_float(v.z));
  ev[3] = Enc<T>::enc(__uint_as_float(v.w));
}

// Raw 4-pixel image word: two 32-bit words of 16-bit pixels, four of floats.
template <class T>
__device__ inline void load_raw(const KParams& p, int64_t base, int64_t xs, int nvalid, int4& m,
                                typename Vec4<T>::V& v) {
  const T* img = (const T*)p.img;
  if (p.vec && nvalid == 4) {
    m = __ldg((const int4*)(p.mask + base + xs));
    v = __ldg((const typename Vec4<T>::V*)(img + base + xs));
  } else {
    int l[4];
    unsigned w[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      l[j] = j < nvalid ? p.mask[base + xs + j] : 0;
      w[j] = 0;
      if (j < nvalid) {
        if constexpr (sizeof(T) == 2) w[j] = (unsigned)(uint16_t)img[base + xs + j];
        else w[j] = __float_as_uint((float)img[base + xs + j]);
      }
    }
    m = make_int4(l[0], l[1], l[2], l[3]);
    if constexpr (sizeof(T) == 2) v = make_uint2(w[0] | w[1] << 16, w[2] | w[3] << 16);
    else v = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

template <class T> __device__ inline bool finite_enc(unsigned) { return true; }
template <> __device__ inline bool finite_enc<float>(unsigned e) { return isfinite(Enc<float>::decf(e)); }

}  // namespace

namespace {

// One open label of a lane: the pixels of its 4-column strip seen so far in
// the current tile and plane.
struct Slot {
  int lab;  // 0: empty
  unsigned cnt, vmn, vmx;
  unsigned xb;  // which of the lane's 4 columns the label covers
  int ymn, ymx;
};

// A slot is opened on a row where it receives pixels.
__device__ inline void slot_open(Slot& s, int lab, int y) {
  s.lab = lab;
  s.cnt = 0;
  s.vmn = 0xFFFFFFFFu;
  s.vmx = 0;
  s.xb = 0;
  s.ymn = s.ymx = y;
}

// Adds pixels j of one row (bit j of m) to the slot.
__device__ inline void slot_add(Slot& s, unsigned m, const unsigned ev[4], int y) {
  s.cnt += __popc(m);
  s.xb |= m;
  if (m) s.ymx = y;  // rows arrive in ascending y within a plane
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const bool in = m >> j & 1;
    s.vmn = min(s.vmn, in ? ev[j] : 0xFFFFFFFFu);
    s.vmx = max(s.vmx, in ? ev[j] : 0u);
  }
}

__device__ inline int slot_xmin(const Slot& s, int xs) { return s.xb ? xs + __ffs(s.xb) - 1 : 0x7FFFFFFF; }
__device__ inline int slot_xmax(const Slot& s, int xs) { return s.xb ? xs + 31 - __clz(s.xb) : (int)0x80000000; }

__device__ inline void acc_merge_run(SlotAcc* s, unsigned cnt, unsigned vmn, unsigned vmx, int xmn, int xmx, int ymn,
                                     int ymx, int z) {
  atomicAdd(&s->count, cnt);
  atomicMin(&s->vmin, vmn);
  atomicMax(&s->vmax, vmx);
  atomicMin(&s->xmin, xmn);
  atomicMax(&s->xmax, xmx);
  atomicMin(&s->ymin, ymn);
  atomicMax(&s->ymax, ymx);
  atomicMin(&s->zmin, z);
  atomicMax(&s->zmax, z);
}

// One label's pixels of one plane into the tile table (the global table when
// the tile holds more than SCAP labels).
__device__ void run_insert(const KParams& p, unsigned long long* s_key, SlotAcc* s_acc, int lab, long long b,
                           unsigned cnt, unsigned vmn, unsigned vmx, int xmn, int xmx, int ymn, int ymx, int z,
                           unsigned& errbits) {
  const unsigned long long k = ((unsigned long long)b << 32) | (unsigned)lab;
  const int s = s_find_insert(s_key, k);
  if (s >= 0) {
    acc_merge_run(&s_acc[s], cnt, vmn, vmx, xmn, xmx, ymn, ymx, z);
  } else {
    const int g = g_find_insert(p, k);
    if (g >= 0) acc_merge_run(&p.slots[g], cnt, vmn, vmx, xmn, xmx, ymn, ymx, z);
    else errbits |= E_HASH_FULL;
  }
}

__device__ inline void slot_insert(const KParams& p, unsigned long long* s_key, SlotAcc* s_acc, const Slot& s, int xs,
                                   int z, long long b, unsigned& errbits) {
  run_insert(p, s_key, s_acc, s.lab, b, s.cnt, s.vmn, s.vmx, slot_xmin(s, xs), slot_xmax(s, xs), s.ymn, s.ymx, z,
             errbits);
}

// Whole warp: lanes whose slot holds the same label merge it with
// match/reduce, and the lowest such lane inserts the result once.
__device__ inline void slot_flush_warp(const KParams& p, unsigned long long* s_key, SlotAcc* s_acc, Slot& s, int xs,
                                       int z, long long b, unsigned& errbits) {
  if (!__any_sync(0xFFFFFFFFu, s.lab > 0)) return;
  const unsigned peers = __match_any_sync(0xFFFFFFFFu, (unsigned)s.lab);
  const unsigned cnt = __reduce_add_sync(peers, s.cnt);
  const unsigned vmn = __reduce_min_sync(peers, s.vmn);
  const unsigned vmx = __reduce_max_sync(peers, s.vmx);
  const int xmn = __reduce_min_sync(peers, slot_xmin(s, xs));
  const int xmx = __reduce_max_sync(peers, slot_xmax(s, xs));
  const int ymn = __reduce_min_sync(peers, s.ymn);
  const int ymx = __reduce_max_sync(peers, s.ymx);
  if (s.lab > 0 && (peers & lanemask_lt()) == 0)
    run_insert(p, s_key, s_acc, s.lab, b, cnt, vmn, vmx, xmn, xmx, ymn, ymx, z, errbits);
  s.lab = 0;
}

template <class T> __device__ inline bool nonfinite_raw(const typename Vec4<T>::V&) { return false; }
template <> __device__ inline bool nonfinite_raw<float>(const uint4& v) {
  const unsigned E = 0x7F800000u;
  return ((v.x & E) == E) | ((v.y & E) == E) | ((v.z & E) == E) | ((v.w & E) == E);
}

// What a lane carries from row to row: its two open labels, the current
// image's intensity range and the error bits.
struct ScanLane {
  Slot A, B;
  unsigned im_mn, im_mx;
  int64_t im_b;
  unsigned errbits;
};

// One row of a lane's 4-column strip (mask words mc, image word vc, nvalid
// of the 4 columns inside the image) at plane position (y, z, b); next_row:
// this is not the warp's first row of the tile, so y advances first (and a
// finished plane is flushed).  Called by the whole warp.
template <class T>
__device__ __forceinline__ void scan_row(const KParams& p, unsigned long long* s_key, SlotAcc* s_acc, ScanLane& S,
                                         const int4 mc, const typename Vec4<T>::V vc, int nvalid, int xs, int lane,
                                         bool next_row, int& y, int& z, int64_t& b) {
  if (next_row && ++y == p.ny) {  // warp-uniform: a new plane (or image) starts
    slot_flush_warp(p, s_key, s_acc, S.A, xs, z, b, S.errbits);
    slot_flush_warp(p, s_key, s_acc, S.B, xs, z, b, S.errbits);
    y = 0;
    if (++z == p.nz) {
      z = 0;
      ++b;
    }
  }
  if (b != S.im_b) {  // warp-uniform: close the previous image's range
    unsigned mn = __reduce_min_sync(0xFFFFFFFFu, S.im_mn), mx = __reduce_max_sync(0xFFFFFFFFu, S.im_mx);
    if (lane == 0 && S.im_b >= 0) {
      atomicMin(&p.img_vmin[S.im_b], mn);
      atomicMax(&p.img_vmax[S.im_b], mx);
    }
    S.im_b = b;
    S.im_mn = 0xFFFFFFFFu;
    S.im_mx = 0;
  }
  int L[4] = {mc.x, mc.y, mc.z, mc.w};
  unsigned ev[4];
  unpack4<T>(vc, ev);
  bool uni;
  unsigned rmn, rmx;
  if (nvalid == 4) {
    rmn = min(min(ev[0], ev[1]), min(ev[2], ev[3]));
    rmx = max(max(ev[0], ev[1]), max(ev[2], ev[3]));
    uni = (L[0] == L[1]) & (L[1] == L[2]) & (L[2] == L[3]);
  } else {  // right edge of the image: pixels past it are background
    rmn = 0xFFFFFFFFu;
    rmx = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (j < nvalid) {
        rmn = min(rmn, ev[j]);
        rmx = max(rmx, ev[j]);
      } else {
        L[j] = 0;
      }
    }
    uni = false;
  }
  S.im_mn = min(S.im_mn, rmn);
  S.im_mx = max(S.im_mx, rmx);
  if ((L[0] | L[1] | L[2] | L[3]) < 0) S.errbits |= E_BAD_LABEL;
  if (nonfinite_raw<T>(vc)) {
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (L[j] > 0 && !finite_enc<T>(ev[j])) S.errbits |= E_NONFINITE;
  }
  if (uni && L[0] <= 0) return;  // background row segment
  if (uni && L[0] == S.A.lab) {
    S.A.cnt += 4;
    S.A.xb = 0xFu;
    S.A.vmn = min(S.A.vmn, rmn);
    S.A.vmx = max(S.A.vmx, rmx);
    S.A.ymx = y;
    return;
  }
  if (uni && L[0] == S.B.lab) {
    S.B.cnt += 4;
    S.B.xb = 0xFu;
    S.B.vmn = min(S.B.vmn, rmn);
    S.B.vmx = max(S.B.vmx, rmx);
    S.B.ymx = y;
    return;
  }
  unsigned mA = 0, mB = 0, mo = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j)
    if (L[j] > 0) {
      if (L[j] == S.A.lab) mA |= 1u << j;
      else if (L[j] == S.B.lab) mB |= 1u << j;
      else mo |= 1u << j;
    }
  while (mo) {  // a label in neither slot: give it a slot
    const int j = __ffs(mo) - 1;
    const int nl = j == 0 ? L[0] : j == 1 ? L[1] : j == 2 ? L[2] : L[3];
    // an empty slot, else one without pixels on this row, else B; the
    // displaced label keeps the pixels it has on this row
    const bool useA = S.A.lab == 0 || (S.B.lab != 0 && mA == 0);
    if (useA) {
      if (S.A.lab > 0) {
        slot_add(S.A, mA, ev, y);
        slot_insert(p, s_key, s_acc, S.A, xs, z, b, S.errbits);
      }
      slot_open(S.A, nl, y);
    } else {
      if (S.B.lab > 0) {
        slot_add(S.B, mB, ev, y);
        slot_insert(p, s_key, s_acc, S.B, xs, z, b, S.errbits);
      }
      slot_open(S.B, nl, y);
    }
    unsigned mn = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if ((mo >> q & 1) && L[q] == nl) mn |= 1u << q;
    mo &= ~mn;
    if (useA) mA = mn;
    else mB = mn;
  }
  slot_add(S.A, mA, ev, y);
  slot_add(S.B, mB, ev, y);
}

// Tile geometry of warp `warp` in tile t: first column of the lane's strip,
// columns of it inside the image, first row and rows (0 past the scan range).
struct ScanTile {
  int64_t xs64, rw0;
  int xs, nvalid, nr;
};
// a / d and its remainder, by 32-bit division when both operands fit
__device__ inline int64_t div_rem(int64_t a, int64_t d, int64_t& r) {
  if (((a | d) >> 31) == 0) {
    const unsigned q = (unsigned)a / (unsigned)d;
    r = a - (int64_t)q * d;
    return q;
  }
  const int64_t q = a / d;
  r = a - q * d;
  return q;
}

__device__ inline ScanTile scan_tile(const KParams& p, int64_t t, int64_t ntx, int64_t r0, int64_t r1, int rpt,
                                     int warp, int lane) {
  ScanTile g;
  int64_t tx;
  const int64_t ty = div_rem(t, ntx, tx);
  g.xs64 = tx * TX + 4 * lane;
  g.xs = (int)g.xs64;
  g.nvalid = (int)max((int64_t)0, min((int64_t)4, p.nx - g.xs64));
  g.rw0 = r0 + ty * (8ll * rpt) + (int64_t)warp * rpt;
  g.nr = (int)max((int64_t)0, min((int64_t)rpt, r1 - g.rw0));
  return g;
}

__device__ inline void scan_lane_init(ScanLane& S) {
  S.im_mn = 0xFFFFFFFFu;
  S.im_mx = 0;
  S.im_b = -1;
  S.errbits = 0;
  S.A.lab = S.B.lab = 0;
}

// End of a tile: the warp's open labels into the tile table, then the whole
// block moves the tile table into the global label table.
__device__ inline void scan_tile_end(const KParams& p, unsigned long long* s_key, SlotAcc* s_acc, ScanLane& S,
                                     int xs, int z, int64_t b) {
  slot_flush_warp(p, s_key, s_acc, S.A, xs, z, b, S.errbits);
  slot_flush_warp(p, s_key, s_acc, S.B, xs, z, b, S.errbits);
  __syncthreads();
  for (int i = threadIdx.x; i < SCAP; i += SCAN_NT) {
    unsigned long long k = s_key[i];
    if (k == EMPTY_KEY) continue;
    int g = g_find_insert(p, k);
    if (g >= 0) acc_merge_acc(&p.slots[g], s_acc[i]);
    else S.errbits |= E_HASH_FULL;
    s_key[i] = EMPTY_KEY;
    acc_identity(s_acc[i]);
  }
  __syncthreads();
}

// The warps' last image ranges and error bits out to global memory: the
// block merges its warps' ranges first, one update per distinct image (a
// warp-per-update scheme sends thousands of updates to the same address).
// Called by the whole block.
__device__ inline void scan_finish(const KParams& p, ScanLane& S, int lane) {
  constexpr int NW = SCAN_NT / 32;
  __shared__ long long s_fb[NW];
  __shared__ unsigned s_fmn[NW], s_fmx[NW];
  const int warp = threadIdx.x >> 5;
  const unsigned mn = __reduce_min_sync(0xFFFFFFFFu, S.im_mn), mx = __reduce_max_sync(0xFFFFFFFFu, S.im_mx);
  const bool any = __any_sync(0xFFFFFFFFu, S.im_b >= 0);
  const long long bb = __reduce_max_sync(0xFFFFFFFFu, (unsigned)(S.im_b + 1)) - 1;  // warp-uniform image index
  if (lane == 0) {
    s_fb[warp] = any ? bb : -1;
    s_fmn[warp] = mn;
    s_fmx[warp] = mx;
  }
  const unsigned e = __reduce_or_sync(0xFFFFFFFFu, S.errbits);
  if (lane == 0 && e) atomicOr(p.err, e);
  __syncthreads();
  if (threadIdx.x < NW) {
    const int w = threadIdx.x;
    const long long b = s_fb[w];
    if (b >= 0) {
      bool first = true;
      unsigned m0 = 0xFFFFFFFFu, m1 = 0;
      for (int v = 0; v < NW; ++v)
        if (s_fb[v] == b) {
          first &= v >= w;
          m0 = min(m0, s_fmn[v]);
          m1 = max(m1, s_fmx[v]);
        }
      if (first) {
        atomicMin(&p.img_vmin[b], m0);
        atomicMax(&p.img_vmax[b], m1);
      }
    }
  }
}

__device__ inline void scan_plane_pos(const KParams& p, int64_t row, int& y, int& z, int64_t& b) {
  int64_t yr, zr;
  const int64_t zb = div_rem(row, p.ny, yr);
  b = div_rem(zb, p.nz, zr);
  y = (int)yr;
  z = (int)zr;
}


// ---- bulk-copy (TMA) staging of the label scan -----------------------------
// Each warp streams its rows through a ring of TMA_NS shared-memory stages of
// TMA_SR rows x 128 columns of mask (int32) then image; one lane issues the
// 2D tensor copies, each stage completes on its own mbarrier.
constexpr int TMA_SR = 2;  // rows per stage
constexpr int TMA_NS = 3;  // stages per warp
template <class T> constexpr int tma_stage_bytes() { return TMA_SR * TX * (4 + (int)sizeof(T)); }
template <class T> constexpr int tma_smem_bytes() { return (SCAN_NT / 32) * TMA_NS * tma_stage_bytes<T>(); }
// resident blocks per SM the register budget is set for: what the staging
// ring leaves of the SM's shared memory
template <class T> constexpr int scan_tma_minb() { return sizeof(T) == 4 ? 3 : 4; }

__device__ inline unsigned smem_addr(const void* ptr) { return (unsigned)__cvta_generic_to_shared(ptr); }

__device__ inline void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// make barrier initialisation visible to the bulk-copy (async) proxy
__device__ inline void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ inline void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ inline bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred P;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, P;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ inline unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for the phase of `parity` to complete; false after about a second
// (the copy never landed: the caller reports E_TIMEOUT and stops).
__device__ inline bool mbar_wait(unsigned long long* bar, unsigned parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (int it = 0; it < (1 << 26); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255) == 255 && global_ns() - t0 > 1000000000ull) return false;
  }
  return false;
}

// 2D tiled tensor copy global -> shared of the box at element (x, y),
// completing `bar`'s transaction count
__device__ inline void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_addr(dst)),
      "l"((unsigned long long)map), "r"(x), "r"(y), "r"(smem_addr(bar))
      : "memory");
}

}  // namespace

// Each warp takes rpt consecutive rows of a 128-column tile (tile height
// 8 * rpt) and each lane a 4-pixel column strip of them.  Blob-shaped ROIs
// keep the labels in a strip the same from row to row, so a lane keeps two
// open labels (two, so that a strip on the border of two touching ROIs
// stays cheap) in registers: a row whose 4 pixels are background or one
// open label costs a few min/max operations, and the shared table is only
// touched when a third label displaces one.  At the end of the tile or of a
// plane the warp merges equal labels with match/reduce and inserts each
// once.  Loads run two rows ahead of the row being processed.
template <class T>
__global__ void __launch_bounds__(SCAN_NT, scan_minb<T>()) k_scan(KParams p, int rpt) {
  __shared__ unsigned long long s_key[SCAP];
  __shared__ SlotAcc s_acc[SCAP];
  for (int i = threadIdx.x; i < SCAP; i += SCAN_NT) {
    s_key[i] = EMPTY_KEY;
    acc_identity(s_acc[i]);
  }
  __syncthreads();
  using V = typename Vec4<T>::V;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t r0 = p.scan_row0, r1 = p.scan_row1 > 0 ? p.scan_row1 : p.rows_total;
  const int64_t ntx = (p.nx + TX - 1) / TX, nty = (r1 - r0 + 8ll * rpt - 1) / (8ll * rpt);
  const int64_t ntiles = ntx * nty;
  ScanLane S;
  scan_lane_init(S);
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const ScanTile g = scan_tile(p, t, ntx, r0, r1, rpt, warp, lane);
    int y = 0, z = 0;
    int64_t b = 0;
    int4 m0, m1;
    V v0, v1;
    if (g.nr > 0) {
      scan_plane_pos(p, g.rw0, y, z, b);
      load_raw<T>(p, g.rw0 * p.nx, g.xs64, g.nvalid, m0, v0);
    }
    if (g.nr > 1) load_raw<T>(p, (g.rw0 + 1) * p.nx, g.xs64, g.nvalid, m1, v1);
    for (int i = 0; i < g.nr; ++i) {
      const int4 mc = m0;
      const V vc = v0;
      m0 = m1;
      v0 = v1;
      if (i + 2 < g.nr) load_raw<T>(p, (g.rw0 + i + 2) * p.nx, g.xs64, g.nvalid, m1, v1);
      scan_row<T>(p, s_key, s_acc, S, mc, vc, g.nvalid, g.xs, lane, i > 0, y, z, b);
    }
    scan_tile_end(p, s_key, s_acc, S, g.xs, z, b);
  }
  scan_finish(p, S, lane);
}

// The same scan with its rows staged by bulk tensor copies (TMA) instead of
// register loads: each warp keeps TMA_NS stages of TMA_SR rows in flight
// (lane 0 issues the copies of the warp's own row sequence, continuing into
// its next tile), so the bytes in flight no longer cost registers; lanes read
// their 4-pixel strip from shared memory (16 B of mask + 8 or 16 B of image,
// consecutive across the warp).  Columns and rows past the image arrive as
// zeros (background).  Used when both tensor maps could be encoded.
template <class T>
__global__ void __launch_bounds__(SCAN_NT, scan_tma_minb<T>())
    k_scan_tma(const __grid_constant__ CUtensorMap tm_mask, const __grid_constant__ CUtensorMap tm_img, KParams p,
               int rpt) {
  __shared__ unsigned long long s_key[SCAP];
  __shared__ SlotAcc s_acc[SCAP];
  __shared__ unsigned long long s_bar[SCAN_NT / 32][TMA_NS];
  extern __shared__ __align__(128) unsigned char st_smem[];
  using V = typename Vec4<T>::V;
  constexpr unsigned STAGE_B = tma_stage_bytes<T>(), MASK_B = TMA_SR * TX * 4;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < SCAP; i += SCAN_NT) {
    s_key[i] = EMPTY_KEY;
    acc_identity(s_acc[i]);
  }
  if (lane == 0) {
    for (int q = 0; q < TMA_NS; ++q) mbar_init(&s_bar[warp][q], 1);
    mbar_init_fence();
  }
  __syncthreads();
  const int64_t r0 = p.scan_row0, r1 = p.scan_row1 > 0 ? p.scan_row1 : p.rows_total;
  const int64_t ntx = (p.nx + TX - 1) / TX, nty = (r1 - r0 + 8ll * rpt - 1) / (8ll * rpt);
  const int64_t ntiles = ntx * nty;
  unsigned char* wst = st_smem + (size_t)warp * TMA_NS * STAGE_B;
  // copy cursor (lane 0): tile and chunk of the next copy, copies issued
  int64_t pt = blockIdx.x;
  int pc = 0;
  unsigned pseq = 0;
  ScanTile pg = scan_tile(p, pt, ntx, r0, r1, rpt, warp, 0);  // of tile pt
  auto issue = [&]() {
    while (pt < ntiles) {
      if (pc * TMA_SR < pg.nr) {
        const unsigned q = pseq % TMA_NS;
        unsigned char* dst = wst + q * STAGE_B;
        const int x = (int)pg.xs64, y = (int)(pg.rw0 + (int64_t)pc * TMA_SR);
        mbar_arrive_expect_tx(&s_bar[warp][q], STAGE_B);
        tma_load_2d(dst, &tm_mask, x, y, &s_bar[warp][q]);
        tma_load_2d(dst + MASK_B, &tm_img, x, y, &s_bar[warp][q]);
        ++pc;
        ++pseq;
        return;
      }
      pt += gridDim.x;
      pc = 0;
      if (pt < ntiles) pg = scan_tile(p, pt, ntx, r0, r1, rpt, warp, 0);
    }
  };
  if (lane == 0)
    for (int q = 0; q < TMA_NS; ++q) issue();
  unsigned cseq = 0;     // chunk being read
  unsigned dead_at = 0;  // first chunk not waited for, once a wait ran out
  bool dead = false;     // warp-uniform
  ScanLane S;
  scan_lane_init(S);
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const ScanTile g = scan_tile(p, t, ntx, r0, r1, rpt, warp, lane);
    int y = 0, z = 0;
    int64_t b = 0;
    if (g.nr > 0) scan_plane_pos(p, g.rw0, y, z, b);
    for (int i = 0; i < g.nr; ++i) {
      const int sub = i % TMA_SR;
      if (sub == 0) {
        if (i > 0) {  // the previous chunk is read: its stage takes the next copy
          __syncwarp();
          if (lane == 0 && !dead) issue();
          ++cseq;
        }
        if (!dead) {
          const bool ok = mbar_wait(&s_bar[warp][cseq % TMA_NS], (cseq / TMA_NS) & 1u);
          dead = !__all_sync(0xFFFFFFFFu, ok);
          if (dead) {
            dead_at = cseq;
            S.errbits |= E_TIMEOUT;
          }
        }
      }
      if (dead) continue;
      const unsigned char* st = wst + (cseq % TMA_NS) * STAGE_B;
      const int4 mc = *(const int4*)(st + 4 * (sub * TX + 4 * lane));
      const V vc = *(const V*)(st + MASK_B + sizeof(T) * (sub * TX + 4 * lane));
      scan_row<T>(p, s_key, s_acc, S, mc, vc, g.nvalid, g.xs, lane, i > 0, y, z, b);
    }
    if (g.nr > 0) {
      __syncwarp();
      if (lane == 0 && !dead) issue();
      ++cseq;
    }
    scan_tile_end(p, s_key, s_acc, S, g.xs, z, b);
  }
  // a warp that gave up still lets its copies in flight land (bounded)
  if (dead && lane == 0)
    for (unsigned q = dead_at; q < pseq; ++q) mbar_wait(&s_bar[warp][q % TMA_NS], (q / TMA_NS) & 1u);
  scan_finish(p, S, lane);
}

// Sort the distinct keys ascending (one block): dense ROI id = rank of its
// (image, label) key.  Keys that differ only in their low 16 bits (one
// image, labels within a 65,536 range) are ranked through a presence bitmap;
// other key sets by an LSD radix sort of 16-bit indices by 8-bit digits over
// the digits that differ at all, with stable ranks from 8 ballots per digit.
// The keys are gathered once into sort_tmp.
__global__ void __launch_bounds__(1024) k_sort_keys(KParams p) {
  extern __shared__ unsigned s_sm[];
  constexpr int NW = 32;
  unsigned* cnt = s_sm;                     // [NW][256]
  unsigned* dtot = cnt + NW * 256;          // [256]
  uint16_t* ix0 = (uint16_t*)(dtot + 256);  // [2][max_rois]
  __shared__ unsigned long long s_or[NW];
  const unsigned n = *p.n_used;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (n > (unsigned)SORT_CAP || (int64_t)n > p.max_rois) {
    if (tid == 0) {
      atomicOr(p.err, n > (unsigned)SORT_CAP ? E_SORT_CAP : E_ROI_CAP);
      *p.n_roi = 0;
      if (p.n_roi_out) *p.n_roi_out = (int64_t)n;
    }
    return;
  }
  unsigned long long* kv = p.sort_tmp;
  uint16_t* src = ix0;
  uint16_t* dst = ix0 + p.max_rois;
  const unsigned long long k0 = n ? p.keys[p.slot_list[0]] : 0ull;
  unsigned long long diff = 0;
  for (unsigned i = tid; i < n; i += blockDim.x) {
    const unsigned long long k = p.keys[p.slot_list[i]];
    kv[i] = k;
    src[i] = (uint16_t)i;
    diff |= k ^ k0;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) diff |= __shfl_xor_sync(0xFFFFFFFFu, diff, o);
  if (lane == 0) s_or[warp] = diff;
  __syncthreads();
  diff = 0;
  for (int w = 0; w < NW; ++w) diff |= s_or[w];
  const int nbits = diff ? 64 - __clzll((long long)diff) : 0;
  if (nbits <= 16) {
    // Keys differ only in their low nbits bits (one image, labels within a
    // 65,536 range): the rank of a key is the number of keys below it, read
    // from a presence bitmap over that range and a prefix of its popcounts.
    const unsigned long long kb = k0 & ~((1ull << nbits) - 1ull);
    const int nwd = nbits > 5 ? 1 << (nbits - 5) : 1;  // bitmap words (<= 2048)
    unsigned* bm = cnt;           // [nwd] presence bits
    unsigned* pre = cnt + 2048;   // [nwd] exclusive prefix of popcounts
    for (int i = tid; i < nwd; i += blockDim.x) bm[i] = 0;
    __syncthreads();
    for (unsigned i = tid; i < n; i += blockDim.x) {
      const unsigned o = (unsigned)(kv[i] - kb);
      atomicOr(&bm[o >> 5], 1u << (o & 31));
    }
    __syncthreads();
    // block-wide exclusive scan, two words per thread
    const int w0 = 2 * tid;
    const unsigned c0 = w0 < nwd ? __popc(bm[w0]) : 0u, c1 = w0 + 1 < nwd ? __popc(bm[w0 + 1]) : 0u;
    unsigned x = c0 + c1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) dtot[warp] = x;
    __syncthreads();
    if (warp == 0) warp_exclusive_scan(dtot, NW);
    __syncthreads();
    const unsigned ex = dtot[warp] + x - (c0 + c1);
    if (w0 < nwd) pre[w0] = ex;
    if (w0 + 1 < nwd) pre[w0 + 1] = ex + c0;
    __syncthreads();
    for (unsigned i = tid; i < n; i += blockDim.x) {
      const unsigned long long k = kv[i];
      const unsigned o = (unsigned)(k - kb);
      p.sorted_keys[pre[o >> 5] + __popc(bm[o >> 5] & ((1u << (o & 31)) - 1u))] = k;
    }
    if (tid == 0) {
      *p.n_roi = n;
      if (p.n_roi_out) *p.n_roi_out = (int64_t)n;
      if ((int64_t)n > p.cap_roi) atomicOr(p.err, E_ROI_CAP);
    }
    return;
  }
  const int seg = (((int)(n + NW - 1) / NW) + 31) & ~31;
  const int lo = min((int)n, warp * seg), hi = min((int)n, lo + seg);
  for (int shift = 0; shift < nbits; shift += 8) {
    if (((diff >> shift) & 255ull) == 0) continue;  // a digit every key shares: no reordering
    for (int i = tid; i < NW * 256; i += blockDim.x) cnt[i] = 0;
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {  // 0: digit counts per warp, 1: stable scatter
      for (int i0 = lo; i0 < hi; i0 += 32) {
        const int i = i0 + lane;
        const bool act = i < hi;
        const unsigned id = act ? src[i] : 0u;
        const unsigned dg = act ? (unsigned)(kv[id] >> shift) & 255u : 0u;
        unsigned peers = __ballot_sync(0xFFFFFFFFu, act);
#pragma unroll
        for (int bit = 0; bit < 8; ++bit) {
          const unsigned bb = __ballot_sync(0xFFFFFFFFu, (dg >> bit) & 1u);
          peers &= ((dg >> bit) & 1u) ? bb : ~bb;
        }
        const unsigned before = __popc(peers & lanemask_lt());
        unsigned base = 0;
        if (act) base = cnt[warp * 256 + dg];
        __syncwarp();
        if (act) {
          if (pass) dst[base + before] = (uint16_t)id;
          if (before == 0) cnt[warp * 256 + dg] = base + __popc(peers);
        }
        __syncwarp();
      }
      __syncthreads();
      if (pass == 0) {  // digit-major, then warp, exclusive offsets
        for (int d = tid; d < 256; d += blockDim.x) {
          unsigned t = 0;
          for (int w = 0; w < NW; ++w) t += cnt[w * 256 + d];
          dtot[d] = t;
        }
        __syncthreads();
        if (warp == 0) warp_exclusive_scan(dtot, 256);
        __syncthreads();
        for (int d = tid; d < 256; d += blockDim.x) {
          unsigned run = dtot[d];
          for (int w = 0; w < NW; ++w) {
            const unsigned c = cnt[w * 256 + d];
            cnt[w * 256 + d] = run;
            run += c;
          }
        }
        __syncthreads();
      }
    }
    uint16_t* t = src;
    src = dst;
    dst = t;
  }
  for (unsigned i = tid; i < n; i += blockDim.x) p.sorted_keys[i] = kv[src[i]];
  if (tid == 0) {
    *p.n_roi = n;
    if (p.n_roi_out) *p.n_roi_out = (int64_t)n;
    if ((int64_t)n > p.cap_roi) atomicOr(p.err, E_ROI_CAP);
  }
}

// ---------------------------------------------------------------------------
// Multi-block key sort for plans above SORT_CAP ROIs: chunks of MSORT_CH keys
// sorted in shared memory (bitonic), then merge passes doubling the run width
// (merge path: each thread finds its split of the two runs by binary search
// and writes MSORT_PT outputs).  Keys are distinct, so no tie rule is needed.
constexpr int MSORT_CH = 4096;
constexpr int MSORT_PT = 8;

__global__ void __launch_bounds__(1024) k_msort_chunks(KParams p, unsigned long long* out) {
  __shared__ unsigned long long s[MSORT_CH];
  const unsigned n = *p.n_used;
  if ((int64_t)n > p.max_rois) return;  // reported by k_msort_done
  for (unsigned c0 = blockIdx.x * MSORT_CH; c0 < n; c0 += gridDim.x * MSORT_CH) {
    for (unsigned i = threadIdx.x; i < MSORT_CH; i += blockDim.x)
      s[i] = c0 + i < n ? p.keys[p.slot_list[c0 + i]] : EMPTY_KEY;
    __syncthreads();
    for (unsigned k = 2; k <= MSORT_CH; k <<= 1) {
      for (unsigned j = k >> 1; j > 0; j >>= 1) {
        for (unsigned i = threadIdx.x; i < MSORT_CH; i += blockDim.x) {
          const unsigned ixj = i ^ j;
          if (ixj > i) {
            const unsigned long long a = s[i], c = s[ixj];
            if ((a > c) == ((i & k) == 0)) {
              s[i] = c;
              s[ixj] = a;
            }
          }
        }
        __syncthreads();
      }
    }
    for (unsigned i = threadIdx.x; i < MSORT_CH && c0 + i < n; i += blockDim.x) out[c0 + i] = s[i];
    __syncthreads();
  }
}

__global__ void k_msort_merge(KParams p, const unsigned long long* src, unsigned long long* dst, unsigned w) {
  const unsigned n = *p.n_used;
  if ((int64_t)n > p.max_rois) return;
  for (unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; t * MSORT_PT < n;
       t += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned k0 = (unsigned)(t * MSORT_PT);
    const unsigned base = k0 / (2 * w) * (2 * w);
    const unsigned la = min(w, n - base), lb = n - base > w ? min(w, n - base - w) : 0u;
    const unsigned long long* A = src + base;
    const unsigned long long* B = src + base + la;
    const unsigned d = k0 - base;
    unsigned lo = d > lb ? d - lb : 0u, hi = min(d, la);
    while (lo < hi) {  // number of A elements among the first d outputs
      const unsigned a = (lo + hi) >> 1;
      if (A[a] < B[d - a - 1]) lo = a + 1;
      else hi = a;
    }
    unsigned ia = lo, ib = d - lo;
    const unsigned end = min(base + la + lb, k0 + MSORT_PT);
    for (unsigned k = k0; k < end; ++k) {
      const bool takeA = ib >= lb || (ia < la && A[ia] < B[ib]);
      dst[k] = takeA ? A[ia++] : B[ib++];
    }
  }
}

__global__ void k_msort_done(KParams p) {
  const unsigned n = *p.n_used;
  const bool over = (int64_t)n > p.max_rois;
  *p.n_roi = over ? 0u : n;
  if (p.n_roi_out) *p.n_roi_out = (int64_t)n;
  if (over) atomicOr(p.err, E_ROI_CAP);
  else if ((int64_t)n > p.cap_roi) atomicOr(p.err, E_ROI_CAP);
}

// Per ROI: gather its scan accumulator, decide the processing class and
// append it to that class's work queue.
__global__ void k_setup(KParams p) {
  const unsigned n = *p.n_roi;
  // padded cells: the GLCM / edge / NGTDM / GLDM raster of k_roi and the
  // GLRLM / GLSZM raster (one border cell) must fit the class
  const int pad = (p.need & (NEED_GLCM | NEED_EDGE | NEED_NGTDM | NEED_GLDM | NEED_GLRLM | NEED_GLSZM)) ? p.pad : 0;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const unsigned long long key = p.sorted_keys[i];
    const int s = g_find(p.keys, p.hmask, key);
    RoiInfo r;
    r.key = key;
    if (s < 0) {  // cannot happen: every sorted key came from the table
      atomicOr(p.err, E_INTERNAL);
      r.n = 0;
      r.cls = BIG_CLASS;
      p.rois[i] = r;
      continue;
    }
    p.slot_dense[s] = (int)i;
    const SlotAcc a = p.slots[s];
    r.n = a.count;
    r.x0 = a.xmin;
    r.y0 = a.ymin;
    r.z0 = a.zmin;
    r.w = a.xmax - a.xmin + 1;
    r.h = a.ymax - a.ymin + 1;
    r.d = a.zmax - a.zmin + 1;
    r.vmin = a.vmin;
    r.vmax = a.vmax;
    const long long cells = (long long)(r.w + 2 * pad) * (r.h + 2 * pad) * (p.ndim == 3 ? r.d + 2 * pad : 1);
    bool pack_ok = p.ndim == 3 ? (r.w + 2 * pad <= 2048 && r.h + 2 * pad <= 2048 && r.d + 2 * pad <= 1024)
                               : (r.w + 2 * pad <= 65535 && r.h + 2 * pad <= 65535);
    int cls = BIG_CLASS;  // beyond every single-block path
    for (int c = N_BLOCK_CLASSES - 1; c >= 0; --c)
      if (pack_ok && r.n <= (unsigned)p.lim_pix[c] && cells <= p.lim_cells[c]) cls = c;
    r.cls = cls;
    r.pad = 0;
    p.rois[i] = r;
    if ((int64_t)i >= p.cap_roi) continue;  // no room for its output row
    if (cls == BIG_CLASS) {  // multi-block class: register the ROI and its arena region
      const unsigned long long cells3 = (unsigned long long)r.w * r.h * (p.ndim == 3 ? r.d : 1);
      if (!p.big || cells3 >= (1ull << 30)) {
        atomicOr(p.err, E_TOO_LARGE);
        continue;
      }
      const int nch = (int)((cells3 + BIG_CHUNK - 1) / BIG_CHUNK);
      // 16-bit order statistics from a value histogram when it is dense
      // (range <= pixels), else from sorted values like float images
      const unsigned span_v = r.vmax - r.vmin + 1;
      const unsigned range = (p.dtype != NYX_F32 && (p.need & NEED_ORDER) && span_v <= r.n) ? span_v : 0u;
      // GLCM spans: a raster of padded cells in shared memory when the largest
      // neighbour displacement leaves room for at least 2,048 cells, else
      // spans of BIG_GSPAN chunks reading neighbours from global memory
      int gsp = 0, nsp = 0, hal = 0, n_g = 0;
      if (p.need & NEED_GLCM) {
        const int dd = p.pad, n_off = p.n_dist * p.n_dirs;
        const long long Wp = r.w + 2 * dd, Hp = r.h + 2 * dd, Dp = p.ndim == 3 ? r.d + 2 * dd : 1;
        long long hmax = 0;
        for (int o = 0; o < n_off; ++o) {
          long long ds = ((long long)p.off[o][2] * Hp + p.off[o][1]) * Wp + p.off[o][0];
          ds = ds < 0 ? -ds : ds;
          hmax = ds > hmax ? ds : hmax;
        }
        const long long rc = glcm_raster_cells(p.ng, n_off), pcells = Wp * Hp * Dp;
        if (rc - hmax >= 2048 && pcells < (1ll << 31)) {
          gsp = (int)(((rc - hmax) / 512) * 512);
          hal = (int)hmax;
          nsp = (int)((pcells + gsp - 1) / gsp);
        } else {
          nsp = (nch + BIG_GSPAN - 1) / BIG_GSPAN;
        }
        const int G = glcm_group(p.ng, n_off);
        n_g = nsp * ((n_off + G - 1) / G);
      }
      const BigLayout L = big_layout(p, nch, nsp, range, r.n);
      const unsigned long long a = atomicAdd(p.big_used, L.total);
      const unsigned long long u1c = atomicAdd(p.big_used + 1, (unsigned long long)nch);
      const unsigned long long u2c = atomicAdd(p.big_used + 2, (unsigned long long)n_g);
      if (a + L.total > p.arena_cap || u1c + nch > 0x3FFFFFull || u2c + n_g > 0x3FFFFFull) {
        atomicOr(p.err, E_TOO_LARGE);
        continue;
      }
      // one atomic hands out the big-ROI index and its first pass and GLCM
      // units, so both grow with the index
      const unsigned long long old =
          atomicAdd(p.big_ctr, (1ull << 44) | ((unsigned long long)nch << 22) | (unsigned long long)n_g);
      BigRoi br;
      br.item = (int)i;
      br.nch = nch;
      br.u1 = big_units1(old);
      br.u2 = big_units2(old);
      br.nsp = nsp;
      br.gsp = gsp;
      br.hal = hal;
      br.range = range;
      br.arena = a;
      p.big[big_count(old)] = br;
      continue;
    }
    unsigned q = atomicAdd(&p.qlen[cls], 1u);
    p.queue[(int64_t)cls * p.max_rois + q] = (int)i;
  }
}

// Return the label table to its empty state (only the slots this call used).
__global__ void k_reset(KParams p) {
  const unsigned n = *p.n_used;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int s = p.slot_list[i];
    p.keys[s] = EMPTY_KEY;
    acc_identity(p.slots[s]);
  }
}

__global__ void k_init_table(KParams p, unsigned cap) {
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < cap; i += gridDim.x * blockDim.x) {
    p.keys[i] = EMPTY_KEY;
    acc_identity(p.slots[i]);
  }
}

// Per-pixel GLCM bin (test hook): IBSI fixed bin number with the ROI's min/max.
template <class T>
__global__ void k_debug_bins(KParams p, uint16_t* out) {
  const int64_t total = p.rows_total * p.nx;
  const int64_t per = p.nx * p.ny * p.nz;
  const T* img = (const T*)p.img;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int L = p.mask[i];
    uint16_t res = 0xFFFF;
    if (L > 0) {
      const unsigned long long key = ((unsigned long long)(i / per) << 32) | (unsigned)L;
      const int s = g_find(p.keys, p.hmask, key);
      if (s >= 0) {
        const RoiInfo r = p.rois[p.slot_dense[s]];
        const unsigned e = Enc<T>::enc(img[i]);
        if (r.vmax == r.vmin) {
          res = 0;
        } else if (Enc<T>::INTEGER) {
          unsigned long long q = (unsigned long long)p.ng * (e - r.vmin) / (r.vmax - r.vmin);
          res = (uint16_t)(q > (unsigned)(p.ng - 1) ? p.ng - 1 : q);
        } else {
          double x = Enc<T>::dec(e), mn = Enc<T>::dec(r.vmin), mx = Enc<T>::dec(r.vmax);
          double q = __ddiv_rn(__dmul_rn((double)p.ng, __dsub_rn(x, mn)), __dsub_rn(mx, mn));
          long long b = (long long)floor(q);
          res = (uint16_t)(b > p.ng - 1 ? p.ng - 1 : (b < 0 ? 0 : b));
        }
      }
    }
    out[i] = res;
  }
}

// ---------------------------------------------------------------------------
// host launchers (kernel templates are launched only from this file)

__global__ void k_begin(KParams p) {
  const int t = threadIdx.x;
  if (t == 0) {
    *p.n_used = 0;
    *p.n_roi = 0;
  }
  if (t < N_BLOCK_CLASSES) {
    p.qlen[t] = 0;
    p.qhead[t] = 0;
  }
  if (t < N_BLOCK_CLASSES && p.rz_head) p.rz_head[t] = 0;
  if (t < 3 && p.big_ctr) {
    if (t == 0) *p.big_ctr = 0;
    p.big_used[t] = 0;
  }
  for (int b = t; b < p.batch; b += blockDim.x) {
    p.img_vmin[b] = 0xFFFFFFFFu;
    p.img_vmax[b] = 0;
  }
}

// cuTensorMapEncodeTiled from the driver, through the runtime (the library
// links no libcuda); null when the driver does not offer it
using EncodeTiledFn = PFN_cuTensorMapEncodeTiled_v12000;
static EncodeTiledFn tma_encoder() {
  static const EncodeTiledFn fn = []() -> EncodeTiledFn {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return (EncodeTiledFn)f;
  }();
  return fn;
}

// Tensor maps of mask (int32) and image (raw 16- or 32-bit words) as 2D
// arrays of rows_total rows x nx columns, box 128 columns x TMA_SR rows.
// False (register-load scan) when the plan asks for register loads, or
// unless both row pitches are multiples of 16 bytes, both bases 16-byte
// aligned and the row count fits 32 bits.
template <class T>
static bool scan_tensor_maps(const KParams& p, CUtensorMap& tm_mask, CUtensorMap& tm_img) {
  const int64_t es = (int64_t)sizeof(T);
  if (p.scan_stage != 0) return false;
  if (p.nx <= 0 || p.rows_total <= 0 || p.nx % 4 || (p.nx * es) % 16 || p.nx > INT32_MAX || p.rows_total > INT32_MAX)
    return false;
  if ((((uintptr_t)p.mask) | ((uintptr_t)p.img)) & 15u) return false;
  const EncodeTiledFn enc = tma_encoder();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)p.nx, (cuuint64_t)p.rows_total};
  const cuuint64_t pitch_m[1] = {(cuuint64_t)p.nx * 4u}, pitch_i[1] = {(cuuint64_t)(p.nx * es)};
  const cuuint32_t box[2] = {(cuuint32_t)TX, (cuuint32_t)TMA_SR}, estr[2] = {1u, 1u};
  if (enc(&tm_mask, CU_TENSOR_MAP_DATA_TYPE_INT32, 2, (void*)p.mask, dims, pitch_m, box, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return false;
  return enc(&tm_img, es == 4 ? CU_TENSOR_MAP_DATA_TYPE_UINT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, (void*)p.img,
             dims, pitch_i, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// rows per warp and tile: the tallest tile that still gives every block
// two tiles (taller tiles spread the per-tile table flush over more rows),
// unless a tuned tile height is set
static int scan_rows_per_warp(const KParams& p, int64_t grid) {
  const int64_t rows = (p.scan_row1 > 0 ? p.scan_row1 : p.rows_total) - p.scan_row0;
  const int64_t ntx = (p.nx + TX - 1) / TX;
  int rpt = SCAN_RPT / 4;
  for (int c = SCAN_RPT; c > SCAN_RPT / 4; c /= 2)
    if (ntx * ((rows + 8ll * c - 1) / (8ll * c)) >= 2 * grid) {
      rpt = c;
      break;
    }
  if (p.scan_rpt > 0) rpt = p.scan_rpt < SCAN_RPT ? p.scan_rpt : SCAN_RPT;
  return rpt;
}

template <class T>
static cudaError_t launch_scan_t(const KParams& p, int nsm, cudaStream_t st) {
  int nb = 0;
  cudaError_t e;
  CUtensorMap tm_mask, tm_img;
  if (scan_tensor_maps<T>(p, tm_mask, tm_img)) {
    constexpr int smem = tma_smem_bytes<T>();
    if ((e = cudaFuncSetAttribute(k_scan_tma<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess)
      return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_scan_tma<T>, SCAN_NT, smem)) != cudaSuccess)
      return e;
    const int64_t grid = (int64_t)(nb > 0 ? nb : 1) * nsm;
    k_scan_tma<T><<<(int)grid, SCAN_NT, smem, st>>>(tm_mask, tm_img, p, scan_rows_per_warp(p, grid));
    return cudaGetLastError();
  }
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_scan<T>, SCAN_NT, 0)) != cudaSuccess) return e;
  const int64_t grid = (int64_t)(nb > 0 ? nb : 1) * nsm;
  k_scan<T><<<(int)grid, SCAN_NT, 0, st>>>(p, scan_rows_per_warp(p, grid));
  return cudaGetLastError();
}

// counters reset + label scan
cudaError_t launch_front(const KParams& p, int nsm, cudaStream_t st) {
  k_begin<<<1, 256, 0, st>>>(p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  switch (p.dtype) {
    case NYX_U16: return launch_scan_t<uint16_t>(p, nsm, st);
    case NYX_I16: return launch_scan_t<int16_t>(p, nsm, st);
    default: return launch_scan_t<float>(p, nsm, st);
  }
}

// key sort (one block up to SORT_CAP keys, else multi-block) + per-ROI setup
cudaError_t launch_sort_setup(const KParams& p, int nsm, cudaStream_t st) {
  cudaError_t e;
  if (p.max_rois <= SORT_CAP) {
    const int smem = (int)(4 * (32 * 256 + 256) + 4 * p.max_rois);  // counts + two u16 index buffers
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    static int configured[64] = {0};
    if (dev < 64 && configured[dev] < smem) {
      e = cudaFuncSetAttribute(k_sort_keys, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e != cudaSuccess) return e;
      configured[dev] = smem;
    }
    k_sort_keys<<<1, 1024, smem, st>>>(p);
  } else {
    // passes until the run width covers max_rois; the chunk sort writes to
    // whichever buffer makes the last pass land in sorted_keys
    int npass = 0;
    for (int64_t w = MSORT_CH; w < p.max_rois; w <<= 1) ++npass;
    unsigned long long* bufs[2] = {p.sorted_keys, p.sort_tmp};
    int cur = npass & 1;
    int64_t nchunk = (p.max_rois + MSORT_CH - 1) / MSORT_CH;
    k_msort_chunks<<<(int)(nchunk < 4 * nsm ? nchunk : 4 * nsm), 1024, 0, st>>>(p, bufs[cur]);
    int64_t nthr = (p.max_rois + MSORT_PT - 1) / MSORT_PT, nb = (nthr + 255) / 256;
    if (nb > 8 * nsm) nb = 8 * nsm;
    unsigned w = MSORT_CH;
    for (int i = 0; i < npass; ++i, w <<= 1) {
      k_msort_merge<<<(int)nb, 256, 0, st>>>(p, bufs[cur], bufs[cur ^ 1], w);
      cur ^= 1;
    }
    k_msort_done<<<1, 1, 0, st>>>(p);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  int g = (int)((p.max_rois + 255) / 256);
  if (g > 4 * nsm) g = 4 * nsm;
  k_setup<<<g, 256, 0, st>>>(p);
  return cudaGetLastError();
}

// pieces of the front for the streamed mosaic: counter reset, and the label
// scan of rows [scan_row0, scan_row1)
cudaError_t launch_begin(const KParams& p, cudaStream_t st) {
  k_begin<<<1, 256, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_scan(const KParams& p, int nsm, cudaStream_t st) {
  switch (p.dtype) {
    case NYX_U16: return launch_scan_t<uint16_t>(p, nsm, st);
    case NYX_I16: return launch_scan_t<int16_t>(p, nsm, st);
    default: return launch_scan_t<float>(p, nsm, st);
  }
}

cudaError_t launch_reset(const KParams& p, int nsm, cudaStream_t st) {
  k_reset<<<2 * nsm, 256, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_init_table(const KParams& p, unsigned cap, cudaStream_t st) {
  k_init_table<<<256, 256, 0, st>>>(p, cap);
  return cudaGetLastError();
}

cudaError_t launch_debug_bins(const KParams& p, uint16_t* out, int nsm, cudaStream_t st) {
  switch (p.dtype) {
    case NYX_U16: k_debug_bins<uint16_t><<<4 * nsm, 256, 0, st>>>(p, out); break;
    case NYX_I16: k_debug_bins<int16_t><<<4 * nsm, 256, 0, st>>>(p, out); break;
    default: k_debug_bins<float><<<4 * nsm, 256, 0, st>>>(p, out); break;
  }
  return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// Allocation-free ROI count.
//
// Some callers cannot allocate device memory for this library: hosts that
// hand every byte of the GPU to their own pool allocator and forbid
// cudaMalloc from plug-ins, applications running under a fixed device-memory
// quota (a shared cloud node, an instrument PC that keeps acquiring while it
// analyses), and code paths where cudaMalloc's implicit device
// synchronisation is not acceptable.  For them nyx_count_rois_noalloc runs
// the label scan with its label table in this fixed file-scope array instead
// of a plan workspace.  Every GPU that loads the library holds the array
// until the process exits.
//
// Layout of the array (bytes): keys[NOALLOC_SLOTS] (8 B each), slot
// accumulators[NOALLOC_SLOTS] (48 B each), slot list[NOALLOC_SLOTS] (4 B each),
// image ranges 2 x NOALLOC_MAX_BATCH (4 B each), 64 B of counters.
constexpr unsigned NOALLOC_SLOTS = 2u * NYX_NOALLOC_MAX_LABELS;  // load factor <= 0.5
constexpr size_t NOALLOC_BYTES = (size_t)NOALLOC_SLOTS * (8 + sizeof(SlotAcc) + 4) +
                                 2ull * 4 * NYX_NOALLOC_MAX_BATCH + 64;
static_assert((NOALLOC_SLOTS & (NOALLOC_SLOTS - 1)) == 0, "the label table's probe mask needs a power of two");
static_assert(sizeof(SlotAcc) % 8 == 0 && (8ull * NOALLOC_SLOTS) % 8 == 0 &&
                  ((8ull + sizeof(SlotAcc) + 4) * NOALLOC_SLOTS) % 8 == 0 && (8ull * NYX_NOALLOC_MAX_BATCH) % 8 == 0,
              "every part of the fixed array starts on an 8-byte boundary");
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

// Device address of g_noalloc_scratch per device.  In host code the array's
// name is only a host-side stand-in, so the address must come from
// cudaGetSymbolAddress, made once per device with that device current.
static void* g_noalloc_ptr[64] = {nullptr};

extern "C" nyx_status nyx_count_rois_noalloc(const nyx_params* prm, const void* d_img, const int32_t* d_mask,
                                             int64_t* n_roi, void* stream) {
  if (!prm || !d_img || !d_mask || !n_roi) return NYX_ERR_ARG;
  if (prm->struct_size != sizeof(nyx_params)) return NYX_ERR_ARG;
  if (((uintptr_t)d_img & 15) || ((uintptr_t)d_mask & 15)) return NYX_ERR_ARG;
  if (prm->ndim != 2 && prm->ndim != 3) return NYX_ERR_SHAPE;
  for (int i = 0; i < 3; ++i)
    if (prm->dims[i] < 1 || prm->dims[i] > (1ll << 31)) return NYX_ERR_SHAPE;
  if (prm->ndim == 2 && prm->dims[2] != 1) return NYX_ERR_SHAPE;
  if (prm->batch < 1) return NYX_ERR_SHAPE;
  if (prm->batch > NYX_NOALLOC_MAX_BATCH) return NYX_ERR_CAPACITY;  // image ranges do not fit the array
  if (prm->dtype < 0 || prm->dtype > 2) return NYX_ERR_DTYPE;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return NYX_ERR_CUDA;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return NYX_ERR_CUDA;
  if (!g_noalloc_ptr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return NYX_ERR_CUDA;
    g_noalloc_ptr[dev] = ptr;
  }
  unsigned char* w = (unsigned char*)g_noalloc_ptr[dev];
  KParams k;
  memset(&k, 0, sizeof k);
  k.img = d_img;
  k.mask = d_mask;
  k.nx = prm->dims[0];
  k.ny = prm->dims[1];
  k.nz = prm->dims[2];
  k.batch = prm->batch;
  k.rows_total = (int64_t)prm->batch * prm->dims[2] * prm->dims[1];
  k.ndim = prm->ndim;
  k.dtype = prm->dtype;
  k.vec = (k.nx % 4) == 0;
  k.keys = (unsigned long long*)w;
  k.slots = (SlotAcc*)(w + 8ull * NOALLOC_SLOTS);
  k.slot_list = (int*)(w + (8ull + sizeof(SlotAcc)) * NOALLOC_SLOTS);
  k.hmask = NOALLOC_SLOTS - 1;
  unsigned char* tail = w + (8ull + sizeof(SlotAcc) + 4) * NOALLOC_SLOTS;
  k.img_vmin = (unsigned*)tail;
  k.img_vmax = (unsigned*)(tail + 4ull * NYX_NOALLOC_MAX_BATCH);
  unsigned* small = (unsigned*)(tail + 8ull * NYX_NOALLOC_MAX_BATCH);
  k.n_used = small + 0;
  k.n_roi = small + 1;
  k.err = small + 2;
  k.qlen = small + 4;
  k.qhead = small + 8;
  k.max_rois = NYX_NOALLOC_MAX_LABELS;
  cudaStream_t st = (cudaStream_t)stream;
  // the array keeps the previous call's contents: start from an empty table
  // and zero counters every time
  if (cudaMemsetAsync(small, 0, 64, st) != cudaSuccess) return NYX_ERR_CUDA;
  k_init_table<<<2 * nsm, 256, 0, st>>>(k, NOALLOC_SLOTS);
  if (cudaGetLastError() != cudaSuccess) return NYX_ERR_CUDA;
  if (launch_front(k, nsm, st) != cudaSuccess) return NYX_ERR_CUDA;
  unsigned h[3] = {0, 0, 0};  // n_used, n_roi (unused), error word
  if (cudaMemcpyAsync(h, small, sizeof h, cudaMemcpyDeviceToHost, st) != cudaSuccess) return NYX_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return NYX_ERR_CUDA;
  if (h[2] & E_BAD_LABEL) return NYX_ERR_BAD_LABEL;
  if (h[2] & E_NONFINITE) return NYX_ERR_NONFINITE;
  if ((h[2] & E_HASH_FULL) || h[0] > (unsigned)NYX_NOALLOC_MAX_LABELS) return NYX_ERR_CAPACITY;
  if (h[2]) return NYX_ERR_STATE;
  *n_roi = h[0];
  return NYX_OK;
}
}  // namespace nyx
