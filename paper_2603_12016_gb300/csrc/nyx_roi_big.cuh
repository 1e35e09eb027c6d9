// nyx_roi_big.cuh -- the multi-block path (class 3) for ROIs beyond the
// single-block classes (more pixels or bounding-box cells than a block stages
// in shared memory, up to ~1e6-voxel ROIs).  Included by nyx_big_<dtype>.cu;
// reuses the finalisers of nyx_roi.cuh so both paths compute every feature
// with the same arithmetic.
//
// The bounding box of a big ROI is cut into chunks of BIG_CHUNK raster
// cells.  Each kernel streams chunk cells straight from global memory (the
// image and mask are L2-resident after the label scan for all but the largest
// inputs), with one 512-thread block per unit:
//   k_big_zero   clear each big ROI's counters and histograms
//   k_big_p1     units (ROI, chunk): exact pass-1 sums (int64 for integer
//                images, Kahan-compensated otherwise), the hist_bins
//                histogram, and for 16-bit images the value histogram over
//                [min, max]; the last unit of an ROI merges the per-chunk
//                partials in chunk order and derives the mean, centroids,
//                histogram features and the order statistics
//   k_big_p2     units (ROI, chunk): one pass for the centred power sums
//                and both sets of central moments, compensated across the
//                block; the last unit merges them in chunk order and hands
//                them to k_stats_final
//   k_big_glcm   units (ROI, span, group of offsets): one dense upper-
//                triangular co-occurrence matrix per offset of the group in
//                shared memory (Ng(Ng+1)/2 counts, diagonal counted twice).
//                A span is a range of the ROI's padded bounding box staged
//                as a raster of bins (plus a forward halo of the largest
//                neighbour displacement), so neighbours are shared-memory
//                loads; ROIs whose halo does not fit read neighbours from
//                global memory.  ROIs of several spans add the triangles
//                into global ones and the last span of the group reduces
//                them to the per-offset sums that k_glcm_final turns into
//                features
//   k_big_ngtdm  units (ROI, chunk): NGTDM neighbourhood sums and GLDM
//                dependence counts over a shared-memory window of bins
//                (chunk plus a plane-and-row halo); the last unit of an ROI
//                derives the features
//   k_big_order  ROIs without a value histogram (float images, 16-bit ROIs
//                whose value range exceeds their pixel count): one block
//                per ROI compacts the values in raster order and sorts them
//                (LSD radix, global memory)
// "Last unit" is decided with a counter in the ROI's arena region after a
// __threadfence, and every merge runs in chunk order, so results do not
// depend on which block ran which unit.
#pragma once

#include "nyx_roi.cuh"

namespace nyx {

constexpr int BIG_NT = 512;
// resident blocks per SM of the pass kernels: two (64 registers a thread) on
// the float path, one on the FP64 path, whose wider state would spill
template <class A> constexpr int big_pass_minb() { return std::is_same<A, float>::value ? 2 : 1; }
constexpr int VH_SMEM = 8192;  // value-histogram words kept in shared memory per chunk
using ClassBig = RoiClass<BIG_NT, 1, 1>;  // thread geometry for the block reductions

// the big ROI owning pass unit u (GLCM unit u with glcm = true); the first
// units u1 and u2 grow with the big-ROI index
__device__ inline int big_of_unit(const KParams& p, int n_big, unsigned u, bool glcm = false) {
  int lo = 0, hi = n_big - 1;
  while (lo < hi) {
    const int m = (lo + hi + 1) >> 1;
    if ((glcm ? p.big[m].u2 : p.big[m].u1) <= u) lo = m;
    else hi = m - 1;
  }
  return lo;
}


// block sum of Kahan pairs: sums and negated corrections reduced separately
// (each compensated), then added; out[] in shared memory for every thread
template <class C, class A, int NV>
__device__ inline void block_sum_k(KSum<A> (&v)[NV], double* scratch, A* out) {
  A hi[NV], lo[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    hi[i] = v[i].s;
    lo[i] = -v[i].c;
  }
  block_sum<C, A, NV>(lo, scratch, out);
  A lo_i = 0;
  if (threadIdx.x < NV) lo_i = out[threadIdx.x];
  __syncthreads();
  block_sum<C, A, NV>(hi, scratch, out);
  if (threadIdx.x < NV) out[threadIdx.x] += lo_i;
  __syncthreads();
}

// Bounding box of one big ROI and the cell -> (x, y, z) decomposition.
struct BigBox {
  int W, H, D;
  unsigned cells;
  FastDiv dw, dh;
  int64_t origin;  // linear index of the box origin in the image batch
  int label;
  __device__ void init(const KParams& p, const RoiInfo& r, int ndim) {
    W = r.w;
    H = r.h;
    D = ndim == 3 ? r.d : 1;
    cells = (unsigned)W * (unsigned)H * (unsigned)D;
    dw.init((unsigned)W);
    dh.init((unsigned)H);
    const int64_t per = p.nx * p.ny * p.nz;
    origin = (int64_t)(r.key >> 32) * per + ((int64_t)r.z0 * p.ny + r.y0) * p.nx + r.x0;
    label = (int)(r.key & 0xFFFFFFFFu);
  }
  __device__ int64_t offset(unsigned c, int& x, int& y, int& z, const KParams& p) const {
    const unsigned zy = dw.div(c);
    x = (int)(c - zy * (unsigned)W);
    const unsigned zz = dh.div(zy);
    y = (int)(zy - zz * (unsigned)H);
    z = (int)zz;
    return origin + ((int64_t)z * p.ny + y) * p.nx + x;
  }
};

// Visit cells [c0, c1) with every thread of the block making the same number
// of iterations, so that f may use warp-synchronous operations:
// f(in, x, y, z, encoded value), in = the cell belongs to the ROI.  Each
// thread issues the mask and image loads of BIG_U cells before using them (a
// cell of the bounding box is always inside the image, so the image load
// needs no mask test): the loop is bound by L2 latency, not bandwidth.
// Edge test of an ROI voxel at bbox-local (x, y, z): a face neighbour
// (4 in 2D, 6 in 3D) outside the bounding box, or inside it under another
// label, makes it an edge voxel.  Neighbour labels are read from the mask.
template <int NDIM>
__device__ inline bool big_edge(const KParams& p, const BigBox& bx, int x, int y, int z) {
  const int64_t here = bx.origin + ((int64_t)z * p.ny + y) * p.nx + x;
  if (x == 0 || x == bx.W - 1 || y == 0 || y == bx.H - 1) return true;
  if (NDIM == 3 && (z == 0 || z == bx.D - 1)) return true;
  // every neighbour is inside the box here: issue all loads, then combine
  const int l0 = __ldg(p.mask + here - 1), l1 = __ldg(p.mask + here + 1);
  const int l2 = __ldg(p.mask + here - p.nx), l3 = __ldg(p.mask + here + p.nx);
  bool e = (l0 != bx.label) | (l1 != bx.label) | (l2 != bx.label) | (l3 != bx.label);
  if (NDIM == 3) {
    const int64_t pl = p.nx * p.ny;
    const int l4 = __ldg(p.mask + here - pl), l5 = __ldg(p.mask + here + pl);
    e |= (l4 != bx.label) | (l5 != bx.label);
  }
  return e;
}

constexpr int BIG_U = 4;
template <class T, class F>
__device__ inline void chunk_cells(const KParams& p, const BigBox& bx, unsigned c0, unsigned c1, F f) {
  const T* img = (const T*)p.img;
#pragma unroll 1
  for (unsigned cb = c0; cb < c1; cb += BIG_U * BIG_NT) {
    int xs[BIG_U], ys[BIG_U], zs[BIG_U], lab[BIG_U];
    T val[BIG_U];
#pragma unroll
    for (int u = 0; u < BIG_U; ++u) {
      const unsigned c = cb + u * BIG_NT + threadIdx.x;
      lab[u] = 0;
      xs[u] = ys[u] = zs[u] = 0;
      if (c < c1) {
        const int64_t off = bx.offset(c, xs[u], ys[u], zs[u], p);
        lab[u] = __ldg(p.mask + off);
        val[u] = __ldg(img + off);
      }
    }
#pragma unroll
    for (int u = 0; u < BIG_U; ++u) {
      const unsigned c = cb + u * BIG_NT + threadIdx.x;
      const bool in = c < c1 && lab[u] == bx.label;
      f(in, xs[u], ys[u], zs[u], in ? Enc<T>::enc(val[u]) : 0u, c);
    }
  }
}

// Visit the ROI voxels of cells [c0, c1) in full warps: cells are streamed
// as in chunk_cells, each warp compacts its ROI cells into a 64-entry queue
// in shared memory (qc: cell index, qe: encoded value) and calls
// f(valid, x, y, z, e) once per 32 queued voxels, then once for the remainder
// (lanes past it have valid = false).  Work per voxel runs on full warps
// instead of on every lane of partly filled ones.
template <class T, class F>
__device__ inline void chunk_voxels(const KParams& p, const BigBox& bx, unsigned c0, unsigned c1, unsigned* qc,
                                    unsigned* qe, F f) {
  const int lane = threadIdx.x & 31;
  int qn = 0;  // warp-uniform queue length (< 32 between flushes)
  auto flush32 = [&]() {
    const unsigned c = qc[lane], e = qe[lane];
    int x, y, z;
    bx.offset(c, x, y, z, p);
    f(true, x, y, z, e);
    __syncwarp();
    if (lane < qn - 32) {
      qc[lane] = qc[32 + lane];
      qe[lane] = qe[32 + lane];
    }
    __syncwarp();
    qn -= 32;
  };
  chunk_cells<T>(p, bx, c0, c1, [&](bool in, int, int, int, unsigned e, unsigned c) {
    const unsigned bal = __ballot_sync(0xFFFFFFFFu, in);
    if (in) {
      const unsigned pos = qn + __popc(bal & lanemask_lt());
      qc[pos] = c;
      qe[pos] = e;
    }
    qn += __popc(bal);
    __syncwarp();
    if (qn >= 32) flush32();
  });
  int x = 0, y = 0, z = 0;
  const bool v = lane < qn;
  if (v) bx.offset(qc[lane], x, y, z, p);
  f(v, x, y, z, v ? qe[lane] : 0u);
}

// true in every thread of the one block that finishes last among `total`
// (counter in global memory; the caller's global writes are fenced first)
__device__ inline bool last_arrival(unsigned* counter, unsigned total, int* s_flag) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) *s_flag = atomicAdd(counter, 1u) == total - 1;
  __syncthreads();
  const bool last = *s_flag != 0;
  if (last) __threadfence();
  return last;
}

// ---------------------------------------------------------------------------

template <class T>  // (templated so each dtype's translation unit owns its copy)
__global__ void __launch_bounds__(BIG_NT) k_big_zero(KParams p) {
  const int n_big = big_count(*p.big_ctr);
  for (int b = blockIdx.x; b < n_big; b += gridDim.x) {
    const BigRoi br = p.big[b];
    const RoiInfo r = p.rois[br.item];
    const BigLayout L = big_layout(p, br.nch, br.nsp, br.range, r.n);
    uint4* z = (uint4*)(p.arena + br.arena);
    const unsigned long long n4 = L.zero_end / 4;
    for (unsigned long long i = threadIdx.x; i < n4; i += BIG_NT) z[i] = make_uint4(0, 0, 0, 0);
  }
}

// Percentiles, mode, robust mean / MAD and median MAD of a 16-bit ROI from its
// value histogram h[0..range) (bin k = encoded value vmin + k).  Every thread
// of the block calls it.  The percentile arithmetic is the FP64 definition
// on the two order statistics around h = (n-1) q, as in finalize_percentiles.
template <class T, class A>
__device__ void hist_order_stats(const KParams& p, double* row, const unsigned* h, unsigned range, unsigned vmin,
                                 int n, double* red, A* s_sc) {
  using C = ClassBig;
  const int tid = threadIdx.x;
  const long long ibias = std::is_same<T, int16_t>::value ? 32768 : 0;
  const A nan = anan<A>();
  __shared__ long long s_rank[14], s_val[14];
  __shared__ long long s_thr[3];
  __shared__ unsigned long long s_best;
  __shared__ long long s_iv[3];
  if (tid < 14) {
    const double qs[7] = {0.01, 0.10, 0.25, 0.50, 0.75, 0.90, 0.99};
    const double hq = __dmul_rn((double)(n - 1), qs[tid >> 1]);
    const long long rk = (long long)floor(hq) + (tid & 1);
    s_rank[tid] = rk > n - 1 ? n - 1 : rk;
  }
  const unsigned seg = (range + BIG_NT - 1) / BIG_NT;
  const unsigned b0 = min(range, tid * seg), b1 = min(range, b0 + seg);
  unsigned segtot = 0;
  unsigned long long best = 0;  // (count << 32) | ~bin: most frequent, then smallest value
  for (unsigned k = b0; k < b1; ++k) {
    const unsigned c = __ldcg(h + k);
    segtot += c;
    const unsigned long long cand = ((unsigned long long)c << 32) | (unsigned)~k;
    if (c && cand > best) best = cand;
  }
  unsigned* scan = (unsigned*)red;
  scan[tid] = segtot;
  __syncthreads();
  if (tid < 32) warp_exclusive_scan(scan, BIG_NT);
  __syncthreads();
  const unsigned long long segbase = scan[tid];
  __syncthreads();
  best = block_max_u64<C>(best, red);
  for (int k = 0; k < 14; ++k) {
    const unsigned long long rk = (unsigned long long)s_rank[k];
    if (rk >= segbase && rk < segbase + segtot) {
      unsigned long long acc = segbase;
      for (unsigned q = b0; q < b1; ++q) {
        acc += __ldcg(h + q);
        if (rk < acc) {
          s_val[k] = (long long)(vmin + q) - ibias;
          break;
        }
      }
    }
  }
  __syncthreads();
  if (tid == 0) {
    const double qs[7] = {0.01, 0.10, 0.25, 0.50, 0.75, 0.90, 0.99};
    const int qcol[7] = {S_P01, S_P10, S_P25, S_MEDIAN, S_P75, S_P90, S_P99};
    double pv_[7];
    for (int k = 0; k < 7; ++k) {
      const double hq = __dmul_rn((double)(n - 1), qs[k]);
      const long long lo = (long long)floor(hq);
      const double a = (double)s_val[2 * k], b = (double)s_val[2 * k + 1];
      pv_[k] = lo >= n - 1 ? a : __dadd_rn(a, __dmul_rn(__dsub_rn(hq, (double)lo), __dsub_rn(b, a)));
      put(p, row, Q_STATS + qcol[k], pv_[k]);
    }
    put(p, row, Q_STATS + S_IQR, __dsub_rn(pv_[4], pv_[2]));
    const float qa = (float)pv_[4], qb = (float)pv_[2];
    put(p, row, Q_STATS + S_QCOD, (qa + qb) != 0.f ? f2d((qa - qb) / (qa + qb)) : f2d(__int_as_float(0x7FC00000)));
    s_thr[0] = (long long)ceil(pv_[1]);    // values >= P10
    s_thr[1] = (long long)floor(pv_[5]);   // values <= P90
    s_thr[2] = (long long)(2.0 * pv_[3]);  // twice the median: an integer (h - floor(h) is 0 or 1/2)
    s_best = best;
  }
  __syncthreads();
  const long long t10 = s_thr[0], t90 = s_thr[1], med2 = s_thr[2];
  // exact integer sums: [0] sum c v over [P10, P90], [1] count there, [2] sum c |2v - 2 median|
  long long iv[3] = {0, 0, 0};
  for (unsigned k = b0; k < b1; ++k) {
    const unsigned c = __ldcg(h + k);
    if (!c) continue;
    const long long v = (long long)(vmin + k) - ibias;
    if (v >= t10 && v <= t90) {
      iv[0] += (long long)c * v;
      iv[1] += c;
    }
    const long long d2 = 2 * v - med2;
    iv[2] += (long long)c * (d2 < 0 ? -d2 : d2);
  }
  block_sum_i64<C, 3>(iv, red, s_iv);
  const long long cntV = s_iv[1];
  const A rmA = cntV > 0 ? (A)s_iv[0] / (A)cntV : nan;
  KSum<A> ra[1];
  for (unsigned k = b0; k < b1; ++k) {
    const unsigned c = __ldcg(h + k);
    if (!c) continue;
    const long long v = (long long)(vmin + k) - ibias;
    if (v < t10 || v > t90) continue;
    const A vA = (A)v;
    ra[0].add((A)c * (vA > rmA ? vA - rmA : rmA - vA));
  }
  block_sum_k<C, A, 1>(ra, red, s_sc + 12);
  if (tid == 0) {
    const unsigned long long bb = s_best;
    put(p, row, Q_STATS + S_MODE, i2d((long long)(vmin + ~(unsigned)(bb & 0xFFFFFFFFu)) - ibias));
    putA(p, row, Q_STATS + S_MODE_PROB, (A)(int)(bb >> 32) / (A)n);
    putA(p, row, Q_STATS + S_RMEAN, rmA);
    putA(p, row, Q_STATS + S_RMAD, cntV > 0 ? s_sc[12] / (A)cntV : nan);
    putA(p, row, Q_STATS + S_MEDAD, (A)s_iv[2] / ((A)2 * (A)n));
  }
  __syncthreads();
}

template <class T, int NDIM, class A>
__global__ void __launch_bounds__(BIG_NT, big_pass_minb<A>()) k_big_p1(KParams p) {
  using C = ClassBig;
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned* hist = (unsigned*)smem;                // [hist_bins]
  unsigned* vh = hist + ((p.hist_bins + 3) & ~3);  // [VH_SMEM]
  __shared__ double red[C::NW * RED_MAX];
  __shared__ long long s_i64[16];
  __shared__ A s_sc[16];
  __shared__ A s_sl[8];  // low parts of the pass-1 float sums
  __shared__ int s_flag;
  __shared__ unsigned s_qc[C::NW * 64], s_qe[C::NW * 64];  // per-warp voxel queues
  const int tid = threadIdx.x;
  const unsigned long long ctr = *p.big_ctr;
  const int n_big = big_count(ctr);
  const unsigned n_units = big_units1(ctr);
  const unsigned need = p.need;
  constexpr bool integer = Enc<T>::INTEGER;
  const long long ibias = std::is_same<T, int16_t>::value ? 32768 : 0;
  for (unsigned u = blockIdx.x; u < n_units; u += gridDim.x) {
    const int b = big_of_unit(p, n_big, u);
    const BigRoi br = p.big[b];
    const int chunk = (int)(u - br.u1);
    const RoiInfo r = p.rois[br.item];
    BigBox bx;
    bx.init(p, r, NDIM);
    const BigLayout L = big_layout(p, br.nch, br.nsp, br.range, r.n);
    unsigned* reg = p.arena + br.arena;
    const unsigned c0 = (unsigned)chunk * BIG_CHUNK, c1 = min(bx.cells, c0 + (unsigned)BIG_CHUNK);
    const unsigned vmin = r.vmin, vmax = r.vmax;
    const float fmn = Enc<T>::decf(vmin), fmx = Enc<T>::decf(vmax);
    const bool do_hist = (need & NEED_HIST) != 0;
    const unsigned range = br.range;
    const bool vh_smem = range > 0 && range <= (unsigned)VH_SMEM;
    FastDiv fd;
    fd.init(vmax > vmin ? vmax - vmin : 1u);
    if (do_hist)
      for (int i = tid; i < p.hist_bins; i += BIG_NT) hist[i] = 0;
    if (vh_smem)
      for (unsigned i = tid; i < range; i += BIG_NT) vh[i] = 0;
    __syncthreads();
    // [0] sum I, [1] sum x I, [2] sum y I, [3] sum z I, [4] sum x, [5] sum y, [6] sum z, [7] sum I^2, [8] count
    long long s[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    KSum<A> fs[5];  // float images: sum I, x I, y I, z I, I^2
    // edge voxels: count, sum d, sum d^2 with d = code - vmin (exact for
    // integer images); float images sum d compensated
    const bool do_edge = (need & NEED_EDGE) != 0;
    long long es[3] = {0, 0, 0};
    KSum<A> ef[1];
    unsigned emn = 0xFFFFFFFFu, emx = 0;
    unsigned* gvh = reg + L.vhist;
    chunk_voxels<T>(p, bx, c0, c1, s_qc + (tid >> 5) * 64, s_qe + (tid >> 5) * 64,
                    [&](bool in, int x, int y, int z, unsigned e) {
      unsigned hb = 0xFFFFFFFFu, vb = 0xFFFFFFFFu;
      if (in && do_edge && big_edge<NDIM>(p, bx, x, y, z)) {
        es[0] += 1;
        emn = min(emn, e);
        emx = max(emx, e);
        if constexpr (integer) {
          const long long d = (long long)(e - vmin);
          es[1] += d;
          es[2] += d * d;
        } else {
          ef[0].add(decA<T, A>(e) - (A)fmn);
        }
      }
      if (in) {
        s[4] += x;
        s[5] += y;
        s[6] += z;
        s[8] += 1;
        if constexpr (integer) {
          const long long v = (long long)e - ibias;
          s[0] += v;
          s[1] += x * v;
          s[2] += y * v;
          s[3] += z * v;
          s[7] += v * v;
        } else {
          const A v = decA<T, A>(e);
          fs[0].add(v);
          fs[1].add((A)x * v);
          fs[2].add((A)y * v);
          fs[3].add((A)z * v);
          fs[4].add(v * v);
        }
        hb = 0;
        if (vmax > vmin) {
          if constexpr (integer) hb = min(fd.div((unsigned)p.hist_bins * (e - vmin)), (unsigned)(p.hist_bins - 1));
          else hb = bin_float(Enc<T>::decf(e), fmn, fmx, p.hist_bins);
        }
        vb = e - vmin;
      }
      if (do_hist) {  // one atomic per run of equal bins in consecutive lanes
        const unsigned len = run_leader(hb, 0xFFFFFFFFu);
        if (len) atomicAdd(&hist[hb], len);
      }
      if (range) {
        const unsigned len = run_leader(vb, 0xFFFFFFFFu);
        if (len) {
          if (vh_smem) atomicAdd(&vh[vb], len);
          else atomicAdd(&gvh[vb], len);
        }
      }
    });
    block_sum_i64<C, 9>(s, red, s_i64);
    if constexpr (!integer) {
      if constexpr (std::is_same<A, float>::value) block_sum_pair<C, 5>(fs, red, s_sc, s_sl);
      else block_sum_k<C, A, 5>(fs, red, s_sc);
    }
    unsigned bmn = 0xFFFFFFFFu, bmx = 0;
    if (do_edge) {
      block_sum_i64<C, 3>(es, red, s_i64 + 9);
      if constexpr (!integer) block_sum_k<C, A, 1>(ef, red, s_sc + 5);
      bmx = (unsigned)block_max_u64<C>(emx, red);
      bmn = 0xFFFFFFFFu - (unsigned)block_max_u64<C>(0xFFFFFFFFu - emn, red);
    }
    if (do_hist)
      for (int i = tid; i < p.hist_bins; i += BIG_NT)
        if (hist[i]) atomicAdd(reg + L.hist + i, hist[i]);
    if (vh_smem)
      for (unsigned i = tid; i < range; i += BIG_NT)
        if (vh[i]) atomicAdd(gvh + i, vh[i]);
    if (tid == 0) {
      long long* pt = (long long*)(reg + L.part1) + (size_t)chunk * (BIG_P1 / 2);
      for (int k = 0; k < 9; ++k) pt[k] = s_i64[k];
      double* pf = (double*)(pt + 9);
      for (int k = 0; k < 5; ++k) {  // float images: the pair hi + lo, exact in FP64
        if constexpr (integer) pf[k] = 0.0;
        else if constexpr (std::is_same<A, float>::value) pf[k] = pair_d(s_sc[k], s_sl[k]);
        else pf[k] = s_sc[k];
      }
      // [14] edge count, [15] sum d (float images: as a double), [16] sum d^2, [17] min code, [18] max code
      pt[14] = do_edge ? s_i64[9] : 0;
      if constexpr (integer) pt[15] = do_edge ? s_i64[10] : 0;
      else ((double*)pt)[15] = do_edge ? to_d(s_sc[5]) : 0.0;
      pt[16] = do_edge ? s_i64[11] : 0;
      pt[17] = bmn;
      pt[18] = bmx;
    }
    if (!last_arrival(reg + L.ctr + 0, (unsigned)br.nch, &s_flag)) continue;

    // ---- last chunk of this ROI: merge in chunk order, per-ROI scalars ----
    const int n = (int)r.n;
    double* row = p.table + (int64_t)br.item * p.n_col;
    const int64_t bimg = (int64_t)(r.key >> 32);
    if (tid == 0) {
      long long t[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
      double fd5[5] = {0, 0, 0, 0, 0};  // float images: chunk sums merged in FP64, chunk order
      for (int ch = 0; ch < br.nch; ++ch) {
        const long long* pt = (const long long*)(reg + L.part1) + (size_t)ch * (BIG_P1 / 2);
        for (int k = 0; k < 9; ++k) t[k] += __ldcg(pt + k);
        if constexpr (!integer) {
          const double* pf = (const double*)(pt + 9);
          for (int k = 0; k < 5; ++k) fd5[k] += __ldcg(pf + k);
        }
      }
      if (t[8] != (long long)n) atomicOr(p.err, E_INTERNAL);
      const A nA = (A)n;
      A sI, en, mhi, mlo;
      double dI, dxI, dyI, dzI;  // FP64 sums for the centroids
      if constexpr (integer) {
        const long long si = t[0];
        sI = (A)si;
        en = (A)t[7];
        dI = (double)si;
        dxI = (double)t[1];
        dyI = (double)t[2];
        dzI = (double)t[3];
        if constexpr (std::is_same<A, float>::value) {
          const long long q = si / n, rm = si - q * n;  // mean = q + rm / n exactly
          mhi = (A)q;
          mlo = (A)rm / nA;
        } else {
          mhi = (A)si / nA;
          mlo = 0;
        }
        put(p, row, Q_STATS + S_II, i2d(si));
        put(p, row, Q_STATS + S_ENERGY, i2d(t[7]));
      } else {
        dI = fd5[0];
        dxI = fd5[1];
        dyI = fd5[2];
        dzI = fd5[3];
        sI = (A)dI;
        en = (A)fd5[4];
        const double md = dI / (double)n;  // mean as an unevaluated pair in A
        mhi = (A)md;
        mlo = (A)(md - (double)mhi);
        put(p, row, Q_STATS + S_II, dI);
        put(p, row, Q_STATS + S_ENERGY, fd5[4]);
      }
      // FP64 centroids (ROI-local): binary from the exact coordinate sums,
      // intensity-weighted from the sums above
      const double bxd = (double)t[4] / n, byd = (double)t[5] / n, bzd = (double)t[6] / n;
      const bool wv = dI != 0;
      double* st = p.big[b].st;
      st[0] = to_d(mhi);
      st[1] = to_d(mlo);
      st[2] = wv ? dxI / dI : bxd;
      st[3] = wv ? dyI / dI : byd;
      st[4] = wv ? dzI / dI : bzd;
      st[5] = bxd;
      st[6] = byd;
      st[7] = bzd;
      st[8] = to_d(sI);
      st[9] = to_d(en);
      put(p, row, Q_LABEL, i2d(bx.label));
      put(p, row, Q_IMAGE, i2d(bimg));
      put(p, row, Q_AREA, i2d(n));
      put(p, row, Q_BB_X, i2d(r.x0));
      put(p, row, Q_BB_Y, i2d(r.y0));
      put(p, row, Q_BB_Z, i2d(r.z0));
      put(p, row, Q_BB_W, i2d(bx.W));
      put(p, row, Q_BB_H, i2d(bx.H));
      put(p, row, Q_BB_D, i2d(bx.D));
      if constexpr (integer) {
        put(p, row, Q_STATS + S_MIN, i2d((long long)vmin - ibias));
        put(p, row, Q_STATS + S_MAX, i2d((long long)vmax - ibias));
        put(p, row, Q_STATS + S_RANGE, i2d((long long)vmax - (long long)vmin));
      } else {
        put(p, row, Q_STATS + S_MIN, f2d(fmn));
        put(p, row, Q_STATS + S_MAX, f2d(fmx));
        put(p, row, Q_STATS + S_RANGE, __dsub_rn(f2d(fmx), f2d(fmn)));
      }
      if (do_edge) {  // edge intensity statistics, merged in chunk order
        long long ne = 0, e1 = 0, e2 = 0;
        unsigned lo_c = 0xFFFFFFFFu, hi_c = 0;
        A eh = 0, el = 0;
        for (int ch = 0; ch < br.nch; ++ch) {
          const long long* pt = (const long long*)(reg + L.part1) + (size_t)ch * (BIG_P1 / 2);
          ne += __ldcg(pt + 14);
          if constexpr (integer) {
            e1 += __ldcg(pt + 15);
          } else {
            const A x = (A)__ldcg((const double*)pt + 15);
            if constexpr (std::is_same<A, float>::value) {
              float sum, err;
              two_sum(eh, x, sum, err);
              eh = sum;
              el += err;
            } else {
              eh += x;
            }
          }
          e2 += __ldcg(pt + 16);
          lo_c = min(lo_c, (unsigned)__ldcg(pt + 17));
          hi_c = max(hi_c, (unsigned)__ldcg(pt + 18));
        }
        A emean;
        double* sv = (need & NEED_SAVE) ? p.saved + (size_t)br.item * SV_WORDS : nullptr;
        if constexpr (integer) {
          const long long sumx = e1 + ne * ((long long)vmin - ibias);
          const __int128 num = (__int128)ne * e2 - (__int128)e1 * e1;  // n^2 var_biased, exact
          emean = (A)sumx / (A)ne;
          const A estd = ne > 1 ? asqrt(i128A<A>(num) / ((A)ne * (A)(ne - 1))) : (A)0;
          put(p, row, Q_EDGE + E_II, i2d(sumx));
          put(p, row, Q_EDGE + E_MAX, i2d((long long)hi_c - ibias));
          put(p, row, Q_EDGE + E_MIN, i2d((long long)lo_c - ibias));
          putA(p, row, Q_EDGE + E_STD, estd);
          if (sv) sv[SV_ESTD] = to_d(estd);
        } else {
          const A sd = eh + el;
          emean = (A)fmn + sd / (A)ne;
          putA(p, row, Q_EDGE + E_II, (A)fmn * (A)ne + sd);
          put(p, row, Q_EDGE + E_MAX, f2d(Enc<T>::decf(hi_c)));
          put(p, row, Q_EDGE + E_MIN, f2d(Enc<T>::decf(lo_c)));
        }
        putA(p, row, Q_EDGE + E_MEAN, emean);
        p.big[b].est[0] = to_d(emean);
        p.big[b].est[1] = i2d(ne);
        if (sv) {
          sv[SV_EMEAN] = to_d(emean);
          sv[SV_ECNT] = i2d(ne);
        }
      }
    }
    // histogram features
    if (do_hist) {
      A hv[2] = {0, 0};
      const A inv = (A)1 / (A)n;
      for (int i = tid; i < p.hist_bins; i += BIG_NT) {
        const unsigned hc = __ldcg(reg + L.hist + i);
        if (hc) {
          const A pr = (A)hc * inv;
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
    if (range) hist_order_stats<T, A>(p, row, gvh, range, vmin, n, red, s_sc);
    __syncthreads();
  }
}

template <class T, int NDIM, class A>
__global__ void __launch_bounds__(BIG_NT, big_pass_minb<A>()) k_big_p2(KParams p) {
  using C = ClassBig;
  constexpr int NM = NDIM == 3 ? 20 : 10;
  constexpr int NV = 8 + 2 * NM;
  __shared__ double red[C::NW * RED_MAX];
  __shared__ A res[NV + 16];
  __shared__ int s_flag;
  __shared__ unsigned s_qc[C::NW * 64], s_qe[C::NW * 64];  // per-warp voxel queues
  const int tid = threadIdx.x, warp = tid >> 5;
  const unsigned long long ctr = *p.big_ctr;
  const int n_big = big_count(ctr);
  const unsigned n_units = big_units1(ctr);
  const unsigned need = p.need;
  const long long ibias = std::is_same<T, int16_t>::value ? 32768 : 0;
  const bool do_st = (need & (NEED_STATS | NEED_SAVE)) != 0;
  const bool do_mi = (need & (NEED_MOM_INT | NEED_SAVE)) != 0;
  const bool do_mb = (need & NEED_MOM_BIN) != 0;
  for (unsigned u = blockIdx.x; u < n_units; u += gridDim.x) {
    const int b = big_of_unit(p, n_big, u);
    const BigRoi br = p.big[b];
    const int chunk = (int)(u - br.u1);
    const RoiInfo r = p.rois[br.item];
    BigBox bx;
    bx.init(p, r, NDIM);
    const BigLayout L = big_layout(p, br.nch, br.nsp, br.range, r.n);
    unsigned* reg = p.arena + br.arena;
    const unsigned c0 = (unsigned)chunk * BIG_CHUNK, c1 = min(bx.cells, c0 + (unsigned)BIG_CHUNK);
    const double* st = p.big[b].st;
    const A mu_hi = (A)__ldcg(st + 0), mu_lo = (A)__ldcg(st + 1);
    // centre of the intensity-weighted moment sums: the weighted centroid if
    // it lies in the bounding box, else the binary one (as in the block classes)
    const double ci0 = __ldcg(st + 2), ci1 = __ldcg(st + 3), ci2 = __ldcg(st + 4);
    const double cb0 = __ldcg(st + 5), cb1 = __ldcg(st + 6), cb2 = __ldcg(st + 7);
    const bool inbox = ci0 >= 0 && ci0 <= bx.W - 1 && ci1 >= 0 && ci1 <= bx.H - 1 &&
                       (NDIM != 3 || (ci2 >= 0 && ci2 <= bx.D - 1));
    const A cx = (A)(inbox ? ci0 : cb0), cy = (A)(inbox ? ci1 : cb1), cz = (A)(inbox ? ci2 : cb2);
    const A bcx = (A)cb0, bcy = (A)cb1, bcz = (A)cb2;
    double* part = (double*)(reg + L.part2) + (size_t)chunk * (BIG_P2 / 2);
    // one pass: centred power sums and both moment sets, plain per-thread
    // sums over at most BIG_CHUNK / BIG_NT = 32 cells (as in the block
    // classes), then compensated block sums and two-sum chunk merges
    A acc[8], mi[NM], mb[NM];
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i] = 0;
#pragma unroll
    for (int i = 0; i < NM; ++i) mi[i] = mb[i] = 0;
    // float images: squared deviations of the edge voxels from their mean
    // (integer images finish their edge statistics exactly in pass 1)
    const bool do_edge = !Enc<T>::INTEGER && (need & NEED_EDGE) != 0;
    const A emean = do_edge ? (A)__ldcg(p.big[b].est + 0) : (A)0;
    A ev[1] = {0};
    chunk_voxels<T>(p, bx, c0, c1, s_qc + warp * 64, s_qe + warp * 64, [&](bool in, int x, int y, int z, unsigned e) {
      if (!in) return;
      const A v = Enc<T>::INTEGER ? (A)((long long)e - ibias) : decA<T, A>(e);
      if (do_edge && big_edge<NDIM>(p, bx, x, y, z)) ev[0] += (v - emean) * (v - emean);
      if (do_st) {
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
#pragma unroll
      for (int w = 0; w < 2; ++w) {
        if (!(w ? do_mb : do_mi)) continue;
        const A u0 = (A)x - (w ? bcx : cx), u1 = (A)y - (w ? bcy : cy), u2 = (A)z - (w ? bcz : cz);
        A px[4], py[4], pz[4];
        px[0] = w ? (A)1 : v;
        py[0] = pz[0] = 1;
#pragma unroll
        for (int q = 1; q < 4; ++q) {
          px[q] = px[q - 1] * u0;
          py[q] = py[q - 1] * u1;
          pz[q] = pz[q - 1] * u2;
        }
#pragma unroll
        for (int a = 0; a <= 3; ++a)
#pragma unroll
          for (int bb = 0; a + bb <= 3; ++bb)
#pragma unroll
            for (int cc = 0; cc <= (NDIM == 3 ? 3 - a - bb : 0); ++cc) {
              const A t = px[a] * py[bb] * pz[cc];
              if (w) mb[midx<NDIM>(a, bb, cc)] += t;
              else mi[midx<NDIM>(a, bb, cc)] += t;
            }
      }
    });
    block_sum<C, A, 8>(acc, red, res);
    if (tid < 8) part[tid] = do_st ? to_d(res[tid]) : 0.0;
    __syncthreads();
    block_sum<C, A, NM>(mi, red, res);
    if (tid < NM) part[8 + tid] = do_mi ? to_d(res[tid]) : 0.0;
    __syncthreads();
    block_sum<C, A, NM>(mb, red, res);
    if (tid < NM) part[8 + NM + tid] = do_mb ? to_d(res[tid]) : 0.0;
    __syncthreads();
    if (do_edge) {
      block_sum<C, A, 1>(ev, red, res);
      if (tid == 0) part[48] = to_d(res[0]);
    }
    if (!last_arrival(reg + L.ctr + 1, (unsigned)br.nch, &s_flag)) continue;

    // ---- last chunk: merge the partials in chunk order, finalise ----------
    if (do_edge && tid == 0) {
      A hi = 0, lo = 0;
      for (int ch = 0; ch < br.nch; ++ch) {
        const A x = (A)__ldcg((const double*)(reg + L.part2) + (size_t)ch * (BIG_P2 / 2) + 48);
        if constexpr (std::is_same<A, float>::value) {
          float sum, err;
          two_sum(hi, x, sum, err);
          hi = sum;
          lo += err;
        } else {
          hi += x;
        }
      }
      const double ne = __ldcg(p.big[b].est + 1);
      const A estd = ne > 1.5 ? asqrt((hi + lo) / (A)(ne - 1.0)) : (A)0;
      putA(p, p.table + (int64_t)br.item * p.n_col, Q_EDGE + E_STD, estd);
      if (need & NEED_SAVE) p.saved[(size_t)br.item * SV_WORDS + SV_ESTD] = to_d(estd);
    }
    if (tid < NV) {
      A hi = 0, lo = 0;
      for (int ch = 0; ch < br.nch; ++ch) {
        const A x = (A)__ldcg((const double*)(reg + L.part2) + (size_t)ch * (BIG_P2 / 2) + tid);
        if constexpr (std::is_same<A, float>::value) {
          float sum, err;
          two_sum(hi, x, sum, err);
          hi = sum;
          lo += err;
        } else {
          hi += x;
        }
      }
      res[tid] = hi + lo;
    }
    __syncthreads();
    const int n = (int)r.n;
    double* row = p.table + (int64_t)br.item * p.n_col;
    const int64_t bimg = (int64_t)(r.key >> 32);
    const A sumI = (A)__ldcg(st + 8), energy = (A)__ldcg(st + 9);
    const bool wvalid = sumI != 0;
    // the merged sums go to k_stats_final like those of the block classes
    double cd[6];
    for (int k = 0; k < 6; ++k) cd[k] = __ldcg(st + 2 + k);
    store_sacc<A>(p, br.item, NM, res, res + 8, res + 8 + NM, mu_hi + mu_lo, sumI, energy, cx, cy, cz, bcx, bcy, bcz,
                  cd);
    (void)n;
    (void)row;
    (void)bimg;
    (void)wvalid;
    __syncthreads();
  }
}

// cell (a, b), a <= b, of the upper-triangular co-occurrence matrix
__device__ inline unsigned tri_idx(unsigned a, unsigned b) { return b * (b + 1) / 2 + a; }
__device__ inline void tri_ab(unsigned f, unsigned& a, unsigned& b) {
  unsigned r = (unsigned)((sqrtf(8.f * (float)f + 1.f) - 1.f) * 0.5f);
  while (r * (r + 1) / 2 > f) --r;
  while ((r + 1) * (r + 2) / 2 <= f) ++r;
  b = r;
  a = f - r * (r + 1) / 2;
}

template <class T, int NDIM, class A>
__global__ void __launch_bounds__(BIG_NT) k_big_glcm(KParams p) {
  using C = ClassBig;
  extern __shared__ __align__(16) unsigned char smem[];
  const int ng = p.ng;
  const int n_off = p.n_dist * p.n_dirs;
  const int G = glcm_group(ng, n_off), n_grp = (n_off + G - 1) / G;
  const unsigned ntri = (unsigned)ng * (ng + 1) / 2, tstride = (ntri + 3) & ~3u;
  unsigned* tris = (unsigned*)smem;  // [G][tstride]
  unsigned* marg = tris + (size_t)G * tstride;
  unsigned* px = marg;
  unsigned* psum = marg + ng;       // index a + b
  unsigned* pdiff = marg + 3 * ng;  // index b - a
  uint16_t* rast = (uint16_t*)(marg + 4 * ng);  // [glcm_raster_cells] bins of padded cells
  __shared__ double red[C::NW * RED_MAX];
  __shared__ long long s_i64[GN + 4];
  __shared__ int s_flag;
  __shared__ unsigned s_qc[C::NW * 64];  // per-warp queues of ROI raster cells
  const int tid = threadIdx.x;
  const unsigned long long ctr = *p.big_ctr;
  const int n_big = big_count(ctr);
  const unsigned n_units = big_units2(ctr);
  const T* img = (const T*)p.img;
  constexpr uint16_t SENT = 0xFFFF;  // padded cell outside the ROI
  for (unsigned g = blockIdx.x; g < n_units; g += gridDim.x) {
    const int b = big_of_unit(p, n_big, g, true);
    const BigRoi br = p.big[b];
    const int loc = (int)(g - br.u2);
    const int sp = loc / n_grp, grp = loc - sp * n_grp;
    const RoiInfo r = p.rois[br.item];
    BigBox bx;
    bx.init(p, r, NDIM);
    const BigLayout L = big_layout(p, br.nch, br.nsp, br.range, r.n);
    unsigned* reg = p.arena + br.arena;
    const int o0 = grp * G, og = min(G, n_off - o0);
    const unsigned vmin = r.vmin, vmax = r.vmax;
    const float fmn = Enc<T>::decf(vmin), fmx = Enc<T>::decf(vmax);
    FastDiv fd;
    fd.init(vmax > vmin ? vmax - vmin : 1u);
    auto gbin = [&](unsigned e) -> unsigned {  // fixed bin number, n = Ng
      if (vmax <= vmin) return 0u;
      if constexpr (Enc<T>::INTEGER) return min(fd.div((unsigned)ng * (e - vmin)), (unsigned)(ng - 1));
      else return bin_float(Enc<T>::decf(e), fmn, fmx, ng);
    };
    for (unsigned i = tid; i < (unsigned)og * tstride; i += BIG_NT) tris[i] = 0;
    if (br.gsp > 0) {
      // ---- raster path: the span's padded cells plus a forward halo ----------
      // Padded box (W + 2d) x (H + 2d) [x (D + 2d)]; every unordered pair of
      // positions at offset +-o is counted once from its earlier cell in
      // raster order, at displacement |o| (the matrix is symmetric).
      const int dd = p.pad;
      const int Wp = bx.W + 2 * dd, Hp = bx.H + 2 * dd, Dp = NDIM == 3 ? bx.D + 2 * dd : 1;
      const unsigned pcells = (unsigned)Wp * (unsigned)Hp * (unsigned)Dp;
      const unsigned P0 = (unsigned)sp * (unsigned)br.gsp;
      const unsigned span = min((unsigned)br.gsp, pcells - P0);
      const unsigned len = min((unsigned)br.gsp + (unsigned)br.hal, pcells - P0);
      FastDiv fwp, fhp;
      fwp.init((unsigned)Wp);
      fhp.init((unsigned)Hp);
      int disp[MAX_DIRS];
#pragma unroll
      for (int j = 0; j < MAX_DIRS; ++j) {
        const int oj = o0 + (j < og ? j : 0);
        const int ds = (p.off[oj][2] * Hp + p.off[oj][1]) * Wp + p.off[oj][0];
        disp[j] = ds < 0 ? -ds : ds;
      }
      // stage: bins of the ROI's cells, SENT elsewhere (loads of BIG_U cells in flight)
      for (unsigned ib = 0; ib < len; ib += BIG_U * BIG_NT) {
        int lab[BIG_U];
        T val[BIG_U];
#pragma unroll
        for (int u = 0; u < BIG_U; ++u) {
          const unsigned i = ib + u * BIG_NT + tid;
          lab[u] = 0;
          if (i < len) {
            const unsigned P = P0 + i;
            const unsigned q = fwp.div(P), zq = fhp.div(q);
            const int x = (int)(P - q * (unsigned)Wp) - dd, y = (int)(q - zq * (unsigned)Hp) - dd;
            const int z = NDIM == 3 ? (int)zq - dd : 0;
            if (x >= 0 && y >= 0 && z >= 0 && x < bx.W && y < bx.H && z < bx.D) {
              const int64_t off = bx.origin + ((int64_t)z * p.ny + y) * p.nx + x;
              lab[u] = __ldg(p.mask + off);
              val[u] = __ldg(img + off);
            }
          }
        }
#pragma unroll
        for (int u = 0; u < BIG_U; ++u) {
          const unsigned i = ib + u * BIG_NT + tid;
          if (i < len) rast[i] = lab[u] == bx.label ? (uint16_t)gbin(Enc<T>::enc(val[u])) : SENT;
        }
      }
      __syncthreads();
      // count: every ROI cell of the span with its neighbour at each offset of
      // the group.  Each warp queues its ROI cells (raster indices) and runs
      // the offset loop on full warps of them; equal cells in consecutive
      // lanes merge into one atomic.
      unsigned* q = s_qc + (tid >> 5) * 64;
      const int lane = tid & 31;
      int qn = 0;  // warp-uniform
      auto count = [&](bool v, unsigned i) {
        const unsigned a = v ? rast[i] : SENT;
#pragma unroll
        for (int j = 0; j < MAX_DIRS; ++j) {
          if (j >= og) break;  // uniform
          unsigned key = 0xFFFFFFFFu;
          if (a != SENT) {
            const unsigned bb = rast[i + disp[j]];
            if (bb != SENT) key = a < bb ? tri_idx(a, bb) : tri_idx(bb, a);
          }
          const unsigned n = run_leader(key, 0xFFFFFFFFu);
          if (n) atomicAdd(&tris[(size_t)j * tstride + key], n);
        }
      };
      for (unsigned ib = 0; ib < span; ib += BIG_NT) {
        const unsigned i = ib + tid;
        const bool in = i < span && rast[i] != SENT;
        const unsigned bal = __ballot_sync(0xFFFFFFFFu, in);
        if (in) q[qn + __popc(bal & lanemask_lt())] = i;
        qn += __popc(bal);
        __syncwarp();
        if (qn >= 32) {
          count(true, q[lane]);
          __syncwarp();
          if (lane < qn - 32) q[lane] = q[32 + lane];
          __syncwarp();
          qn -= 32;
        }
      }
      count(lane < qn, lane < qn ? q[lane] : 0u);
      __syncthreads();
    } else {
      // ---- global-memory path (the halo does not fit): BIG_GSPAN chunks ------
      __syncthreads();
      const unsigned c0 = (unsigned)sp * BIG_GSPAN * BIG_CHUNK;
      const unsigned c1 = (unsigned)min((unsigned long long)bx.cells,
                                        (unsigned long long)c0 + (unsigned long long)BIG_GSPAN * BIG_CHUNK);
      chunk_cells<T>(p, bx, c0, c1, [&](bool in, int x, int y, int z, unsigned e, unsigned) {
        const unsigned a = in ? gbin(e) : 0u;
        const int64_t here = bx.origin + ((int64_t)z * p.ny + y) * p.nx + x;
        int nl[MAX_DIRS];
        T nv[MAX_DIRS];
#pragma unroll
        for (int j = 0; j < MAX_DIRS; ++j) {
          nl[j] = 0;
          if (j < og && in) {
            const int dx = p.off[o0 + j][0], dy = p.off[o0 + j][1], dz = p.off[o0 + j][2];
            const int X = x + dx, Y = y + dy, Z = z + dz;
            if (X >= 0 && Y >= 0 && Z >= 0 && X < bx.W && Y < bx.H && Z < bx.D) {
              const int64_t off = here + ((int64_t)dz * p.ny + dy) * p.nx + dx;
              nl[j] = __ldg(p.mask + off);
              nv[j] = __ldg(img + off);
            }
          }
        }
#pragma unroll
        for (int j = 0; j < MAX_DIRS; ++j) {
          if (j >= og) break;  // uniform
          unsigned key = 0xFFFFFFFFu;
          if (nl[j] == bx.label) {
            const unsigned bb = gbin(Enc<T>::enc(nv[j]));
            key = a < bb ? tri_idx(a, bb) : tri_idx(bb, a);
          }
          const unsigned n = run_leader(key, 0xFFFFFFFFu);
          if (n) atomicAdd(&tris[(size_t)j * tstride + key], n);
        }
      });
      __syncthreads();
    }
    if (br.nsp > 1) {  // add into the ROI's global triangles; the last span reduces them
      for (int j = 0; j < og; ++j) {
        unsigned* gt = reg + L.tri + (size_t)(o0 + j) * ntri;
        for (unsigned i = tid; i < ntri; i += BIG_NT)
          if (tris[(size_t)j * tstride + i]) atomicAdd(gt + i, tris[(size_t)j * tstride + i]);
      }
      if (!last_arrival(reg + L.ctr + 4 + grp, (unsigned)br.nsp, &s_flag)) continue;
      for (int j = 0; j < og; ++j) {
        const unsigned* gt = reg + L.tri + (size_t)(o0 + j) * ntri;
        for (unsigned i = tid; i < ntri; i += BIG_NT) tris[(size_t)j * tstride + i] = __ldcg(gt + i);
      }
      __syncthreads();
    }
    for (int j = 0; j < og; ++j) {
      const int oi = o0 + j;
      const unsigned* tri = tris + (size_t)j * tstride;
      // ---- GLCM sums of this offset from the complete triangle ---------------
      const bool dbg = p.dbg_roi == (int64_t)br.item;
      for (int i = tid; i < 4 * ng; i += BIG_NT) marg[i] = 0;
      __syncthreads();
      long long iv[GN];
#pragma unroll
      for (int k = 0; k < GN; ++k) iv[k] = 0;
      for (unsigned f = tid; f < ntri; f += BIG_NT) {
        const unsigned cnt = tri[f];
        if (!cnt) continue;
        unsigned a, bb;
        tri_ab(f, a, bb);
        atomicAdd(&px[a], cnt);
        atomicAdd(&px[bb], cnt);
        atomicAdd(&psum[a + bb], 2 * cnt);
        atomicAdd(&pdiff[bb - a], 2 * cnt);
        const long long Cm = 2 * (long long)cnt;
        const long long k = a + bb + 2, d = bb - a, k2 = k * k;
        iv[0] += Cm;
        iv[1] += Cm * k;
        iv[2] += Cm * k2;
        iv[3] += Cm * k2 * k;
        iv[4] += Cm * k2 * k2;
        iv[5] += Cm * d;
        iv[6] += Cm * d * d;
        iv[7] += (long long)cnt * ((long long)(a + 1) * (a + 1) + (long long)(bb + 1) * (bb + 1));
        const long long Cc = a == bb ? 2 * (long long)cnt : (long long)cnt;
        const long long mult = a == bb ? 1 : 2;
        iv[8] += mult * Cc * Cc;
        iv[9] += mult * clog_fx<A>(p.clog, (unsigned)Cc);
        iv[11] = Cc > iv[11] ? Cc : iv[11];
        if (dbg) {
          p.dbg_glcm[(int64_t)oi * ng * ng + a * ng + bb] = (unsigned)Cc;
          p.dbg_glcm[(int64_t)oi * ng * ng + bb * ng + a] = (unsigned)Cc;
        }
      }
      __syncthreads();
      long long Tl;
      {
        long long t1[1] = {0};
        for (int a = tid; a < ng; a += BIG_NT) t1[0] += px[a];
        block_sum_i64<C, 1>(t1, red, s_i64 + GN);
        Tl = s_i64[GN];
      }
      if (Tl == 0) {  // no pair for this offset: every feature NaN
        store_gacc(p, br.item, oi, iv, true);
        __syncthreads();
        continue;
      }
      // marginal entropies and inverse differences (exact fixed-point sums),
      // mutual information over the cells
      for (int a = tid; a < ng; a += BIG_NT)
        if (px[a]) iv[12] += clog_fx<A>(p.clog, px[a]);
      for (int k = tid; k < 2 * ng - 1; k += BIG_NT)
        if (psum[k]) iv[13] += clog_fx<A>(p.clog, psum[k]);
      for (int k = tid; k < ng; k += BIG_NT)
        if (pdiff[k]) {
          iv[14] += clog_fx<A>(p.clog, pdiff[k]);
          invdiff_fx<A>(p, pdiff[k], k, iv);
        }
      for (unsigned f = tid; f < ntri; f += BIG_NT) {
        const unsigned cnt = tri[f];
        if (!cnt) continue;
        unsigned a, bb;
        tri_ab(f, a, bb);
        const long long mult = a == bb ? 1 : 2;
        const unsigned Cc = a == bb ? 2 * cnt : cnt;
        iv[10] += mult * mi_fx<A>(Cc, Tl, px[a], px[bb]);
      }
      block_sum_glcm<C>(iv, red, s_i64);
      if (tid < GN) {  // entropy sums as numerators T log2 T - sum c log2 c
        const long long TL = tid == 9 || tid >= 12 ? tlog_fx(p.clog, Tl) : 0;
        s_i64[tid] = gacc_value(tid, s_i64[tid], TL);
      }
      store_gacc(p, br.item, oi, s_i64, false);  // features: k_glcm_final
      __syncthreads();
    }
  }
}

// NGTDM (Table S3 rows 246-250) and GLDM (rows 251-264) of big ROIs: units
// (ROI, chunk) as in the pass kernels.  A unit stages the bins of its chunk
// plus a halo of one plane and one row on each side (the Chebyshev-1
// reach), in the raster of the box padded by one sentinel cell, in shared
// memory, then visits each ROI voxel's neighbours there at fixed
// displacements; when the window exceeds NGT_WIN cells (very wide planes)
// the neighbours come from global memory instead, one plane of up to 9
// loads of each issued together.  The visit gives the NGTDM level sum and
// count and the GLDM dependence (1 + the neighbours at the voxel's own
// level).  NGTDM per-level counts and fixed-point sums, and the dense GLDM
// (level, dependence) counts stored after the window, gather in shared
// memory and go to the ROI's arena; the last chunk derives the features.
constexpr int NGT_WIN = 49152;  // window cells (2-byte bins) in dynamic shared memory

template <class T, int NDIM, class A>
__global__ void __launch_bounds__(BIG_NT, big_pass_minb<A>()) k_big_ngtdm(KParams p) {
  using C = ClassBig;
  extern __shared__ __align__(16) unsigned char smem[];
  uint16_t* rast = (uint16_t*)smem;  // [NGT_WIN]
  unsigned* sP = (unsigned*)(smem + 2 * NGT_WIN);  // [ng * nj] GLDM counts (launched with them when needed)
  __shared__ unsigned long long sS[256];
  __shared__ unsigned snL[256], slst[256];
  __shared__ double red[C::NW * RED_MAX];
  __shared__ long long s_i64[4];
  __shared__ A s_sc[16];
  __shared__ int s_flag;
  __shared__ unsigned s_qc[C::NW * 64], s_qe[C::NW * 64];  // per-warp voxel queues
  constexpr uint16_t SENT = 0xFFFF;
  const int tid = threadIdx.x;
  const unsigned long long ctr = *p.big_ctr;
  const int n_big = big_count(ctr);
  const unsigned n_units = big_units1(ctr);
  const int ng = p.ng;
  const int nj = NDIM == 3 ? 27 : 9;
  const bool do_ngtdm = (p.need & NEED_NGTDM) != 0, do_gldm = (p.need & NEED_GLDM) != 0;
  const T* img = (const T*)p.img;
  for (unsigned u = blockIdx.x; u < n_units; u += gridDim.x) {
    const int b = big_of_unit(p, n_big, u);
    const BigRoi br = p.big[b];
    const int chunk = (int)(u - br.u1);
    const RoiInfo r = p.rois[br.item];
    BigBox bx;
    bx.init(p, r, NDIM);
    const BigLayout L = big_layout(p, br.nch, br.nsp, br.range, r.n);
    unsigned* reg = p.arena + br.arena;
    unsigned long long* gS = (unsigned long long*)(reg + L.ngt);
    unsigned* gn = (unsigned*)(gS + ng);
    unsigned* gP = reg + L.gld;  // [ng * nj]
    const unsigned c0 = (unsigned)chunk * BIG_CHUNK, c1 = min(bx.cells, c0 + (unsigned)BIG_CHUNK);
    const unsigned vmin = r.vmin, vmax = r.vmax;
    const float fmn = Enc<T>::decf(vmin), fmx = Enc<T>::decf(vmax);
    FastDiv fd;
    fd.init(vmax > vmin ? vmax - vmin : 1u);
    auto gbin = [&](unsigned e) -> int {  // fixed bin number, n = Ng
      if (vmax <= vmin) return 0;
      if constexpr (Enc<T>::INTEGER) return (int)min(fd.div((unsigned)ng * (e - vmin)), (unsigned)(ng - 1));
      else return (int)bin_float(Enc<T>::decf(e), fmn, fmx, ng);
    };
    for (int i = tid; i < ng; i += BIG_NT) {
      sS[i] = 0;
      snL[i] = 0;
    }
    if (do_gldm)
      for (int i = tid; i < ng * nj; i += BIG_NT) sP[i] = 0;
    // window in the padded box (one sentinel cell around the bounding box),
    // so that every neighbour is a fixed displacement without bounds tests
    const int Wp = bx.W + 2, Hp = bx.H + 2;
    const unsigned plane = (unsigned)Wp * (unsigned)Hp;
    const unsigned pcells = plane * (unsigned)(NDIM == 3 ? bx.D + 2 : 1);
    auto pidx = [&](unsigned c) -> unsigned {  // padded index of bounding-box cell c
      int x, y, z;
      bx.offset(c, x, y, z, p);
      return ((unsigned)(NDIM == 3 ? z + 1 : 0) * (unsigned)Hp + (unsigned)(y + 1)) * (unsigned)Wp + (unsigned)(x + 1);
    };
    const unsigned halo = (NDIM == 3 ? plane : 0u) + (unsigned)Wp + 1u;
    const unsigned p_lo = pidx(c0), p_hi = pidx(c1 - 1) + 1u;
    const unsigned w0 = p_lo > halo ? p_lo - halo : 0u, w1 = min(pcells, p_hi + halo);
    if (w1 - w0 <= (unsigned)NGT_WIN) {
      // ---- shared-memory window: bins of padded cells [w0, w1), SENT off the ROI ----
      FastDiv fwp, fhp;
      fwp.init((unsigned)Wp);
      fhp.init((unsigned)Hp);
      for (unsigned ib = w0; ib < w1; ib += BIG_U * BIG_NT) {
        int lab[BIG_U];
        T val[BIG_U];
#pragma unroll
        for (int q = 0; q < BIG_U; ++q) {  // loads of BIG_U cells in flight
          const unsigned P = ib + q * BIG_NT + tid;
          lab[q] = 0;
          if (P < w1) {
            const unsigned rq = fwp.div(P), zq = fhp.div(rq);
            const int x = (int)(P - rq * (unsigned)Wp) - 1, y = (int)(rq - zq * (unsigned)Hp) - 1;
            const int z = NDIM == 3 ? (int)zq - 1 : 0;
            if (x >= 0 && y >= 0 && z >= 0 && x < bx.W && y < bx.H && z < bx.D) {
              const int64_t off = bx.origin + ((int64_t)z * p.ny + y) * p.nx + x;
              lab[q] = __ldg(p.mask + off);
              val[q] = __ldg(img + off);
            }
          }
        }
#pragma unroll
        for (int q = 0; q < BIG_U; ++q) {
          const unsigned P = ib + q * BIG_NT + tid;
          if (P < w1) rast[P - w0] = lab[q] == bx.label ? (uint16_t)gbin(Enc<T>::enc(val[q])) : SENT;
        }
      }
      __syncthreads();
      for (unsigned c = c0 + tid; c < c1; c += BIG_NT) {
        const int here = (int)(pidx(c) - w0);
        const unsigned a = rast[here];
        if (a == SENT) continue;
        int sum = 0, cnt = 0, same = 0;
#pragma unroll
        for (int dz = (NDIM == 3 ? -1 : 0); dz <= (NDIM == 3 ? 1 : 0); ++dz)
#pragma unroll
          for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
              if (dx == 0 && dy == 0 && dz == 0) continue;
              const unsigned bnb = rast[here + (dz * Hp + dy) * Wp + dx];
              if (bnb != SENT) {
                sum += (int)bnb + 1;
                ++cnt;
              }
              same += bnb == a;
            }
        if (do_ngtdm && cnt) {
          atomicAdd(&snL[a], 1u);
          atomicAdd(&sS[a], ngtdm_term((int)a + 1, sum, cnt));
        }
        if (do_gldm) atomicAdd(&sP[a * nj + same], 1u);
      }
    } else {
      // ---- neighbours from global memory ----
      __syncthreads();
      chunk_voxels<T>(p, bx, c0, c1, s_qc + (tid >> 5) * 64, s_qe + (tid >> 5) * 64,
                      [&](bool in, int x, int y, int z, unsigned e) {
        const int64_t here = bx.origin + ((int64_t)z * p.ny + y) * p.nx + x;
        const int a = in ? gbin(e) : -1;
        int sum = 0, cnt = 0, same = 0;
#pragma unroll 1
        for (int dz = (NDIM == 3 ? -1 : 0); dz <= (NDIM == 3 ? 1 : 0); ++dz) {
          if (!in || z + dz < 0 || z + dz >= bx.D) continue;
          int lab[9];
          T val[9];
#pragma unroll
          for (int q = 0; q < 9; ++q) {  // every load of the plane first
            const int dy = q / 3 - 1, dx = q % 3 - 1;
            lab[q] = 0;
            const bool inb = !(dz == 0 && dy == 0 && dx == 0) && y + dy >= 0 && y + dy < bx.H && x + dx >= 0 &&
                             x + dx < bx.W;
            if (inb) {
              const int64_t o = here + ((int64_t)dz * p.ny + dy) * p.nx + dx;
              lab[q] = __ldg(p.mask + o);
              val[q] = __ldg(img + o);
            }
          }
#pragma unroll
          for (int q = 0; q < 9; ++q)
            if (lab[q] == bx.label) {
              const int lq = gbin(Enc<T>::enc(val[q]));
              sum += lq + 1;
              ++cnt;
              same += lq == a;
            }
        }
        if (do_ngtdm && cnt) {
          atomicAdd(&snL[a], 1u);
          atomicAdd(&sS[a], ngtdm_term(a + 1, sum, cnt));
        }
        if (do_gldm && in) atomicAdd(&sP[a * nj + same], 1u);
      });
    }
    __syncthreads();
    if (do_ngtdm)
      for (int i = tid; i < ng; i += BIG_NT)
        if (snL[i]) {
          atomicAdd(gn + i, snL[i]);
          atomicAdd(gS + i, sS[i]);
        }
    if (do_gldm)
      for (int i = tid; i < ng * nj; i += BIG_NT)
        if (sP[i]) atomicAdd(gP + i, sP[i]);
    if (!last_arrival(reg + L.ctr + 2, (unsigned)br.nch, &s_flag)) continue;
    double* row = p.table + (int64_t)br.item * p.n_col;
    if (do_ngtdm) {
      for (int i = tid; i < ng; i += BIG_NT) {
        snL[i] = __ldcg(gn + i);
        sS[i] = __ldcg(gS + i);
      }
      __syncthreads();
      ngtdm_features<C, A>(p, row, ng, snL, sS, slst, red, s_sc, s_i64);  // ends with a barrier
    }
    if (do_gldm) {
      // column sums and the entropy share from the ROI's dense counts, then
      // the per-level sums read back by the feature pass
      unsigned* scol = slst;  // [nj]
      if (tid < nj) scol[tid] = 0;
      __syncthreads();
      long long ent = 0;
      for (int i = tid; i < ng * nj; i += BIG_NT) {
        const unsigned c = __ldcg(gP + i);
        if (c) {
          atomicAdd(&scol[i % nj], c);
          ent += clog_fx<A>(p.clog, c);
        }
      }
      __syncthreads();
      gldm_features<C, A>(
          p, row, ng, nj,
          [&](int a, unsigned long long& r, unsigned long long& c2, unsigned long long& cm) {
            r = 0;
            c2 = 0;
            cm = 0;
            for (int j = 0; j < nj; ++j) {
              const unsigned long long c = __ldcg(gP + a * nj + j);
              r += c;
              c2 += c * (unsigned long long)((j + 1) * (j + 1));
              cm += c * inv_sq_fx((unsigned)(j + 1));
            }
          },
          scol, ent, red, s_sc, s_i64);
    }
  }
}

// Order statistics of big ROIs without a value histogram (float images, and
// 16-bit ROIs whose value range exceeds their pixel count): one block per ROI
// compacts the values in raster order and sorts them with an LSD radix sort
// in the ROI's arena region (stable ranks from 8 ballots per digit, as in the
// block path).
constexpr int BIG_SORT_SMEM = 23552;  // values sorted in shared memory (two buffers, 188 KB)

template <class T, class A>
__global__ void __launch_bounds__(BIG_NT) k_big_order(KParams p, int ndim) {
  using C = ClassBig;
  extern __shared__ __align__(16) unsigned char smem_o[];
  __shared__ unsigned cnt[C::NW * 256];
  __shared__ unsigned dtot[256];
  __shared__ double red[C::NW * RED_MAX];
  __shared__ unsigned s_wc[C::NW], s_wb[C::NW + 1];
  __shared__ double s_sd[4];
  __shared__ unsigned s_bnd[4];
  __shared__ A s_sc[16];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n_big = big_count(*p.big_ctr);
  const T* img = (const T*)p.img;
  for (int b = blockIdx.x; b < n_big; b += gridDim.x) {
    const BigRoi br = p.big[b];
    if (br.range) continue;  // value histogram path (pass 1)
    const RoiInfo r = p.rois[br.item];
    BigBox bx;
    bx.init(p, r, ndim);
    const BigLayout L = big_layout(p, br.nch, br.nsp, br.range, r.n);
    const int n = (int)r.n;
    // ping-pong buffers in shared memory when the values fit, else in the
    // ROI's arena region
    const bool in_smem = n <= BIG_SORT_SMEM;
    unsigned* src = in_smem ? (unsigned*)smem_o : p.arena + br.arena + L.fsort;
    unsigned* dst = in_smem ? src + BIG_SORT_SMEM : src + n;
    // compaction in raster order
    if (tid == 0) s_wb[C::NW] = 0;
    __syncthreads();
    for (unsigned base = 0; base < bx.cells; base += BIG_NT) {
      const unsigned c = base + tid;
      bool in = false;
      unsigned e = 0;
      if (c < bx.cells) {
        int x, y, z;
        const int64_t off = bx.offset(c, x, y, z, p);
        in = __ldg(p.mask + off) == bx.label;
        if (in) e = Enc<T>::enc(__ldg(img + off));
      }
      const unsigned bal = __ballot_sync(0xFFFFFFFFu, in);
      if (lane == 0) s_wc[warp] = __popc(bal);
      __syncthreads();
      if (tid == 0) {
        unsigned acc = s_wb[C::NW];
        for (int w = 0; w < C::NW; ++w) {
          s_wb[w] = acc;
          acc += s_wc[w];
        }
        s_wb[C::NW] = acc;
      }
      __syncthreads();
      if (in) {
        const unsigned pos = s_wb[warp] + __popc(bal & lanemask_lt());
        if (pos < (unsigned)n) src[pos] = e;
      }
      __syncthreads();
    }
    if (tid == 0 && s_wb[C::NW] != (unsigned)n) atomicOr(p.err, E_INTERNAL);
    __threadfence_block();
    __syncthreads();
    // LSD radix sort, 8-bit digits; warp w owns the segment [w seg, (w+1) seg)
    const int seg = (((n + C::NW - 1) / C::NW) + 31) & ~31;
    const int lo = min(n, warp * seg), hi = min(n, lo + seg);
    for (int shift = 0; shift < Enc<T>::BITS; shift += 8) {
      for (int i = tid; i < C::NW * 256; i += BIG_NT) cnt[i] = 0;
      __syncthreads();
      for (int i0 = lo; i0 < hi; i0 += 32) {  // digit counts per warp
        const int i = i0 + lane;
        const bool act = i < hi;
        const unsigned dg = act ? (src[i] >> shift) & 255u : 0u;
        unsigned peers = __ballot_sync(0xFFFFFFFFu, act);
#pragma unroll
        for (int bit = 0; bit < 8; ++bit) {
          const unsigned bb = __ballot_sync(0xFFFFFFFFu, (dg >> bit) & 1u);
          peers &= ((dg >> bit) & 1u) ? bb : ~bb;
        }
        if (act && __popc(peers & lanemask_lt()) == 0) cnt[warp * 256 + dg] += __popc(peers);
        __syncwarp();
      }
      __syncthreads();
      for (int d = tid; d < 256; d += BIG_NT) {
        unsigned t = 0;
        for (int w = 0; w < C::NW; ++w) t += cnt[w * 256 + d];
        dtot[d] = t;
      }
      __syncthreads();
      if (warp == 0) warp_exclusive_scan(dtot, 256);
      __syncthreads();
      for (int d = tid; d < 256; d += BIG_NT) {
        unsigned run = dtot[d];
        for (int w = 0; w < C::NW; ++w) {
          const unsigned c = cnt[w * 256 + d];
          cnt[w * 256 + d] = run;
          run += c;
        }
      }
      __syncthreads();
      for (int i0 = lo; i0 < hi; i0 += 32) {  // stable scatter, same walk
        const int i = i0 + lane;
        const bool act = i < hi;
        const unsigned k = act ? src[i] : 0u;
        const unsigned dg = (k >> shift) & 255u;
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
          dst[b0 + before] = k;
          if (before == 0) cnt[warp * 256 + dg] = b0 + __popc(peers);
        }
        __syncwarp();
      }
      __threadfence_block();
      __syncthreads();
      unsigned* t = src;
      src = dst;
      dst = t;
    }
    double* row = p.table + (int64_t)br.item * p.n_col;
    order_tail<T, C, A>(p, row, src, n, red, s_sd, s_bnd, s_sc);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// launchers (kernel templates are launched only from the translation unit
// that instantiates them)

template <auto K>
static cudaError_t big_launch(int smem, int nsm, const KParams& p, cudaStream_t st) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  static int configured[64] = {0};
  if (smem > 0 && (dev >= 64 || configured[dev] < smem)) {
    e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    if (dev < 64) configured[dev] = smem;
  }
  int nb = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, K, BIG_NT, smem);
  if (e != cudaSuccess) return e;
  if (nb < 1) return cudaErrorInvalidConfiguration;
  K<<<nb * nsm, BIG_NT, smem, st>>>(p);
  return cudaGetLastError();
}

template <class T, int NDIM, class A>
cudaError_t launch_big_one(const KParams& p, int nsm, cudaStream_t st) {
  cudaError_t e = big_launch<k_big_zero<T>>(0, nsm, p, st);
  if (e != cudaSuccess) return e;
  const int smem1 = 4 * (((p.hist_bins + 3) & ~3) + VH_SMEM);
  if ((e = big_launch<k_big_p1<T, NDIM, A>>(smem1, nsm, p, st)) != cudaSuccess) return e;
  if ((e = big_launch<k_big_p2<T, NDIM, A>>(0, nsm, p, st)) != cudaSuccess) return e;
  if (p.need & NEED_GLCM) {
    if ((e = big_launch<k_big_glcm<T, NDIM, A>>(GLCM_SMEM_BYTES, nsm, p, st)) != cudaSuccess) return e;
  }
  if (p.need & (NEED_NGTDM | NEED_GLDM)) {
    const int smem = 2 * NGT_WIN + ((p.need & NEED_GLDM) ? 4 * p.ng * (NDIM == 3 ? 27 : 9) : 0);
    if ((e = big_launch<k_big_ngtdm<T, NDIM, A>>(smem, nsm, p, st)) != cudaSuccess) return e;
  }
  if (p.need & NEED_ORDER) {
    auto kern = k_big_order<T, A>;
    const int smem = 8 * BIG_SORT_SMEM;
    static int configured[64] = {0};
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if (dev >= 64 || !configured[dev]) {
      if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess) return e;
      if (dev < 64) configured[dev] = 1;
    }
    int nb = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, BIG_NT, smem)) != cudaSuccess) return e;
    kern<<<(nb > 0 ? nb : 1) * nsm, BIG_NT, smem, st>>>(p, NDIM);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <class T>
cudaError_t launch_big_t(const KParams& p, int fp64, int nsm, cudaStream_t st) {
  if (p.ndim == 3) return fp64 ? launch_big_one<T, 3, double>(p, nsm, st) : launch_big_one<T, 3, float>(p, nsm, st);
  return fp64 ? launch_big_one<T, 2, double>(p, nsm, st) : launch_big_one<T, 2, float>(p, nsm, st);
}

}  // namespace nyx
