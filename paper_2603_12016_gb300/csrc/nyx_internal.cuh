// nyx_internal.cuh -- device-side data structures and helpers shared by the
// kernels of libnyxgpu (GB300 / sm_103a).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "nyx.h"

namespace nyx {

// ---------------------------------------------------------------------------
// device error word bits (reported through nyx_sync_status)
enum : unsigned {
  E_BAD_LABEL = 1u,   // negative label in the mask
  E_NONFINITE = 2u,   // NaN/Inf float pixel inside an ROI
  E_HASH_FULL = 4u,   // more distinct labels than the plan's label table holds
  E_ROI_CAP = 8u,     // more ROIs than cap_roi
  E_TOO_LARGE = 16u,  // an ROI exceeds the per-ROI size limits of every path
  E_TIMEOUT = 32u,    // a bounded wait ran out
  E_SORT_CAP = 64u,   // more ROIs than the label sort handles
  E_INTERNAL = 128u,  // staged pixel count disagrees with the scan (never expected)
};

constexpr unsigned long long EMPTY_KEY = 0xFFFFFFFFFFFFFFFFull;
constexpr int MAX_DIST = 8;
constexpr int MAX_DIRS = 13;
constexpr int NGLCM = 30;
constexpr int SORT_CAP = 16384;  // ROIs sortable by the single-block label sort
constexpr int N_BLOCK_CLASSES = NYX_N_CLASSES;  // warp, small, medium, large block classes
constexpr int BIG_CLASS = N_BLOCK_CLASSES;      // class index of the multi-block path
constexpr int GI_HOST = 12, GF_HOST = 8;  // GLCM accumulator sizes (int64 sums, float sums)
// c log2 c (2^-24 units) of every count c < CLOG_N comes from the plan's table,
// rounded once from FP64: it covers every count of the block classes (at
// most 2 x 8,192 pairs per offset)
constexpr int CLOG_N = 16385;
// round(2^63 / s^2) of every run length / zone area up to RZ_STAB (the
// largest of the block classes) comes from the plan's table
constexpr int RZ_STAB = 16384;

// Per (image, label) accumulator filled by the label scan.  Intensities use
// an order-preserving uint32 encoding so that min/max are integer atomics.
struct SlotAcc {
  unsigned count;
  unsigned vmin, vmax;
  int xmin, xmax, ymin, ymax, zmin, zmax;
  unsigned pad[3];
};

// Per ROI, in output (ascending key) order.
struct RoiInfo {
  unsigned long long key;  // image << 32 | label
  unsigned n;              // pixel count
  int x0, y0, z0, w, h, d; // bounding box (image coordinates, extents)
  unsigned vmin, vmax;     // encoded intensity range
  int cls;                 // processing class
  int pad;
};

// Per ROI of the multi-block class (class 3), registered by k_setup.  The
// ROI's bounding box is cut into chunks of BIG_CHUNK raster cells; pass units
// are (ROI, chunk), GLCM units (ROI, BIG_GSPAN chunks, group of offsets whose
// triangles fit in shared memory together).  Everything the ROI needs in
// global memory (counters, histograms, per-offset co-occurrence
// triangles, per-chunk partial sums, sort buffers) is one region of the big
// arena starting at word `arena`.
constexpr int BIG_CHUNK = 16384;   // pass-unit cells (32 per thread of a 512-thread block)
constexpr int BIG_GSPAN = 4;       // fallback GLCM unit: this many pass chunks
constexpr int GLCM_TRI_WORDS = 30720;   // shared-memory words for the co-occurrence triangles of a GLCM unit
constexpr int GLCM_SMEM_BYTES = 200 * 1024;  // dynamic shared memory of a GLCM unit (triangles, marginals, raster)

// Offsets whose triangles fit in one GLCM unit's shared memory together.
__host__ __device__ inline int glcm_group(int ng, int n_off) {
  const int tri = ng * (ng + 1) / 2;
  const int padded = (tri + 3) & ~3;
  int g = padded > 0 ? GLCM_TRI_WORDS / padded : n_off;
  if (g < 1) g = 1;
  if (g > MAX_DIRS) g = MAX_DIRS;  // per-lane neighbour arrays hold one direction set
  return g < n_off ? g : n_off;
}

// u16 raster cells left for a GLCM unit next to its triangles and marginals.
__host__ __device__ inline int glcm_raster_cells(int ng, int n_off) {
  const int g = glcm_group(ng, n_off);
  const int tstride = ((ng * (ng + 1) / 2) + 3) & ~3;
  return (GLCM_SMEM_BYTES - 4 * g * tstride - 16 * ng) / 2;
}
struct BigRoi {
  int item;                 // ROI index (output row)
  int nch;                  // bounding-box chunks
  unsigned u1;              // first pass unit (prefix over the big ROIs)
  unsigned range;           // value-histogram words (16-bit order statistics), else 0
  unsigned long long arena; // word offset of the ROI's arena region
  unsigned u2;              // first GLCM unit (prefix over the big ROIs)
  int nsp;                  // GLCM spans
  int gsp;                  // padded raster cells per GLCM span; 0 = global-memory neighbours
  int hal;                  // raster halo: the largest neighbour displacement in padded cells
  double st[10];            // pass-1 scalars: mean (hi, lo), centroids, sum I, energy
  double est[2];            // edge pixels: mean, count (float images finish their deviation in pass 2)
};

// ---------------------------------------------------------------------------
// output quantity index space.  The host maps each quantity to an output
// column (or -1) in col_map[].
enum : int {
  Q_LABEL = 0, Q_IMAGE, Q_AREA, Q_BB_X, Q_BB_Y, Q_BB_Z, Q_BB_W, Q_BB_H, Q_BB_D, Q_CEN_X, Q_CEN_Y, Q_CEN_Z,
  Q_STATS = 12,
  N_STATS = 41,
  Q_MOM = Q_STATS + N_STATS,          // + (weighting*5 + family)*20 + k
  Q_GLCM_D = Q_MOM + 200,             // + di*30 + g
  Q_GLCM_O = Q_GLCM_D + MAX_DIST * NGLCM,  // + (di*13 + dir)*30 + g
  Q_EDGE = Q_GLCM_O + MAX_DIST * MAX_DIRS * NGLCM,  // + e (edge intensity statistics)
  N_EDGE = 5,
  Q_NGTDM = Q_EDGE + N_EDGE,          // + k (NGTDM features)
  N_NGTDM = 5,
  Q_GLDM = Q_NGTDM + N_NGTDM,         // + k (GLDM features)
  N_GLDM = 14,
  Q_GLRLM = Q_GLDM + N_GLDM,          // + k (GLRLM features, direction means)
  N_GLRLM = 16,
  Q_GLSZM = Q_GLRLM + N_GLRLM,        // + k (GLSZM features)
  N_GLSZM = 18,
  Q_TOTAL = Q_GLSZM + N_GLSZM
};

// NGTDM features (Table S3 rows 246-250), index within Q_NGTDM
enum : int { NT_COARSENESS = 0, NT_CONTRAST, NT_BUSYNESS, NT_COMPLEXITY, NT_STRENGTH };

// GLDM features (Table S3 rows 251-264), index within Q_GLDM
enum : int {
  GD_SDE = 0, GD_LDE, GD_GLN, GD_DN, GD_DNN, GD_GLV, GD_DV, GD_DE, GD_LGLE, GD_HGLE, GD_SDLGLE, GD_SDHGLE,
  GD_LDLGLE, GD_LDHGLE
};

// edge intensity statistics (Table S1 rows 3-7, Table S5), index within Q_EDGE
enum : int { E_II = 0, E_MAX, E_MIN, E_MEAN, E_STD };

// first-order statistics (Table S1 / S5), index within Q_STATS
enum : int {
  S_MEAN = 0, S_MIN, S_MAX, S_RANGE, S_VAR, S_VAR_B, S_STD, S_STD_B, S_SKEW, S_KURT, S_EXKURT, S_HSKEW, S_HFLAT,
  S_ENERGY, S_RMS, S_SE, S_MAD, S_MEDAD, S_II, S_WCX, S_WCY, S_WCZ, S_MD, S_COV, S_COVERED, S_PIU, S_MEDIAN,
  S_P01, S_P10, S_P25, S_P75, S_P90, S_P99, S_IQR, S_QCOD, S_RMEAN, S_RMAD, S_MODE, S_MODE_PROB, S_ENTROPY,
  S_UNIFORMITY
};

// moment families
enum : int { F_M = 0, F_MU = 1, F_ETA = 2, F_NU = 3, F_HU = 4 };

// GLCM features (Table S3 rows 140-174 without AVEAMP), index g
enum : int {
  G_ASM = 0, G_ACOR, G_CLUPROM, G_CLUSHADE, G_CLUTEND, G_CONTRAST, G_CORR, G_DIFAVE, G_DIFENTRO, G_DIFVAR, G_DIS,
  G_ENERGY, G_ENTROPY, G_HOM1, G_HOM2, G_IDM, G_INFOMEAS1, G_INFOMEAS2, G_IDMN, G_ID, G_IDN, G_IV, G_JAVE, G_JE,
  G_JMAX, G_SUMAVE, G_SUMENT, G_JVAR, G_SUMVAR, G_VARIANCE
};

// computation groups derived from the feature selection
enum : unsigned {
  NEED_STATS = 1u,    // central power sums of the intensities
  NEED_ORDER = 2u,    // sorted values (percentiles, mode, robust stats)
  NEED_HIST = 4u,     // entropy / uniformity histogram
  NEED_MOM_INT = 8u,  // intensity-weighted moments
  NEED_MOM_BIN = 16u, // binary moments
  NEED_GLCM = 32u,
  NEED_SAVE = 64u,    // keep per-ROI state for the backward pass
  NEED_EDGE = 128u,   // edge intensity statistics
  NEED_NGTDM = 256u,  // neighbourhood grey-tone difference matrix
  NEED_GLDM = 512u,   // grey-level dependence matrix
  NEED_GLRLM = 1024u, // grey-level run-length matrices
  NEED_GLSZM = 2048u, // grey-level size-zone matrix
};

// saved per-ROI state for the backward pass (FP64 words per ROI)
enum : int {
  SV_N = 0, SV_MEAN, SV_M2, SV_M3, SV_M4, SV_M5, SV_M6, SV_SGN, SV_ENERGY, SV_SUMI,
  SV_CX, SV_CY, SV_CZ,          // intensity centroid, ROI-local
  SV_BX, SV_BY, SV_BZ,          // binary centroid, image coordinates
  SV_X0, SV_Y0, SV_Z0,          // bounding-box origin
  SV_MU = 19,                   // 20 central intensity moments
  SV_EMEAN = SV_MU + 20,        // edge pixels: mean, unbiased deviation, count
  SV_ESTD, SV_ECNT,
  SV_WORDS
};

// Kernel parameters (by value).
struct KParams {
  const void* img;
  const int32_t* mask;
  int64_t nx, ny, nz, rows_total;  // rows_total = batch * nz * ny
  int batch, ndim, dtype, vec;     // vec: 16-byte vector loads are legal
  int ng, n_dist, n_dirs, per_offset, hist_bins, pad;
  int dists[MAX_DIST];
  int off[MAX_DIST * MAX_DIRS][3]; // (dx, dy, dz) of every offset
  unsigned need;
  const int* col_map;
  int n_col;
  // label table
  unsigned long long* keys;
  SlotAcc* slots;
  unsigned hmask;                  // capacity - 1 (power of two)
  int* slot_list;
  unsigned* n_used;
  unsigned* img_vmin;
  unsigned* img_vmax;
  // ROI table
  unsigned long long* sorted_keys;
  RoiInfo* rois;
  int* slot_dense;
  int* queue;                      // [N_BLOCK_CLASSES][max_rois], one per block class
  unsigned* qlen;                  // [N_BLOCK_CLASSES]
  unsigned* qhead;                 // [N_BLOCK_CLASSES]
  unsigned* n_roi;                 // device ROI count
  unsigned* err;
  int64_t max_rois, cap_roi;
  double* table;
  int64_t* n_roi_out;
  double* saved;
  // debug hook
  int64_t dbg_roi;
  unsigned* dbg_glcm;              // [n_off][ng*ng]
  // class limits (pixels, padded raster cells): 0 warp path, 1 small
  // block path, 2 medium block path, 3 large block path
  int lim_pix[N_BLOCK_CLASSES], lim_cells[N_BLOCK_CLASSES];
  // multi-block class
  BigRoi* big;                     // [max_rois]
  unsigned long long* big_ctr;     // (n_big << 44) | (n_pass_units << 22) | n_glcm_units
  unsigned long long* big_used;    // [0] arena words handed out, [1] pass units, [2] GLCM units
  unsigned* arena;
  unsigned long long arena_cap;    // words
  unsigned char* gacc;             // [max rows][n_off] GLCM accumulators
  unsigned char* sacc;             // [max rows] statistics / moment sums for k_stats_final
  const float* wtab_f;             // [Ng][5] inverse-difference weights 1/(1+k), 1/(1+k^2),
  const double* wtab_d;            //   1/(1+k/Ng), 1/(1+k^2/Ng^2), 1/k^2 (0 at k = 0)
  const long long* clog;           // [CLOG_N] c log2 c in units of 2^-24, rounded once from FP64 (128 KB)
  // label scan over rows [scan_row0, scan_row1) of the batch (scan_row1 = 0:
  // all rows); the mosaic path scans each band of tiles as it arrives
  int64_t scan_row0, scan_row1;
  int scan_rpt;                    // label-scan rows per warp (tile height / 8); 0: chosen by tile count
  int scan_stage;                  // label-scan staging: 0 bulk tensor copies where legal, 1 register loads
  unsigned long long* sort_tmp;    // key buffer of the key sorts [max_rois]
  // GLRLM / GLSZM: work counters of the two block tiers; zone parents and
  // areas of the multi-block ROIs, one word per image pixel (GLSZM only)
  unsigned* rz_head;               // [N_BLOCK_CLASSES]
  const unsigned long long* rz_qi; // [257] round(2^63 / i^2), levels i = 1..256
  const unsigned long long* rz_qs; // [RZ_STAB + 1] round(2^63 / s^2), sizes s = 1..RZ_STAB
  unsigned* ztag;                  // (multi-block ROI index + 1) << 9 | level of its pixels, else 0
  unsigned* zpar;
  unsigned* zcnt;
};

// Fields of the packed big-ROI counter (one atomic hands out the big-ROI
// index, its first pass unit and its first GLCM unit together).
__host__ __device__ inline int big_count(unsigned long long c) { return (int)(c >> 44); }
__host__ __device__ inline unsigned big_units1(unsigned long long c) { return (unsigned)(c >> 22) & 0x3FFFFFu; }
__host__ __device__ inline unsigned big_units2(unsigned long long c) { return (unsigned)c & 0x3FFFFFu; }

// Word offsets (u32 units) of the parts of one big ROI's arena region: pass
// counters, histograms, per-offset co-occurrence triangles (multi-chunk ROIs),
// NGTDM per-level sums, GLDM counts (level-major, 9 / 27 dependences),
// per-chunk partial sums, float sort buffers.  The prefix [0, zero_end) must
// be zero when the passes start.
constexpr int BIG_P1 = 38;   // pass-1 partial per chunk: 9 int64 + 5 doubles + 5 edge words (8 bytes each)
constexpr int BIG_P2 = 98;   // pass-2 partial per chunk: 48 doubles + the edge squared deviations
struct BigLayout {
  unsigned long long ctr, hist, vhist, tri, ngt, gld, rzh, zero_end, part1, part2, fsort, total;
};

// GLRLM / GLSZM sets of the selection: one per unit direction, one for the zones
__host__ __device__ inline int rz_sets(const KParams& p) {
  return ((p.need & NEED_GLRLM) ? (p.ndim == 3 ? 13 : 4) : 0) + ((p.need & NEED_GLSZM) ? 1 : 0);
}
// Slots of each set's item table of a multi-block ROI: a set holds at most
// min(n, sqrt(2 n Ng)) distinct (level, size) keys (its sizes sum to at most
// n), kept at a load of at most two thirds; a power of two.
__host__ __device__ inline unsigned long long rz_hcap(const KParams& p, unsigned n) {
  if (!rz_sets(p)) return 0;
  double b = sqrt(2.0 * (double)n * (double)p.ng) + 2.0;
  if (b > (double)n) b = (double)n;
  const unsigned long long keys = (unsigned long long)b + 16;
  unsigned long long cap = 64;
  while (cap < keys + keys / 2) cap <<= 1;
  return cap;
}
constexpr int RZ_NV_HOST = 26;  // reduced values per set (u64), kept per set in the arena
// words of a multi-block ROI's GLRLM / GLSZM region (a multiple of 4)
__host__ __device__ inline unsigned long long rz_words(const KParams& p, unsigned n) {
  const int sets = rz_sets(p);
  return sets ? (((unsigned long long)sets * (3ull * rz_hcap(p, n) + 2ull * RZ_NV_HOST) + 4 + 3) & ~3ull) : 0ull;
}

__host__ __device__ inline BigLayout big_layout(const KParams& p, int nch, int nsp, unsigned range, unsigned n) {
  const unsigned long long n_off = (unsigned long long)p.n_dist * p.n_dirs;
  const bool glcm = (p.need & NEED_GLCM) != 0;
  const unsigned long long tri = glcm ? (unsigned long long)p.ng * (p.ng + 1) / 2 : 0;
  const bool fsort = (p.need & NEED_ORDER) && range == 0;  // sorted values instead of a value histogram
  BigLayout L;
  unsigned long long o = 0;
  L.ctr = o;      o = (o + 4 + n_off + 3) & ~3ull;  // [0] pass 1, [1] pass 2, [2] NGTDM / GLDM, [4 + k] offset group k
  L.hist = o;     o = (o + ((p.need & NEED_HIST) ? p.hist_bins : 0) + 3) & ~3ull;
  L.vhist = o;    o = (o + range + 3) & ~3ull;
  L.tri = o;      o = (o + (nsp > 1 ? n_off * tri : 0) + 3) & ~3ull;
  L.ngt = o;      o = (o + ((p.need & NEED_NGTDM) ? 3ull * p.ng : 0) + 3) & ~3ull;  // S[ng] int64, then n[ng] u32
  L.gld = o;      o = (o + ((p.need & NEED_GLDM) ? (unsigned long long)p.ng * (p.ndim == 3 ? 27 : 9) : 0) + 3) & ~3ull;
  L.zero_end = o;
  L.part1 = o;    o += (unsigned long long)nch * BIG_P1;
  L.part2 = o;    o += (unsigned long long)nch * BIG_P2;
  L.fsort = o;    o += fsort ? 2ull * n : 0;
  // GLRLM / GLSZM (cleared by their own first kernel, which runs beside the
  // multi-block kernels): per set u64 keys (0 = empty) of rz_hcap slots; the
  // u32 counts of every set; each set's reduced values (u64); a counter
  o = (o + 3) & ~3ull;
  L.rzh = o;      o += rz_words(p, n);
  L.total = (o + 3) & ~3ull;
  return L;
}

// ---------------------------------------------------------------------------
// order-preserving encodings of pixel values
template <class T> struct Enc;
template <> struct Enc<uint16_t> {
  __host__ __device__ static unsigned enc(uint16_t v) { return v; }
  __host__ __device__ static double dec(unsigned e) { return (double)e; }
  __host__ __device__ static float decf(unsigned e) { return (float)e; }
  static constexpr int BITS = 16;
  static constexpr bool INTEGER = true;
};
template <> struct Enc<int16_t> {
  __host__ __device__ static unsigned enc(int16_t v) { return (unsigned)((int)v + 32768); }
  __host__ __device__ static double dec(unsigned e) { return (double)((int)e - 32768); }
  __host__ __device__ static float decf(unsigned e) { return (float)((int)e - 32768); }
  static constexpr int BITS = 16;
  static constexpr bool INTEGER = true;
};
template <> struct Enc<float> {
  __device__ static unsigned enc(float v) {
    unsigned b = __float_as_uint(v);
    return b ^ ((b & 0x80000000u) ? 0xFFFFFFFFu : 0x80000000u);
  }
  __device__ static float decf(unsigned e) {
    unsigned b = (e & 0x80000000u) ? (e ^ 0x80000000u) : ~e;
    return __uint_as_float(b);
  }
  __device__ static double dec(unsigned e) { return (double)decf(e); }
  static constexpr int BITS = 32;
  static constexpr bool INTEGER = false;
};

__host__ __device__ inline unsigned long long mix64(unsigned long long k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return k;
}

// Find the slot of `key` in the global label table (read-only), -1 if absent.
__device__ inline int g_find(const unsigned long long* keys, unsigned hmask, unsigned long long key) {
  unsigned h = (unsigned)mix64(key) & hmask;
  for (unsigned i = 0; i <= hmask; ++i) {
    unsigned long long k = keys[h];
    if (k == key) return (int)h;
    if (k == EMPTY_KEY) return -1;
    h = (h + 1) & hmask;
  }
  return -1;
}

// Division by an invariant 32-bit divisor (Granlund & Montgomery 1994,
// "Division by invariant integers using multiplication", unsigned case):
// exact for every 32-bit dividend.
struct FastDiv {
  unsigned m;
  int s1, s2;
  __device__ void init(unsigned d) {
    int l = 0;
    while (l < 32 && (1ull << l) < (unsigned long long)d) ++l;  // l = ceil(log2 d)
    unsigned long long num = ((1ull << l) - d) << 32;
    m = (unsigned)(num / d + 1);
    s1 = l < 1 ? l : 1;
    s2 = l - 1 > 0 ? l - 1 : 0;
  }
  __device__ unsigned div(unsigned n) const {
    unsigned t = __umulhi(m, n);
    return (t + ((n - t) >> s1)) >> s2;
  }
};

// Two-sum (Knuth): s + e = a + b exactly.
__device__ inline void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
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

__device__ inline unsigned lanemask_lt() {
  unsigned m;
  asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

}  // namespace nyx
