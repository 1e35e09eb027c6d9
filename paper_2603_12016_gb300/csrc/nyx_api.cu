// nyx_api.cu -- host side of the C ABI declared in include/nyx.h: parameter
// validation, column registry, plan workspace, and the stream-ordered launch
// sequence of one extraction:
//   k_begin -> k_scan -> k_sort_keys -> k_setup -> k_roi (per size class)
//   -> k_reset
// All data stays on the device; the host reads back only the 4-byte error
// word (and the ROI count in nyx_count_rois).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "nyx_internal.cuh"

namespace nyx {
cudaError_t launch_roi_u16(const KParams& p, int cls, int fp64, int nsm, cudaStream_t st);
cudaError_t launch_roi_i16(const KParams& p, int cls, int fp64, int nsm, cudaStream_t st);
cudaError_t launch_roi_f32(const KParams& p, int cls, int fp64, int nsm, cudaStream_t st);
cudaError_t launch_big_u16(const KParams& p, int fp64, int nsm, cudaStream_t st);
cudaError_t launch_big_i16(const KParams& p, int fp64, int nsm, cudaStream_t st);
cudaError_t launch_big_f32(const KParams& p, int fp64, int nsm, cudaStream_t st);
cudaError_t launch_glcm_final(const KParams& p, int fp64, int nsm, cudaStream_t st);
cudaError_t launch_rz_u16(const KParams& p, int big, int nsm, cudaStream_t st);
cudaError_t launch_rz_i16(const KParams& p, int big, int nsm, cudaStream_t st);
cudaError_t launch_rz_f32(const KParams& p, int big, int nsm, cudaStream_t st);
cudaError_t launch_front(const KParams& p, int nsm, cudaStream_t st);
cudaError_t launch_begin(const KParams& p, cudaStream_t st);
cudaError_t launch_scan(const KParams& p, int nsm, cudaStream_t st);
cudaError_t launch_sort_setup(const KParams& p, int nsm, cudaStream_t st);
cudaError_t launch_reset(const KParams& p, int nsm, cudaStream_t st);
cudaError_t launch_init_table(const KParams& p, unsigned cap, cudaStream_t st);
cudaError_t launch_debug_bins(const KParams& p, uint16_t* out, int nsm, cudaStream_t st);
cudaError_t launch_backward(const KParams& p, const double* gtab, float* gimg, int nsm, cudaStream_t st);
}  // namespace nyx

using namespace nyx;

// ---------------------------------------------------------------------------
// feature registry: ids 0..40 statistics, 41..50 moment families, 51..80 GLCM,
// 81..85 edge intensity statistics, 86..90 NGTDM, 91..104 GLDM, 105..120
// GLRLM, 121..138 GLSZM

namespace {

const char* STAT_NAMES[N_STATS] = {
    "MEAN", "MIN", "MAX", "RANGE", "VARIANCE", "VARIANCE_BIASED", "STDDEV", "STDDEV_BIASED", "SKEWNESS", "KURTOSIS",
    "EXCESS_KURTOSIS", "HYPERSKEWNESS", "HYPERFLATNESS", "ENERGY", "ROOT_MEAN_SQUARED", "STANDARD_ERROR",
    "MEAN_ABSOLUTE_DEVIATION", "MEDIAN_ABSOLUTE_DEVIATION", "INTEGRATED_INTENSITY", "WEIGHTED_CENTROID_X",
    "WEIGHTED_CENTROID_Y", "WEIGHTED_CENTROID_Z", "MASS_DISPLACEMENT", "COV", "COVERED_IMAGE_INTENSITY_RANGE",
    "UNIFORMITY_PIU", "MEDIAN", "P01", "P10", "P25", "P75", "P90", "P99", "INTERQUARTILE_RANGE", "QCOD", "ROBUST_MEAN",
    "ROBUST_MEAN_ABSOLUTE_DEVIATION", "MODE", "MODE_PROBABILITY", "ENTROPY", "UNIFORMITY"};
const char* MOM_FAMILY[5] = {"M", "MU", "ETA", "NU", "HU"};
const char* GLCM_NAMES[NGLCM] = {
    "ASM", "ACOR", "CLUPROM", "CLUSHADE", "CLUTEND", "CONTRAST", "CORR", "DIFAVE", "DIFENTRO", "DIFVAR",
    "DIS", "ENERGY", "ENTROPY", "HOM1", "HOM2", "IDM", "INFOMEAS1", "INFOMEAS2", "IDMN", "ID",
    "IDN", "IV", "JAVE", "JE", "JMAX", "SUMAVE", "SUMENT", "JVAR", "SUMVAR", "VARIANCE"};
const char* EDGE_NAMES[N_EDGE] = {"EDGE_INTEGRATED_INTENSITY", "EDGE_MAX_INTENSITY", "EDGE_MIN_INTENSITY",
                                  "EDGE_MEAN_INTENSITY", "EDGE_STDDEV_INTENSITY"};
constexpr int FID_MOM = N_STATS;         // 41
constexpr int FID_GLCM = N_STATS + 10;   // 51
const char* NGTDM_NAMES[N_NGTDM] = {"NGTDM_COARSENESS", "NGTDM_CONTRAST", "NGTDM_BUSYNESS", "NGTDM_COMPLEXITY",
                                    "NGTDM_STRENGTH"};
constexpr int FID_EDGE = FID_GLCM + NGLCM;  // 81
const char* GLDM_NAMES[N_GLDM] = {"GLDM_SDE",    "GLDM_LDE",  "GLDM_GLN",    "GLDM_DN",     "GLDM_DNN",
                                  "GLDM_GLV",    "GLDM_DV",   "GLDM_DE",     "GLDM_LGLE",   "GLDM_HGLE",
                                  "GLDM_SDLGLE", "GLDM_SDHGLE", "GLDM_LDLGLE", "GLDM_LDHGLE"};
constexpr int FID_NGTDM = FID_EDGE + N_EDGE;  // 86
constexpr int FID_GLDM = FID_NGTDM + N_NGTDM; // 91
const char* GLRLM_NAMES[N_GLRLM] = {"GLRLM_SRE",    "GLRLM_LRE",    "GLRLM_GLNU",   "GLRLM_GLNUN",
                                    "GLRLM_RLNU",   "GLRLM_RLNUN",  "GLRLM_RP",     "GLRLM_GLV",
                                    "GLRLM_RV",     "GLRLM_RE",     "GLRLM_LGLRE",  "GLRLM_HGLRE",
                                    "GLRLM_SRLGLE", "GLRLM_SRHGLE", "GLRLM_LRLGLE", "GLRLM_LRHGLE"};
const char* GLSZM_NAMES[N_GLSZM] = {"GLSZM_SAE",    "GLSZM_LAE",    "GLSZM_GLNU",   "GLSZM_GLNUN", "GLSZM_SZNU",
                                    "GLSZM_SZNUN",  "GLSZM_ZP",     "GLSZM_GLV",    "GLSZM_ZV",    "GLSZM_ZE",
                                    "GLSZM_LGLZE",  "GLSZM_HGLZE",  "GLSZM_SALGLE", "GLSZM_SAHGLE", "GLSZM_LALGLE",
                                    "GLSZM_LAHGLE", "GLSZM_GLM",    "GLSZM_ZSM"};
constexpr int FID_GLRLM = FID_GLDM + N_GLDM;    // 105
constexpr int FID_GLSZM = FID_GLRLM + N_GLRLM;  // 121
constexpr int N_FID = FID_GLSZM + N_GLSZM;      // 139

bool is_order_stat(int s) {
  return s == S_MEDIAN || s == S_P01 || s == S_P10 || s == S_P25 || s == S_P75 || s == S_P90 || s == S_P99 ||
         s == S_IQR || s == S_QCOD || s == S_RMEAN || s == S_RMAD || s == S_MODE || s == S_MODE_PROB || s == S_MEDAD;
}

bool fbit(const nyx_params& p, int id) { return (p.feature_mask[id >> 6] >> (id & 63)) & 1ull; }

}  // namespace

struct nyx_ctx {
  int device = 0;
  int nsm = 0;
  std::string err;
};

struct nyx_plan {
  nyx_ctx* ctx = nullptr;
  nyx_params prm{};
  std::vector<std::string> col_names;
  std::vector<int> col_map;  // Q_TOTAL entries
  KParams kp{};
  unsigned hcap = 0;
  void* ws = nullptr;         // one device allocation for the workspace
  int* d_col_map = nullptr;
  double* d_saved = nullptr;
  unsigned* d_dbg = nullptr;
  bool have_saved = false;
  // after a forward pass saved for backward, the label table (label -> ROI
  // map) stays filled for the backward pass on the same image and mask
  bool table_live = false;
  const void* live_img = nullptr;
  const int32_t* live_mask = nullptr;
  int64_t saved_rows = 0;
  int n_off = 0;
  int64_t dbg_roi = -1;
  int prof_slots = 0;                // ring of event sets, 0 = off
  int64_t prof_count = 0;            // profiled extracts so far
  std::vector<cudaEvent_t> ev;       // prof_slots * (NYX_N_PHASES + 1)
  // phase events inside the captured graph (begin / end per phase, recorded
  // on the stream the phase runs on); null when off
  bool gph = false;
  cudaEvent_t gev[2 * NYX_N_GPHASES] = {};
  // CUDA graphs of the extraction sequence, keyed by its kernel parameters
  // (a few entries, least recently used replaced)
  static constexpr int NGRAPH = 4;
  bool use_graphs = true;
  cudaStream_t cap_stream = nullptr;  // capture only; graphs launch on the caller's stream
  // branches of the extraction that run beside the caller's stream (the
  // medium class, the multi-block path, the GLCM feature kernel, the label
  // table reset), with the events that fork and join them
  cudaStream_t side[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t fork_ev[8] = {};
  cudaGraphExec_t graph_exec[NGRAPH] = {};
  KParams graph_key[NGRAPH];
  int64_t graph_used[NGRAPH] = {};
  int64_t graph_clock = 0;
  int64_t graph_captures = 0;
  // pinned staging buffers of the streamed mosaic path (two tiles in flight)
  void* stage[2] = {nullptr, nullptr};
  size_t stage_bytes = 0;
  cudaEvent_t stage_ev[2] = {nullptr, nullptr};
};

// staging capacities (pixels, padded raster cells) of the block classes:
// warp, small (128 threads), medium (256), large (512)
static const int c_class_pix[N_BLOCK_CLASSES] = {256, 1024, 4096, 8192};
static const int c_class_cells[N_BLOCK_CLASSES] = {1024, 4096, 8192, 16384};

static void drop_graph(nyx_plan* pl) {
  for (int i = 0; i < nyx_plan::NGRAPH; ++i) {
    if (pl->graph_exec[i]) cudaGraphExecDestroy(pl->graph_exec[i]);
    pl->graph_exec[i] = nullptr;
  }
}


static nyx_status fail(nyx_ctx* c, nyx_status s, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return s;
}

#define NYX_CUDA(ctx, call)                                                                 \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return fail(ctx, NYX_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));      \
  } while (0)

static nyx_status err_to_status(unsigned e) {
  if (e & E_BAD_LABEL) return NYX_ERR_BAD_LABEL;
  if (e & E_NONFINITE) return NYX_ERR_NONFINITE;
  if (e & (E_HASH_FULL | E_ROI_CAP | E_TOO_LARGE | E_SORT_CAP)) return NYX_ERR_CAPACITY;
  if (e & E_TIMEOUT) return NYX_ERR_TIMEOUT;
  if (e) return NYX_ERR_STATE;
  return NYX_OK;
}

extern "C" {

nyx_status nyx_params_default(nyx_params* p, int64_t nx, int64_t ny) {
  if (!p) return NYX_ERR_ARG;
  memset(p, 0, sizeof *p);
  p->struct_size = sizeof(nyx_params);
  p->ndim = 2;
  p->dims[0] = nx;
  p->dims[1] = ny;
  p->dims[2] = 1;
  p->batch = 1;
  p->dtype = NYX_U16;
  for (int i = 0; i < 4; ++i) p->feature_mask[i] = ~0ull;
  p->glcm_levels = 64;
  p->n_dist = 1;
  p->dists[0] = 1;
  p->glcm_per_offset_cols = 0;
  p->hist_bins = 256;
  p->precision = NYX_PREC_FP32_COMP;
  p->max_rois = 65536;
  return NYX_OK;
}

nyx_status nyx_create(nyx_ctx** out, int device) {
  if (!out) return NYX_ERR_ARG;
  *out = nullptr;
  nyx_ctx* c = new (std::nothrow) nyx_ctx();
  if (!c) return NYX_ERR_OOM;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    delete c;
    return NYX_ERR_CUDA;
  }
  c->device = device;
  if (cudaSetDevice(device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    delete c;
    return NYX_ERR_CUDA;
  }
  *out = c;
  return NYX_OK;
}

void nyx_destroy(nyx_ctx* ctx) { delete ctx; }

const char* nyx_last_error(const nyx_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int nyx_feature_id(const char* name) {
  if (!name) return -1;
  for (int i = 0; i < N_STATS; ++i)
    if (!strcmp(name, STAT_NAMES[i])) return i;
  for (int w = 0; w < 2; ++w)
    for (int f = 0; f < 5; ++f) {
      char b[32];
      snprintf(b, sizeof b, "%s_%s", w ? "BIN" : "INT", MOM_FAMILY[f]);
      if (!strcmp(name, b)) return FID_MOM + w * 5 + f;
    }
  for (int g = 0; g < NGLCM; ++g) {
    char b[48];
    snprintf(b, sizeof b, "GLCM_%s", GLCM_NAMES[g]);
    if (!strcmp(name, b)) return FID_GLCM + g;
  }
  for (int e = 0; e < N_EDGE; ++e)
    if (!strcmp(name, EDGE_NAMES[e])) return FID_EDGE + e;
  for (int q = 0; q < N_NGTDM; ++q)
    if (!strcmp(name, NGTDM_NAMES[q])) return FID_NGTDM + q;
  for (int q = 0; q < N_GLDM; ++q)
    if (!strcmp(name, GLDM_NAMES[q])) return FID_GLDM + q;
  for (int q = 0; q < N_GLRLM; ++q)
    if (!strcmp(name, GLRLM_NAMES[q])) return FID_GLRLM + q;
  for (int q = 0; q < N_GLSZM; ++q)
    if (!strcmp(name, GLSZM_NAMES[q])) return FID_GLSZM + q;
  return -1;
}

static nyx_status validate(nyx_ctx* c, const nyx_params* p) {
  if (p->struct_size != sizeof(nyx_params))
    return fail(c, NYX_ERR_ARG, "params.struct_size %u != %zu", p->struct_size, sizeof(nyx_params));
  if (p->ndim != 2 && p->ndim != 3) return fail(c, NYX_ERR_SHAPE, "ndim must be 2 or 3");
  for (int i = 0; i < 3; ++i)
    if (p->dims[i] < 1 || p->dims[i] > (1ll << 31)) return fail(c, NYX_ERR_SHAPE, "dims[%d] out of range", i);
  if (p->ndim == 2 && p->dims[2] != 1) return fail(c, NYX_ERR_SHAPE, "2D images need dims[2] = 1");
  if (p->batch < 1 || p->batch > (1 << 20)) return fail(c, NYX_ERR_SHAPE, "batch out of range");
  if (p->dtype < 0 || p->dtype > 2) return fail(c, NYX_ERR_DTYPE, "unsupported dtype %d", p->dtype);
  if (p->glcm_levels != 0 && (p->glcm_levels < 2 || p->glcm_levels > 256))
    return fail(c, NYX_ERR_ARG, "glcm_levels must be 0 or 2..256");
  if (p->n_dist < 1 || p->n_dist > MAX_DIST) return fail(c, NYX_ERR_ARG, "n_dist must be 1..8");
  for (int i = 0; i < p->n_dist; ++i)
    if (p->dists[i] < 1 || p->dists[i] > 8) return fail(c, NYX_ERR_ARG, "dists[%d] must be 1..8", i);
  if (p->hist_bins < 2 || p->hist_bins > 4096) return fail(c, NYX_ERR_ARG, "hist_bins must be 2..4096");
  if (p->precision != NYX_PREC_FP32_COMP && p->precision != NYX_PREC_FP64_PLAIN)
    return fail(c, NYX_ERR_ARG, "unknown precision");
  if (p->max_rois < 1 || p->max_rois > (1ll << 24)) return fail(c, NYX_ERR_ARG, "max_rois must be 1..2^24");
  if (p->glcm_per_offset_cols != 0 && p->glcm_per_offset_cols != 1)
    return fail(c, NYX_ERR_ARG, "glcm_per_offset_cols must be 0 or 1");
  return NYX_OK;
}

// Build the column list and the quantity -> column map.
static void build_columns(nyx_plan* pl) {
  const nyx_params& p = pl->prm;
  const bool d3 = p.ndim == 3;
  pl->col_map.assign(Q_TOTAL, -1);
  pl->col_names.clear();
  auto add = [&](int q, const std::string& nm) {
    pl->col_map[q] = (int)pl->col_names.size();
    pl->col_names.push_back(nm);
  };
  add(Q_LABEL, "LABEL");
  add(Q_IMAGE, "IMAGE");
  add(Q_AREA, "AREA");
  add(Q_BB_X, "BBOX_XMIN");
  add(Q_BB_Y, "BBOX_YMIN");
  if (d3) add(Q_BB_Z, "BBOX_ZMIN");
  add(Q_BB_W, "BBOX_WIDTH");
  add(Q_BB_H, "BBOX_HEIGHT");
  if (d3) add(Q_BB_D, "BBOX_DEPTH");
  add(Q_CEN_X, "CENTROID_X");
  add(Q_CEN_Y, "CENTROID_Y");
  if (d3) add(Q_CEN_Z, "CENTROID_Z");
  for (int s = 0; s < N_STATS; ++s) {
    if (s == S_WCZ && !d3) continue;
    if (fbit(p, s)) add(Q_STATS + s, STAT_NAMES[s]);
  }
  const int nm = d3 ? 20 : 10;
  for (int w = 0; w < 2; ++w)
    for (int f = 0; f < 5; ++f) {
      if (!fbit(p, FID_MOM + w * 5 + f)) continue;
      if (d3 && (f == F_NU || f == F_HU)) continue;
      if (f == F_HU) {
        for (int h = 0; h < 7; ++h)
          add(Q_MOM + (w * 5 + f) * 20 + h, std::string(w ? "BIN_HU" : "INT_HU") + std::to_string(h + 1));
        continue;
      }
      for (int k = 0; k < nm; ++k) {
        // lexicographic (p, q, r) with p + q + r <= 3, same order as the kernel
        int idx = 0, pp = 0, qq = 0, rr = 0;
        for (int a = 0; a <= 3; ++a)
          for (int b = 0; a + b <= 3; ++b)
            for (int c = 0; c <= (d3 ? 3 - a - b : 0); ++c) {
              if (idx == k) {
                pp = a;
                qq = b;
                rr = c;
              }
              ++idx;
            }
        if (f == F_ETA && pp + qq + rr < 2) continue;
        std::string nmc = std::string(w ? "BIN_" : "INT_") + MOM_FAMILY[f] + std::to_string(pp) + std::to_string(qq);
        if (d3) nmc += std::to_string(rr);
        add(Q_MOM + (w * 5 + f) * 20 + k, nmc);
      }
    }
  if (p.glcm_levels > 0) {
    const int ndirs = d3 ? 13 : 4;
    for (int di = 0; di < p.n_dist; ++di)
      for (int g = 0; g < NGLCM; ++g)
        if (fbit(p, FID_GLCM + g))
          add(Q_GLCM_D + di * NGLCM + g, std::string("GLCM_") + GLCM_NAMES[g] + "_D" + std::to_string(p.dists[di]));
    if (p.glcm_per_offset_cols)
      for (int di = 0; di < p.n_dist; ++di)
        for (int o = 0; o < ndirs; ++o)
          for (int g = 0; g < NGLCM; ++g)
            if (fbit(p, FID_GLCM + g))
              add(Q_GLCM_O + (di * MAX_DIRS + o) * NGLCM + g,
                  std::string("GLCM_") + GLCM_NAMES[g] + "_D" + std::to_string(p.dists[di]) +
                      (d3 ? "_O" + std::to_string(o) : "_A" + std::to_string(45 * o)));
  }
  for (int e = 0; e < N_EDGE; ++e)
    if (fbit(p, FID_EDGE + e)) add(Q_EDGE + e, EDGE_NAMES[e]);
  if (p.glcm_levels > 0)
    for (int q = 0; q < N_NGTDM; ++q)
      if (fbit(p, FID_NGTDM + q)) add(Q_NGTDM + q, NGTDM_NAMES[q]);
  if (p.glcm_levels > 0)
    for (int q = 0; q < N_GLDM; ++q)
      if (fbit(p, FID_GLDM + q)) add(Q_GLDM + q, GLDM_NAMES[q]);
  if (p.glcm_levels > 0)
    for (int q = 0; q < N_GLRLM; ++q)
      if (fbit(p, FID_GLRLM + q)) add(Q_GLRLM + q, GLRLM_NAMES[q]);
  if (p.glcm_levels > 0)
    for (int q = 0; q < N_GLSZM; ++q)
      if (fbit(p, FID_GLSZM + q)) add(Q_GLSZM + q, GLSZM_NAMES[q]);
}

// GLCM unit directions: 2D angles 0/45/90/135 degrees as (dx,dy) = (1,0),
// (1,-1), (0,-1), (-1,-1) with the row index growing downward; 3D the 13
// vectors of {-1,0,1}^3 whose first nonzero component in (dz, dy, dx) order
// is positive, dz outermost and dx fastest.
static void unit_dirs(int ndim, int dirs[13][3]) {
  if (ndim == 2) {
    const int d2[4][2] = {{1, 0}, {1, -1}, {0, -1}, {-1, -1}};
    for (int k = 0; k < 4; ++k) {
      dirs[k][0] = d2[k][0];
      dirs[k][1] = d2[k][1];
      dirs[k][2] = 0;
    }
    return;
  }
  int k = 0;
  for (int z = -1; z <= 1; ++z)
    for (int y = -1; y <= 1; ++y)
      for (int x = -1; x <= 1; ++x) {
        const int first = z != 0 ? z : (y != 0 ? y : x);
        if (first <= 0) continue;
        dirs[k][0] = x;
        dirs[k][1] = y;
        dirs[k][2] = z;
        ++k;
      }
}

static size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

nyx_status nyx_plan_create(nyx_ctx* ctx, const nyx_params* params, nyx_plan** out) {
  if (!ctx || !params || !out) return fail(ctx, NYX_ERR_ARG, "null argument");
  *out = nullptr;
  nyx_status st = validate(ctx, params);
  if (st != NYX_OK) return st;
  NYX_CUDA(ctx, cudaSetDevice(ctx->device));
  nyx_plan* pl = new (std::nothrow) nyx_plan();
  if (!pl) return fail(ctx, NYX_ERR_OOM, "host allocation failed");
  pl->ctx = ctx;
  pl->prm = *params;
  build_columns(pl);
  const nyx_params& p = pl->prm;
  unsigned hcap = 1024;
  while (hcap < 2 * (uint64_t)p.max_rois) hcap <<= 1;
  pl->hcap = hcap;
  const int64_t mr = p.max_rois;
  // workspace carve-up
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = up256(off + bytes);
    return o;
  };
  const size_t o_keys = take(8ull * hcap), o_slots = take(sizeof(SlotAcc) * hcap), o_slist = take(4ull * hcap),
               o_sdense = take(4ull * hcap), o_sorted = take(8ull * mr), o_rois = take(sizeof(RoiInfo) * mr),
               o_queue = take(4ull * N_BLOCK_CLASSES * mr), o_small = take(64), o_imin = take(4ull * p.batch),
               o_imax = take(4ull * p.batch), o_cmap = take(4ull * Q_TOTAL), o_big = take(sizeof(BigRoi) * mr),
               o_bigctr = take(64);
  // big-ROI arena: the per-ROI regions of the multi-block class (value
  // histograms, co-occurrence triangles, partial sums, float sort buffers).
  // Sorting needs 2 words per ROI pixel; the rest is per-ROI bookkeeping.
  const unsigned long long total_px = (unsigned long long)p.batch * p.dims[0] * p.dims[1] * p.dims[2];
  bool want_rl = false, want_sz = false;  // GLRLM / GLSZM selected
  if (p.glcm_levels > 0) {
    for (int q = 0; q < N_GLRLM; ++q) want_rl |= fbit(p, FID_GLRLM + q);
    for (int q = 0; q < N_GLSZM; ++q) want_sz |= fbit(p, FID_GLSZM + q);
  }
  if (want_sz && total_px >= (1ull << 32)) {
    delete pl;
    return fail(ctx, NYX_ERR_SHAPE, "GLSZM features need fewer than 2^32 pixels per call (32-bit zone parents)");
  }
  // the run / zone item tables of the multi-block ROIs: a few words per pixel
  unsigned long long arena_words = (want_rl || want_sz ? 11ull : 3ull) * total_px + (1ull << 24);
  if (arena_words > (1ull << 30)) arena_words = 1ull << 30;  // 4 GiB: large mosaics hold few multi-block ROIs
  const size_t o_arena = take(4ull * arena_words);
  // zone parents and areas of the multi-block ROIs (GLSZM): one word each per pixel
  // multi-block GLRLM / GLSZM, one word each per pixel, cleared together every
  // call: the (ROI, level) tag of every multi-block ROI pixel, then (GLSZM)
  // the zone parents and areas
  const size_t o_zbuf = (want_rl || want_sz) ? take((want_sz ? 12ull : 4ull) * total_px) : 0;
  // per (ROI, offset) GLCM accumulators (GI int64 + GF sums in 8-byte slots)
  const int n_off_all = p.glcm_levels > 0 ? p.n_dist * (p.ndim == 3 ? 13 : 4) : 0;
  const size_t o_gacc = take((size_t)mr * n_off_all * (8 * (GI_HOST + GF_HOST)));
  // inverse-difference weights per difference level (float and double)
  const int ngw = p.glcm_levels > 0 ? p.glcm_levels : 1;
  const size_t o_wtab_f = take(4ull * 5 * ngw), o_wtab_d = take(8ull * 5 * ngw);
  // c log2 c (2^-24 units) of the small counts of the entropy sums
  const size_t o_clog = take(8ull * CLOG_N);
  // round(2^63 / i^2) per level and round(2^63 / s^2) per run length / zone area (GLRLM / GLSZM)
  const size_t o_rzqi = take(8ull * 257), o_rzqs = take(8ull * (RZ_STAB + 1));
  // per-ROI statistics / moment sums (64 eight-byte slots)
  const size_t o_sacc = take((size_t)mr * 512);
  // key buffer of the key sorts (gathered keys; second run buffer of the multi-block sort)
  const size_t o_sorttmp = take(8ull * mr);
  cudaError_t e = cudaMalloc(&pl->ws, off);
  if (e != cudaSuccess) {
    delete pl;
    return fail(ctx, NYX_ERR_OOM, "workspace allocation of %zu bytes failed: %s", off, cudaGetErrorString(e));
  }
  char* w = (char*)pl->ws;
  KParams& k = pl->kp;
  memset(&k, 0, sizeof k);
  k.nx = p.dims[0];
  k.ny = p.dims[1];
  k.nz = p.dims[2];
  k.batch = p.batch;
  k.rows_total = (int64_t)p.batch * p.dims[2] * p.dims[1];
  k.ndim = p.ndim;
  k.dtype = p.dtype;
  k.ng = p.glcm_levels;
  k.n_dist = p.n_dist;
  k.n_dirs = p.ndim == 3 ? 13 : 4;
  k.per_offset = p.glcm_per_offset_cols;
  k.hist_bins = p.hist_bins;
  int dmax = 0;
  int dirs[13][3];
  unit_dirs(p.ndim, dirs);
  for (int di = 0; di < p.n_dist; ++di) {
    k.dists[di] = p.dists[di];
    if (p.dists[di] > dmax) dmax = p.dists[di];
    for (int o = 0; o < k.n_dirs; ++o)
      for (int a = 0; a < 3; ++a) k.off[di * k.n_dirs + o][a] = dirs[o][a] * p.dists[di];
  }
  k.pad = dmax;
  pl->n_off = p.n_dist * k.n_dirs;
  // computation groups
  unsigned need = 0;
  for (int s = 0; s < N_STATS; ++s) {
    if (!fbit(p, s)) continue;
    if (is_order_stat(s)) need |= NEED_ORDER;
    else if (s == S_ENTROPY || s == S_UNIFORMITY) need |= NEED_HIST;
    else need |= NEED_STATS;
  }
  for (int f = 0; f < 5; ++f) {
    if (fbit(p, FID_MOM + f)) need |= NEED_MOM_INT;
    if (fbit(p, FID_MOM + 5 + f)) need |= NEED_MOM_BIN;
  }
  if (p.glcm_levels > 0)
    for (int g = 0; g < NGLCM; ++g)
      if (fbit(p, FID_GLCM + g)) need |= NEED_GLCM;
  for (int e = 0; e < N_EDGE; ++e)
    if (fbit(p, FID_EDGE + e)) need |= NEED_EDGE;
  if (p.glcm_levels > 0)  // NGTDM grey levels are the GLCM bins
    for (int q = 0; q < N_NGTDM; ++q)
      if (fbit(p, FID_NGTDM + q)) need |= NEED_NGTDM;
  if (p.glcm_levels > 0)  // so are the GLDM grey levels
    for (int q = 0; q < N_GLDM; ++q)
      if (fbit(p, FID_GLDM + q)) need |= NEED_GLDM;
  // the edge test and the NGTDM / GLDM neighbourhoods read neighbours from
  // the padded bin raster
  if (want_rl) need |= NEED_GLRLM;
  if (want_sz) need |= NEED_GLSZM;
  // (and the run / zone kernels' own raster has one border cell, which the
  // class cell limits must cover)
  if ((need & (NEED_EDGE | NEED_NGTDM | NEED_GLDM | NEED_GLRLM | NEED_GLSZM)) && k.pad < 1) k.pad = 1;
  k.need = need;
  k.keys = (unsigned long long*)(w + o_keys);
  k.slots = (SlotAcc*)(w + o_slots);
  k.hmask = hcap - 1;
  k.slot_list = (int*)(w + o_slist);
  k.slot_dense = (int*)(w + o_sdense);
  k.sorted_keys = (unsigned long long*)(w + o_sorted);
  k.rois = (RoiInfo*)(w + o_rois);
  k.queue = (int*)(w + o_queue);
  unsigned* small = (unsigned*)(w + o_small);
  k.n_used = small + 0;
  k.n_roi = small + 1;
  k.err = small + 2;
  k.qlen = small + 4;
  k.qhead = small + 8;
  k.rz_head = small + 12;
  k.ztag = (want_rl || want_sz) ? (unsigned*)(w + o_zbuf) : nullptr;
  k.zpar = want_sz ? (unsigned*)(w + o_zbuf) + total_px : nullptr;
  k.zcnt = want_sz ? (unsigned*)(w + o_zbuf) + 2 * total_px : nullptr;
  k.img_vmin = (unsigned*)(w + o_imin);
  k.img_vmax = (unsigned*)(w + o_imax);
  k.big = (BigRoi*)(w + o_big);
  k.big_ctr = (unsigned long long*)(w + o_bigctr);
  k.big_used = k.big_ctr + 1;  // three counters (the block holds 8 words)
  k.arena = (unsigned*)(w + o_arena);
  k.arena_cap = arena_words;
  k.gacc = (unsigned char*)(w + o_gacc);
  k.sacc = (unsigned char*)(w + o_sacc);
  k.wtab_f = (const float*)(w + o_wtab_f);
  k.wtab_d = (const double*)(w + o_wtab_d);
  k.clog = (const long long*)(w + o_clog);
  k.rz_qi = (const unsigned long long*)(w + o_rzqi);
  k.rz_qs = (const unsigned long long*)(w + o_rzqs);
  std::vector<float> wf(5ull * ngw);
  std::vector<double> wd(5ull * ngw);
  for (int kk = 0; kk < ngw; ++kk) {
    const double d = kk, g = ngw;
    const double ww[5] = {1.0 / (1.0 + d), 1.0 / (1.0 + d * d), 1.0 / (1.0 + d / g), 1.0 / (1.0 + d * d / (g * g)),
                          kk >= 1 ? 1.0 / (d * d) : 0.0};
    for (int i = 0; i < 5; ++i) {
      wd[5 * kk + i] = ww[i];
      wf[5 * kk + i] = (float)ww[i];
    }
  }
  k.sort_tmp = (unsigned long long*)(w + o_sorttmp);
  pl->d_col_map = (int*)(w + o_cmap);
  k.col_map = pl->d_col_map;
  k.n_col = (int)pl->col_names.size();
  k.max_rois = mr;
  k.dbg_roi = -1;
  for (int c = 0; c < N_BLOCK_CLASSES; ++c) {  // staging capacities of the block classes
    k.lim_pix[c] = c_class_pix[c];
    k.lim_cells[c] = c_class_cells[c];
  }
  e = cudaMemcpy(pl->d_col_map, pl->col_map.data(), 4ull * Q_TOTAL, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(w + o_wtab_f, wf.data(), 4ull * 5 * ngw, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(w + o_wtab_d, wd.data(), 8ull * 5 * ngw, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    std::vector<long long> cl(CLOG_N, 0);
    for (int c = 2; c < CLOG_N; ++c) cl[c] = llround((double)c * log2((double)c) * 16777216.0);
    e = cudaMemcpy(w + o_clog, cl.data(), 8ull * CLOG_N, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) {  // round(2^63 / d) for d = i^2 and d = s^2, exact integer arithmetic
    auto q63 = [](unsigned long long d) { return d == 1 ? (1ull << 63) : ((1ull << 63) + d / 2) / d; };
    std::vector<unsigned long long> qi(257, 0), qs(RZ_STAB + 1, 0);
    for (unsigned long long i = 1; i <= 256; ++i) qi[i] = q63(i * i);
    for (unsigned long long v = 1; v <= (unsigned long long)RZ_STAB; ++v) qs[v] = q63(v * v);
    e = cudaMemcpy(w + o_rzqi, qi.data(), 8ull * 257, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(w + o_rzqs, qs.data(), 8ull * (RZ_STAB + 1), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaMemset(small, 0, 64);
  if (e == cudaSuccess) {
    e = launch_init_table(k, hcap, 0);
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&pl->cap_stream, cudaStreamNonBlocking);
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaStreamCreateWithFlags(&pl->side[i], cudaStreamNonBlocking);
  for (int i = 0; i < 8 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&pl->fork_ev[i], cudaEventDisableTiming);
  if (e != cudaSuccess) {
    cudaFree(pl->ws);
    delete pl;
    return fail(ctx, NYX_ERR_CUDA, "plan initialisation failed: %s", cudaGetErrorString(e));
  }
  *out = pl;
  return NYX_OK;
}

void nyx_plan_destroy(nyx_plan* pl) {
  if (!pl) return;
  cudaSetDevice(pl->ctx->device);
  for (cudaEvent_t e : pl->ev) cudaEventDestroy(e);
  for (cudaEvent_t e : pl->gev)
    if (e) cudaEventDestroy(e);
  drop_graph(pl);
  if (pl->cap_stream) cudaStreamDestroy(pl->cap_stream);
  for (int i = 0; i < 3; ++i)
    if (pl->side[i]) cudaStreamDestroy(pl->side[i]);
  for (int i = 0; i < 8; ++i)
    if (pl->fork_ev[i]) cudaEventDestroy(pl->fork_ev[i]);
  for (int i = 0; i < 2; ++i) {
    if (pl->stage[i]) cudaFreeHost(pl->stage[i]);
    if (pl->stage_ev[i]) cudaEventDestroy(pl->stage_ev[i]);
  }
  cudaFree(pl->ws);
  if (pl->d_saved) cudaFree(pl->d_saved);
  if (pl->d_dbg) cudaFree(pl->d_dbg);
  delete pl;
}

nyx_status nyx_num_columns(const nyx_plan* pl, int* n_col) {
  if (!pl || !n_col) return NYX_ERR_ARG;
  *n_col = (int)pl->col_names.size();
  return NYX_OK;
}

nyx_status nyx_column_name(const nyx_plan* pl, int col, char* buf, size_t cap) {
  if (!pl || !buf || cap == 0 || col < 0 || col >= (int)pl->col_names.size()) return NYX_ERR_ARG;
  snprintf(buf, cap, "%s", pl->col_names[col].c_str());
  return NYX_OK;
}

static nyx_status check_ptrs(nyx_plan* pl, const void* img, const int32_t* mask) {
  if (!img || !mask) return fail(pl->ctx, NYX_ERR_ARG, "null image or mask pointer");
  if (((uintptr_t)img & 15) || ((uintptr_t)mask & 15))
    return fail(pl->ctx, NYX_ERR_ARG, "image and mask must be 16-byte aligned");
  return NYX_OK;
}

// Front half of every call: counters and label scan; then key sort + setup.
static nyx_status run_front(nyx_plan* pl, KParams& k, cudaStream_t st) {
  NYX_CUDA(pl->ctx, launch_front(k, pl->ctx->nsm, st));
  return NYX_OK;
}

static nyx_status run_sort_setup(nyx_plan* pl, KParams& k, cudaStream_t st) {
  NYX_CUDA(pl->ctx, launch_sort_setup(k, pl->ctx->nsm, st));
  return NYX_OK;
}

static nyx_status run_reset(nyx_plan* pl, KParams& k, cudaStream_t st) {
  NYX_CUDA(pl->ctx, launch_reset(k, pl->ctx->nsm, st));
  return NYX_OK;
}

static nyx_status read_err(nyx_plan* pl, cudaStream_t st) {
  unsigned h = 0;
  NYX_CUDA(pl->ctx, cudaMemcpyAsync(&h, pl->kp.err, 4, cudaMemcpyDeviceToHost, st));
  NYX_CUDA(pl->ctx, cudaStreamSynchronize(st));
  if (h) {
    NYX_CUDA(pl->ctx, cudaMemsetAsync(pl->kp.err, 0, 4, st));
    NYX_CUDA(pl->ctx, cudaStreamSynchronize(st));
    return fail(pl->ctx, err_to_status(h), "device reported error bits 0x%x", h);
  }
  return NYX_OK;
}

// Empty the label table left filled by a forward pass saved for backward
// (stream-ordered before the caller's next scan).
static nyx_status flush_live(nyx_plan* pl, cudaStream_t st) {
  if (!pl->table_live) return NYX_OK;
  pl->table_live = false;
  KParams k;
  memcpy(&k, &pl->kp, sizeof k);
  return run_reset(pl, k, st);
}

nyx_status nyx_count_rois(nyx_plan* pl, const void* d_img, const int32_t* d_mask, int64_t* n_roi, void* stream) {
  if (!pl || !n_roi) return NYX_ERR_ARG;
  nyx_status s = check_ptrs(pl, d_img, d_mask);
  if (s != NYX_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  NYX_CUDA(pl->ctx, cudaSetDevice(pl->ctx->device));
  if ((s = flush_live(pl, st)) != NYX_OK) return s;
  KParams k = pl->kp;
  k.img = d_img;
  k.mask = d_mask;
  k.vec = (k.nx % 4) == 0;
  if ((s = run_front(pl, k, st)) != NYX_OK) return s;
  unsigned h = 0;
  NYX_CUDA(pl->ctx, cudaMemcpyAsync(&h, k.n_used, 4, cudaMemcpyDeviceToHost, st));
  if ((s = run_reset(pl, k, st)) != NYX_OK) return s;
  s = read_err(pl, st);
  *n_roi = h;
  return s;
}

// The launch sequence of one extraction (label scan, key sort + setup, the
// four size classes, GLCM features, table reset).  `ev` (profiling) records
// the phase boundaries; it is null when the sequence is captured.
static nyx_status enqueue_back(nyx_plan* pl, const KParams& k, cudaEvent_t* ev, cudaStream_t st,
                               cudaEvent_t* gev = nullptr);

// Graph phase event: begin (end = 0) or end (end = 1) of phase `ph`, as an
// external event node of the graph being captured on stream `s`.
static inline cudaError_t gmark(cudaEvent_t* gev, int ph, int end, cudaStream_t s) {
  return gev ? cudaEventRecordWithFlags(gev[2 * ph + end], s, cudaEventRecordExternal) : cudaSuccess;
}

static nyx_status enqueue_extract(nyx_plan* pl, const KParams& k, cudaEvent_t* ev, cudaStream_t st,
                                  cudaEvent_t* gev = nullptr) {
  nyx_ctx* c = pl->ctx;
  nyx_status s;
  if (k.dbg_glcm) NYX_CUDA(c, cudaMemsetAsync(pl->d_dbg, 0, 4ull * pl->n_off * k.ng * k.ng, st));
  NYX_CUDA(c, gmark(gev, NYX_GPH_ALL, 0, st));
  if (ev) NYX_CUDA(c, cudaEventRecord(ev[0], st));
  NYX_CUDA(c, gmark(gev, NYX_GPH_SCAN, 0, st));
  if ((s = run_front(pl, const_cast<KParams&>(k), st)) != NYX_OK) return s;
  NYX_CUDA(c, gmark(gev, NYX_GPH_SCAN, 1, st));
  if (ev) NYX_CUDA(c, cudaEventRecord(ev[1], st));
  if ((s = enqueue_back(pl, k, ev, st, gev)) != NYX_OK) return s;
  NYX_CUDA(c, gmark(gev, NYX_GPH_ALL, 1, st));
  return NYX_OK;
}

static cudaError_t launch_class(const KParams& k, int cls, int fp64, int nsm, cudaStream_t st) {
  switch (k.dtype) {
    case NYX_U16: return launch_roi_u16(k, cls, fp64, nsm, st);
    case NYX_I16: return launch_roi_i16(k, cls, fp64, nsm, st);
    default: return launch_roi_f32(k, cls, fp64, nsm, st);
  }
}

// GLRLM / GLSZM: the block path (big = 0) or the multi-block path (big = 1)
static cudaError_t launch_rz(const KParams& k, int big, int nsm, cudaStream_t st) {
  switch (k.dtype) {
    case NYX_U16: return launch_rz_u16(k, big, nsm, st);
    case NYX_I16: return launch_rz_i16(k, big, nsm, st);
    default: return launch_rz_f32(k, big, nsm, st);
  }
}

static cudaError_t launch_big(const KParams& k, int fp64, int nsm, cudaStream_t st) {
  switch (k.dtype) {
    case NYX_U16: return launch_big_u16(k, fp64, nsm, st);
    case NYX_I16: return launch_big_i16(k, fp64, nsm, st);
    default: return launch_big_f32(k, fp64, nsm, st);
  }
}

// Everything after the label scan: key sort + setup, the four size classes,
// GLCM features, table reset.  The size classes work on disjoint ROIs, and
// the GLCM feature and statistics kernels on disjoint sums, so outside
// profiling they run as parallel branches: the medium class and the
// multi-block path on the plan's side streams, the warp and small classes on
// `st`, joined before the kernels that read every ROI's sums; then the GLCM
// feature kernel beside the statistics kernel.  Blocks of one class fill the
// SMs that another class's tail leaves idle.  A class whose pixel limit is 0
// receives no ROI and is not launched.
static nyx_status enqueue_back(nyx_plan* pl, const KParams& k, cudaEvent_t* ev, cudaStream_t st,
                               cudaEvent_t* gev) {
  nyx_ctx* c = pl->ctx;
  nyx_status s;
  NYX_CUDA(c, gmark(gev, NYX_GPH_SORT, 0, st));
  if ((s = run_sort_setup(pl, const_cast<KParams&>(k), st)) != NYX_OK) return s;
  NYX_CUDA(c, gmark(gev, NYX_GPH_SORT, 1, st));
  if (ev) NYX_CUDA(c, cudaEventRecord(ev[2], st));
  const int fp64 = pl->prm.precision == NYX_PREC_FP64_PLAIN;
  const bool fork = ev == nullptr && pl->side[0] != nullptr;
  const bool rz = (k.need & (NEED_GLRLM | NEED_GLSZM)) != 0;
  cudaStream_t s_med = st, s_big = st, s_rz = st;
  NYX_CUDA(c, gmark(gev, NYX_GPH_ROI, 0, st));
  if (fork) {
    NYX_CUDA(c, cudaEventRecord(pl->fork_ev[0], st));
    for (int i = 0; i < (rz ? 3 : 2); ++i) NYX_CUDA(c, cudaStreamWaitEvent(pl->side[i], pl->fork_ev[0], 0));
    s_med = pl->side[0];
    s_big = pl->side[1];
    if (rz) s_rz = pl->side[2];
  }
  for (int cls = 0; cls < N_BLOCK_CLASSES; ++cls) {
    cudaStream_t sc = cls >= 2 ? s_med : st;  // medium and large classes on one side branch
    NYX_CUDA(c, gmark(gev, NYX_GPH_WARP + cls, 0, sc));
    const cudaError_t e = k.lim_pix[cls] > 0 ? launch_class(k, cls, fp64, c->nsm, sc) : cudaSuccess;
    if (e != cudaSuccess) return fail(c, NYX_ERR_CUDA, "ROI kernel launch failed: %s", cudaGetErrorString(e));
    NYX_CUDA(c, gmark(gev, NYX_GPH_WARP + cls, 1, sc));
    if (ev) NYX_CUDA(c, cudaEventRecord(ev[3 + cls], st));
  }
  if (rz) {  // block-class GLRLM / GLSZM: reads the image and ROI table only, writes its own columns
    NYX_CUDA(c, gmark(gev, NYX_GPH_RZ, 0, s_rz));
    cudaError_t e = launch_rz(k, 0, c->nsm, s_rz);
    if (e == cudaSuccess) e = launch_rz(k, 1, c->nsm, s_rz);  // then the multi-block ROIs, on the same branch
    if (e != cudaSuccess) return fail(c, NYX_ERR_CUDA, "GLRLM / GLSZM kernel launch failed: %s", cudaGetErrorString(e));
    NYX_CUDA(c, gmark(gev, NYX_GPH_RZ, 1, s_rz));
  } else {
    NYX_CUDA(c, gmark(gev, NYX_GPH_RZ, 0, st));
    NYX_CUDA(c, gmark(gev, NYX_GPH_RZ, 1, st));
  }
  {
    NYX_CUDA(c, gmark(gev, NYX_GPH_BIG, 0, s_big));
    const cudaError_t e = launch_big(k, fp64, c->nsm, s_big);
    if (e != cudaSuccess) return fail(c, NYX_ERR_CUDA, "multi-block ROI kernel launch failed: %s", cudaGetErrorString(e));
    NYX_CUDA(c, gmark(gev, NYX_GPH_BIG, 1, s_big));
    if (ev) NYX_CUDA(c, cudaEventRecord(ev[7], st));
  }
  if (fork) {  // join, then fork the GLCM feature kernel
    NYX_CUDA(c, cudaEventRecord(pl->fork_ev[1], s_med));
    NYX_CUDA(c, cudaEventRecord(pl->fork_ev[2], s_big));
    NYX_CUDA(c, cudaStreamWaitEvent(st, pl->fork_ev[1], 0));
    NYX_CUDA(c, cudaStreamWaitEvent(st, pl->fork_ev[2], 0));
    if (rz) {
      NYX_CUDA(c, cudaEventRecord(pl->fork_ev[6], s_rz));
      NYX_CUDA(c, cudaStreamWaitEvent(st, pl->fork_ev[6], 0));
    }
  }
  NYX_CUDA(c, gmark(gev, NYX_GPH_ROI, 1, st));
  // the GLCM feature kernel, the statistics kernel and the label-table reset
  // touch disjoint data: three branches
  const bool reset = !(k.need & NEED_SAVE);  // a pass saved for backward keeps the label table
  cudaStream_t s_gl = st, s_rs = st;
  if (fork) {
    NYX_CUDA(c, cudaEventRecord(pl->fork_ev[3], st));
    if (k.need & NEED_GLCM) {
      NYX_CUDA(c, cudaStreamWaitEvent(pl->side[0], pl->fork_ev[3], 0));
      s_gl = pl->side[0];
    }
    if (reset) {
      NYX_CUDA(c, cudaStreamWaitEvent(pl->side[1], pl->fork_ev[3], 0));
      s_rs = pl->side[1];
    }
  }
  NYX_CUDA(c, gmark(gev, NYX_GPH_GLCMF, 0, s_gl));
  if (k.need & NEED_GLCM) {
    cudaError_t e = launch_glcm_final(k, fp64, c->nsm, s_gl);
    if (e != cudaSuccess) return fail(c, NYX_ERR_CUDA, "GLCM feature kernel launch failed: %s", cudaGetErrorString(e));
  }
  NYX_CUDA(c, gmark(gev, NYX_GPH_GLCMF, 1, s_gl));
  if (reset && s_rs != st) {
    NYX_CUDA(c, gmark(gev, NYX_GPH_RESET, 0, s_rs));
    if ((s = run_reset(pl, const_cast<KParams&>(k), s_rs)) != NYX_OK) return s;
    NYX_CUDA(c, gmark(gev, NYX_GPH_RESET, 1, s_rs));
  }
  {  // statistics, moments and Hu invariants from the per-ROI sums
    NYX_CUDA(c, gmark(gev, NYX_GPH_STATSF, 0, st));
    const cudaError_t e = launch_class(k, N_BLOCK_CLASSES, fp64, c->nsm, st);
    if (e != cudaSuccess) return fail(c, NYX_ERR_CUDA, "statistics kernel launch failed: %s", cudaGetErrorString(e));
    NYX_CUDA(c, gmark(gev, NYX_GPH_STATSF, 1, st));
  }
  if (s_gl != st) {
    NYX_CUDA(c, cudaEventRecord(pl->fork_ev[4], s_gl));
    NYX_CUDA(c, cudaStreamWaitEvent(st, pl->fork_ev[4], 0));
  }
  if (s_rs != st) {
    NYX_CUDA(c, cudaEventRecord(pl->fork_ev[5], s_rs));
    NYX_CUDA(c, cudaStreamWaitEvent(st, pl->fork_ev[5], 0));
  }
  if (ev) NYX_CUDA(c, cudaEventRecord(ev[8], st));
  if (reset && s_rs == st) {
    NYX_CUDA(c, gmark(gev, NYX_GPH_RESET, 0, st));
    if ((s = run_reset(pl, const_cast<KParams&>(k), st)) != NYX_OK) return s;
    NYX_CUDA(c, gmark(gev, NYX_GPH_RESET, 1, st));
  } else if (!reset) {  // no reset in this sequence: an empty phase
    NYX_CUDA(c, gmark(gev, NYX_GPH_RESET, 0, st));
    NYX_CUDA(c, gmark(gev, NYX_GPH_RESET, 1, st));
  }
  if (ev) NYX_CUDA(c, cudaEventRecord(ev[NYX_N_PHASES], st));
  return NYX_OK;
}

// Replay the cached graph of this exact launch sequence (same kernel
// parameters, byte for byte), or capture it on the plan's own stream first.
// The instantiated graph is then launched on the caller's stream, which may
// be the legacy default stream.
static nyx_status launch_graph(nyx_plan* pl, const KParams& k, cudaStream_t st) {
  nyx_ctx* c = pl->ctx;
  int slot = -1, victim = 0;
  for (int i = 0; i < nyx_plan::NGRAPH; ++i) {
    if (pl->graph_exec[i] && memcmp(&pl->graph_key[i], &k, sizeof(KParams)) == 0) slot = i;
    if (!pl->graph_exec[i] || (pl->graph_exec[victim] && pl->graph_used[i] < pl->graph_used[victim])) victim = i;
  }
  if (slot < 0) {
    slot = victim;
    if (pl->graph_exec[slot]) cudaGraphExecDestroy(pl->graph_exec[slot]);
    pl->graph_exec[slot] = nullptr;
    NYX_CUDA(c, cudaStreamBeginCapture(pl->cap_stream, cudaStreamCaptureModeRelaxed));
    const nyx_status s = enqueue_extract(pl, k, nullptr, pl->cap_stream, pl->gph ? pl->gev : nullptr);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(pl->cap_stream, &g);
    if (s != NYX_OK) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    if (e != cudaSuccess) return fail(c, NYX_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
    const cudaError_t ei = cudaGraphInstantiate(&pl->graph_exec[slot], g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      pl->graph_exec[slot] = nullptr;
      return fail(c, NYX_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(ei));
    }
    memcpy(&pl->graph_key[slot], &k, sizeof(KParams));
    ++pl->graph_captures;
  }
  pl->graph_used[slot] = ++pl->graph_clock;
  NYX_CUDA(c, cudaGraphLaunch(pl->graph_exec[slot], st));
  return NYX_OK;
}

nyx_status nyx_extract(nyx_plan* pl, const void* d_img, const int32_t* d_mask, double* d_table, int64_t cap_roi,
                       int64_t* d_n_roi, uint32_t flags, void* stream) {
  if (!pl) return NYX_ERR_ARG;
  nyx_status s = check_ptrs(pl, d_img, d_mask);
  if (s != NYX_OK) return s;
  if (!d_table && cap_roi > 0) return fail(pl->ctx, NYX_ERR_ARG, "null table");
  if (cap_roi < 0) return fail(pl->ctx, NYX_ERR_ARG, "cap_roi < 0");
  if ((uintptr_t)d_table & 7) return fail(pl->ctx, NYX_ERR_ARG, "table must be 8-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  nyx_ctx* c = pl->ctx;
  NYX_CUDA(c, cudaSetDevice(c->device));
  // kernel parameters: a byte copy of the plan's (zero-padded) template, so
  // that equal launches compare equal byte for byte
  KParams k;
  memcpy(&k, &pl->kp, sizeof k);
  k.img = d_img;
  k.mask = d_mask;
  k.vec = (k.nx % 4) == 0;
  k.table = d_table;
  k.cap_roi = cap_roi < pl->prm.max_rois ? cap_roi : pl->prm.max_rois;
  k.n_roi_out = d_n_roi;
  if (flags & NYX_SAVE_FOR_BACKWARD) {
    if (!pl->d_saved) {
      // saved per-ROI state, then the backward pass's per-ROI coefficients (40 floats)
      cudaError_t e = cudaMalloc(&pl->d_saved, (8ull * SV_WORDS + 4ull * 40) * pl->prm.max_rois);
      if (e != cudaSuccess) {
        pl->d_saved = nullptr;
        return fail(c, NYX_ERR_OOM, "saved-state allocation failed");
      }
    }
    k.saved = pl->d_saved;
    k.need |= NEED_SAVE;
    pl->have_saved = true;
  } else {
    pl->have_saved = false;
  }
  if (pl->dbg_roi >= 0 && pl->d_dbg && (k.need & NEED_GLCM)) {
    k.dbg_roi = pl->dbg_roi;
    k.dbg_glcm = pl->d_dbg;
  }
  if ((s = flush_live(pl, st)) != NYX_OK) return s;
  if (pl->prof_slots > 0) {  // profiled: direct launches with phase events
    cudaEvent_t* ev = &pl->ev[(size_t)(pl->prof_count % pl->prof_slots) * (NYX_N_PHASES + 1)];
    if ((s = enqueue_extract(pl, k, ev, st)) != NYX_OK) return s;
    ++pl->prof_count;
  } else if (pl->use_graphs) {
    if ((s = launch_graph(pl, k, st)) != NYX_OK) return s;
  } else {
    if ((s = enqueue_extract(pl, k, nullptr, st)) != NYX_OK) return s;
  }
  if (k.need & NEED_SAVE) {
    pl->table_live = true;
    pl->live_img = d_img;
    pl->live_mask = d_mask;
  }
  if (flags & NYX_SYNC) return read_err(pl, st);
  return NYX_OK;
}

nyx_status nyx_extract_tiles(nyx_plan* pl, int64_t tile_w, int64_t tile_h, nyx_tile_fn fn, void* user, void* d_img,
                             int32_t* d_mask, double* d_table, int64_t cap_roi, int64_t* d_n_roi, uint32_t flags,
                             void* stream) {
  if (!pl || !fn) return NYX_ERR_ARG;
  nyx_ctx* c = pl->ctx;
  const nyx_params& prm = pl->prm;
  if (prm.ndim != 2 || prm.batch != 1) return fail(c, NYX_ERR_SHAPE, "tiled extraction needs a 2D plan with batch 1");
  if (tile_w < 1 || tile_h < 1) return fail(c, NYX_ERR_ARG, "tile extent must be positive");
  nyx_status s = check_ptrs(pl, d_img, d_mask);
  if (s != NYX_OK) return s;
  if (!d_table && cap_roi > 0) return fail(c, NYX_ERR_ARG, "null table");
  if (cap_roi < 0 || ((uintptr_t)d_table & 7)) return fail(c, NYX_ERR_ARG, "bad table or cap_roi");
  if (flags & NYX_SAVE_FOR_BACKWARD) return fail(c, NYX_ERR_ARG, "tiled extraction does not keep backward state");
  cudaStream_t st = (cudaStream_t)stream;
  NYX_CUDA(c, cudaSetDevice(c->device));
  const int64_t W = prm.dims[0], H = prm.dims[1];
  const size_t isz = prm.dtype == NYX_F32 ? 4 : 2;
  const int64_t tw = tile_w < W ? tile_w : W, th = tile_h < H ? tile_h : H;
  const size_t need = (((size_t)tw * th * isz + 15) & ~(size_t)15) + (size_t)tw * th * 4;
  if (pl->stage_bytes < need) {
    for (int i = 0; i < 2; ++i) {
      if (pl->stage[i]) cudaFreeHost(pl->stage[i]);
      pl->stage[i] = nullptr;
    }
    pl->stage_bytes = 0;
    for (int i = 0; i < 2; ++i)
      if (cudaHostAlloc(&pl->stage[i], need, cudaHostAllocDefault) != cudaSuccess) {
        pl->stage[i] = nullptr;
        return fail(c, NYX_ERR_OOM, "pinned staging allocation of %zu bytes failed", need);
      }
    pl->stage_bytes = need;
  }
  for (int i = 0; i < 2; ++i)
    if (!pl->stage_ev[i]) NYX_CUDA(c, cudaEventCreateWithFlags(&pl->stage_ev[i], cudaEventDisableTiming));
  KParams k;
  memcpy(&k, &pl->kp, sizeof k);
  k.img = d_img;
  k.mask = d_mask;
  k.vec = (k.nx % 4) == 0;
  k.table = d_table;
  k.cap_roi = cap_roi < prm.max_rois ? cap_roi : prm.max_rois;
  k.n_roi_out = d_n_roi;
  pl->have_saved = false;
  if ((s = flush_live(pl, st)) != NYX_OK) return s;
  NYX_CUDA(c, launch_begin(k, st));
  // make sure both staging buffers are free before the first fill
  for (int i = 0; i < 2; ++i) NYX_CUDA(c, cudaEventRecord(pl->stage_ev[i], st));
  int slot = 0;
  bool failed = false;
  for (int64_t y0 = 0; y0 < H && !failed; y0 += tile_h) {
    const int64_t h = H - y0 < tile_h ? H - y0 : tile_h;
    for (int64_t x0 = 0; x0 < W; x0 += tile_w) {
      const int64_t w = W - x0 < tile_w ? W - x0 : tile_w;
      NYX_CUDA(c, cudaEventSynchronize(pl->stage_ev[slot]));  // its previous copy is done
      unsigned char* himg = (unsigned char*)pl->stage[slot];
      int32_t* hmask = (int32_t*)(himg + (((size_t)w * h * isz + 15) & ~(size_t)15));
      if (fn(user, x0, y0, w, h, himg, hmask) != 0) {
        failed = true;
        break;
      }
      NYX_CUDA(c, cudaMemcpy2DAsync((unsigned char*)d_img + ((size_t)y0 * W + x0) * isz, (size_t)W * isz, himg,
                                    (size_t)w * isz, (size_t)w * isz, (size_t)h, cudaMemcpyHostToDevice, st));
      NYX_CUDA(c, cudaMemcpy2DAsync(d_mask + (size_t)y0 * W + x0, (size_t)W * 4, hmask, (size_t)w * 4, (size_t)w * 4,
                                    (size_t)h, cudaMemcpyHostToDevice, st));
      NYX_CUDA(c, cudaEventRecord(pl->stage_ev[slot], st));
      slot ^= 1;
    }
    if (failed) break;
    // the band's tiles are in: label-scan its rows while the next band streams
    k.scan_row0 = y0;
    k.scan_row1 = y0 + h;
    NYX_CUDA(c, launch_scan(k, c->nsm, st));
  }
  k.scan_row0 = 0;
  k.scan_row1 = 0;
  if (failed) {  // return the label table to its empty state
    run_reset(pl, k, st);
    cudaStreamSynchronize(st);
    return fail(c, NYX_ERR_ARG, "tile source reported an error");
  }
  if ((s = enqueue_back(pl, k, nullptr, st)) != NYX_OK) return s;
  if (flags & NYX_SYNC) return read_err(pl, st);
  return NYX_OK;
}

nyx_status nyx_use_graphs(nyx_plan* pl, int enable) {
  if (!pl) return NYX_ERR_ARG;
  pl->use_graphs = enable != 0;
  if (!pl->use_graphs) drop_graph(pl);
  return NYX_OK;
}

nyx_status nyx_graph_captures(const nyx_plan* pl, int64_t* n) {
  if (!pl || !n) return NYX_ERR_ARG;
  *n = pl->graph_captures;
  return NYX_OK;
}

// Median device time of `reps` extractions, each after an L2 flush (a
// write of `flush_bytes` over `flush`), with the plan's current settings.
static nyx_status time_config(nyx_plan* pl, const void* d_img, const int32_t* d_mask, double* d_table,
                              int64_t cap_roi, int reps, cudaStream_t st, void* flush, size_t flush_bytes,
                              cudaEvent_t e0, cudaEvent_t e1, float* ms_out) {
  nyx_ctx* c = pl->ctx;
  nyx_status s = nyx_extract(pl, d_img, d_mask, d_table, cap_roi, nullptr, NYX_SYNC, st);  // warm-up + check
  if (s != NYX_OK) return s;
  float t[100];
  for (int r = 0; r < reps; ++r) {
    if (flush) NYX_CUDA(c, cudaMemsetAsync(flush, r & 0xFF, flush_bytes, st));
    NYX_CUDA(c, cudaEventRecord(e0, st));
    if ((s = nyx_extract(pl, d_img, d_mask, d_table, cap_roi, nullptr, 0, st)) != NYX_OK) return s;
    NYX_CUDA(c, cudaEventRecord(e1, st));
    NYX_CUDA(c, cudaEventSynchronize(e1));
    NYX_CUDA(c, cudaEventElapsedTime(&t[r], e0, e1));
  }
  for (int i = 1; i < reps; ++i)  // insertion sort, then the median
    for (int j = i; j > 0 && t[j] < t[j - 1]; --j) {
      const float x = t[j];
      t[j] = t[j - 1];
      t[j - 1] = x;
    }
  *ms_out = t[reps / 2];
  return NYX_OK;
}

// Median device time of the label scan alone (counter reset + scan), each
// call after the same L2 flush; its label table is reset outside the timed
// region.
static nyx_status time_scan(nyx_plan* pl, const void* d_img, const int32_t* d_mask, int reps, cudaStream_t st,
                            void* flush, size_t flush_bytes, cudaEvent_t e0, cudaEvent_t e1, float* ms_out) {
  nyx_ctx* c = pl->ctx;
  nyx_status s;
  if ((s = flush_live(pl, st)) != NYX_OK) return s;
  KParams k = pl->kp;
  k.img = d_img;
  k.mask = d_mask;
  k.vec = (k.nx % 4) == 0;
  if ((s = run_front(pl, k, st)) != NYX_OK) return s;  // warm-up
  if ((s = run_reset(pl, k, st)) != NYX_OK) return s;
  float t[100];
  for (int r = 0; r < reps; ++r) {
    if (flush) NYX_CUDA(c, cudaMemsetAsync(flush, r & 0xFF, flush_bytes, st));
    NYX_CUDA(c, cudaEventRecord(e0, st));
    if ((s = run_front(pl, k, st)) != NYX_OK) return s;
    NYX_CUDA(c, cudaEventRecord(e1, st));
    NYX_CUDA(c, cudaEventSynchronize(e1));
    NYX_CUDA(c, cudaEventElapsedTime(&t[r], e0, e1));
    if ((s = run_reset(pl, k, st)) != NYX_OK) return s;
  }
  if ((s = read_err(pl, st)) != NYX_OK) return s;
  for (int i = 1; i < reps; ++i)
    for (int j = i; j > 0 && t[j] < t[j - 1]; --j) {
      const float x = t[j];
      t[j] = t[j - 1];
      t[j - 1] = x;
    }
  *ms_out = t[reps / 2];
  return NYX_OK;
}

nyx_status nyx_autotune(nyx_plan* pl, const void* d_img, const int32_t* d_mask, double* d_table, int64_t cap_roi,
                        int reps, void* stream, int32_t* h_lim_pix) {
  if (!pl || reps < 1 || reps > 100) return NYX_ERR_ARG;
  nyx_status s = check_ptrs(pl, d_img, d_mask);
  if (s != NYX_OK) return s;
  nyx_ctx* c = pl->ctx;
  cudaStream_t st = (cudaStream_t)stream;
  NYX_CUDA(c, cudaSetDevice(c->device));
  // candidate pixel thresholds of the warp, small, medium and large classes
  // (0 = class unused; the cell limits stay at each class's staging
  // capacity), then, timing the label scan alone, its rows per warp (tile
  // heights 64/128/256) under either staging of its rows
  static const int cw[] = {0, 64, 128, 256}, cs[] = {0, 512, 1024}, cm[] = {0, 2048, 4096}, cl[] = {0, 8192},
                   cr[] = {8, 16, 32};
  const int saved_prof = pl->prof_slots;
  pl->prof_slots = 0;
  int best[N_BLOCK_CLASSES];
  for (int i = 0; i < N_BLOCK_CLASSES; ++i) best[i] = pl->kp.lim_pix[i];
  int best_rpt = pl->kp.scan_rpt, best_stage = pl->kp.scan_stage;
  float best_ms = 3.0e38f;
  // an L2-sized write between timed calls, so that every candidate starts
  // from cold caches as a new image would (an offline call: it may allocate)
  const size_t flush_bytes = 256ull << 20;
  void* flush = nullptr;
  if (cudaMalloc(&flush, flush_bytes) != cudaSuccess) flush = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  NYX_CUDA(c, cudaEventCreate(&e0));
  NYX_CUDA(c, cudaEventCreate(&e1));
  for (int a : cw)
    for (int b : cs)
      for (int m : cm)
        for (int l : cl) {
          // nonzero limits must increase with the class, and some block class
          // must take ROIs above the warp class
          const int lim[N_BLOCK_CLASSES] = {a, b, m, l};
          int top = 0;
          bool ok = true;
          for (int i = 0; i < N_BLOCK_CLASSES; ++i)
            if (lim[i]) {
              ok = ok && lim[i] > top;
              top = lim[i];
            }
          if (!ok || (b == 0 && m == 0 && l == 0)) continue;
          for (int i = 0; i < N_BLOCK_CLASSES; ++i) pl->kp.lim_pix[i] = lim[i];
          float ms = 0;
          s = time_config(pl, d_img, d_mask, d_table, cap_roi, reps, st, flush, flush_bytes, e0, e1, &ms);
          if (s == NYX_ERR_CAPACITY) {  // these limits overflow the multi-block arena: not a candidate
            s = NYX_OK;
            continue;
          }
          if (s != NYX_OK) break;
          if (ms < best_ms) {
            best_ms = ms;
            for (int i = 0; i < N_BLOCK_CLASSES; ++i) best[i] = lim[i];
          }
        }
  for (int i = 0; i < N_BLOCK_CLASSES; ++i) pl->kp.lim_pix[i] = best[i];
  if (s == NYX_OK) {
    best_ms = 3.0e38f;
    for (int g = 0; g < 2 && s == NYX_OK; ++g)  // bulk tensor copies (where legal), then register loads
      for (int r : cr) {
        pl->kp.scan_rpt = r;
        pl->kp.scan_stage = g;
        float ms = 0;
        s = time_scan(pl, d_img, d_mask, reps, st, flush, flush_bytes, e0, e1, &ms);
        if (s != NYX_OK) break;
        if (ms < best_ms) {
          best_ms = ms;
          best_rpt = r;
          best_stage = g;
        }
      }
  }
  pl->kp.scan_rpt = best_rpt;
  pl->kp.scan_stage = best_stage;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (flush) cudaFree(flush);
  drop_graph(pl);
  pl->prof_slots = saved_prof;
  if (s != NYX_OK) return s;
  if (h_lim_pix)
    for (int i = 0; i < N_BLOCK_CLASSES; ++i) h_lim_pix[i] = best[i];
  return NYX_OK;
}

nyx_status nyx_set_tuning(nyx_plan* pl, const int32_t* t) {
  if (!pl || !t) return NYX_ERR_ARG;
  const int r = t[N_BLOCK_CLASSES];
  if (r != 0 && r != 4 && r != 8 && r != 16 && r != 32)
    return fail(pl->ctx, NYX_ERR_ARG, "scan rows per warp must be 0, 4, 8, 16 or 32");
  nyx_status s = nyx_set_class_limits(pl, t);
  if (s != NYX_OK) return s;
  pl->kp.scan_rpt = r;
  drop_graph(pl);
  return NYX_OK;
}

nyx_status nyx_get_tuning(const nyx_plan* pl, int32_t* t) {
  if (!pl || !t) return NYX_ERR_ARG;
  for (int i = 0; i < N_BLOCK_CLASSES; ++i) t[i] = pl->kp.lim_pix[i];
  t[N_BLOCK_CLASSES] = pl->kp.scan_rpt;
  return NYX_OK;
}

nyx_status nyx_set_scan_staging(nyx_plan* pl, int mode) {
  if (!pl) return NYX_ERR_ARG;
  if (mode != 0 && mode != 1) return fail(pl->ctx, NYX_ERR_ARG, "scan staging must be 0 or 1");
  pl->kp.scan_stage = mode;
  drop_graph(pl);
  return NYX_OK;
}

nyx_status nyx_get_scan_staging(const nyx_plan* pl, int* mode) {
  if (!pl || !mode) return NYX_ERR_ARG;
  *mode = pl->kp.scan_stage;
  return NYX_OK;
}

nyx_status nyx_set_class_limits(nyx_plan* pl, const int32_t* lim_pix) {
  if (!pl || !lim_pix) return NYX_ERR_ARG;
  for (int i = 0; i < N_BLOCK_CLASSES; ++i)
    if (lim_pix[i] < 0 || lim_pix[i] > c_class_pix[i])
      return fail(pl->ctx, NYX_ERR_ARG, "class limit %d out of 0..%d", i, c_class_pix[i]);
  for (int i = 0; i < N_BLOCK_CLASSES; ++i) pl->kp.lim_pix[i] = lim_pix[i];
  drop_graph(pl);
  return NYX_OK;
}

nyx_status nyx_profile_enable(nyx_plan* pl, int slots) {
  if (!pl || slots < 0 || slots > 1024) return NYX_ERR_ARG;
  NYX_CUDA(pl->ctx, cudaSetDevice(pl->ctx->device));
  NYX_CUDA(pl->ctx, cudaDeviceSynchronize());
  for (cudaEvent_t e : pl->ev) cudaEventDestroy(e);
  pl->ev.assign((size_t)slots * (NYX_N_PHASES + 1), nullptr);
  for (auto& e : pl->ev) NYX_CUDA(pl->ctx, cudaEventCreate(&e));
  pl->prof_slots = slots;
  pl->prof_count = 0;
  return NYX_OK;
}

nyx_status nyx_graph_phase_events(nyx_plan* pl, int enable) {
  if (!pl) return NYX_ERR_ARG;
  NYX_CUDA(pl->ctx, cudaSetDevice(pl->ctx->device));
  if (enable && !pl->gev[0])
    for (auto& e : pl->gev) NYX_CUDA(pl->ctx, cudaEventCreate(&e));
  if ((enable != 0) != pl->gph) {
    NYX_CUDA(pl->ctx, cudaDeviceSynchronize());
    drop_graph(pl);  // the captured sequences differ by the event nodes
  }
  pl->gph = enable != 0;
  return NYX_OK;
}

nyx_status nyx_graph_phase_times(nyx_plan* pl, float* ms, int n) {
  if (!pl || !ms) return NYX_ERR_ARG;
  if (!pl->gph || !pl->use_graphs) return fail(pl->ctx, NYX_ERR_STATE, "graph phase events are off");
  NYX_CUDA(pl->ctx, cudaEventSynchronize(pl->gev[2 * NYX_GPH_ALL + 1]));
  for (int i = 0; i < n && i < NYX_N_GPHASES; ++i)
    NYX_CUDA(pl->ctx, cudaEventElapsedTime(&ms[i], pl->gev[2 * i], pl->gev[2 * i + 1]));
  return NYX_OK;
}

nyx_status nyx_phase_times(nyx_plan* pl, int back, float* ms, int n) {
  if (!pl || !ms || back < 0 || back >= pl->prof_slots) return NYX_ERR_ARG;
  if (back >= pl->prof_count) return fail(pl->ctx, NYX_ERR_STATE, "extract not recorded");
  const int64_t which = pl->prof_count - 1 - back;
  cudaEvent_t* ev = &pl->ev[(size_t)(which % pl->prof_slots) * (NYX_N_PHASES + 1)];
  NYX_CUDA(pl->ctx, cudaEventSynchronize(ev[NYX_N_PHASES]));
  for (int i = 0; i < n && i < NYX_N_PHASES; ++i) NYX_CUDA(pl->ctx, cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]));
  return NYX_OK;
}

nyx_status nyx_sync_status(nyx_plan* pl, void* stream) {
  if (!pl) return NYX_ERR_ARG;
  NYX_CUDA(pl->ctx, cudaSetDevice(pl->ctx->device));
  return read_err(pl, (cudaStream_t)stream);
}

nyx_status nyx_debug_select(nyx_plan* pl, int64_t roi) {
  if (!pl) return NYX_ERR_ARG;
  pl->dbg_roi = roi;
  if (roi >= 0 && !pl->d_dbg && pl->prm.glcm_levels > 0) {
    NYX_CUDA(pl->ctx, cudaSetDevice(pl->ctx->device));
    NYX_CUDA(pl->ctx, cudaMalloc(&pl->d_dbg, 4ull * pl->n_off * pl->prm.glcm_levels * pl->prm.glcm_levels));
  }
  return NYX_OK;
}

nyx_status nyx_debug_glcm(nyx_plan* pl, int off, uint32_t* h_counts) {
  if (!pl || !h_counts || off < 0 || off >= pl->n_off || !pl->d_dbg) return NYX_ERR_ARG;
  const int ng = pl->prm.glcm_levels;
  NYX_CUDA(pl->ctx, cudaSetDevice(pl->ctx->device));
  NYX_CUDA(pl->ctx, cudaDeviceSynchronize());
  NYX_CUDA(pl->ctx, cudaMemcpy(h_counts, pl->d_dbg + (size_t)off * ng * ng, 4ull * ng * ng, cudaMemcpyDeviceToHost));
  return NYX_OK;
}

nyx_status nyx_debug_bins(nyx_plan* pl, const void* d_img, const int32_t* d_mask, uint16_t* d_bins, void* stream) {
  if (!pl || !d_bins) return NYX_ERR_ARG;
  nyx_status s = check_ptrs(pl, d_img, d_mask);
  if (s != NYX_OK) return s;
  if (pl->prm.glcm_levels < 2) return fail(pl->ctx, NYX_ERR_ARG, "plan has no GLCM levels");
  cudaStream_t st = (cudaStream_t)stream;
  nyx_ctx* c = pl->ctx;
  NYX_CUDA(c, cudaSetDevice(c->device));
  KParams k = pl->kp;
  k.img = d_img;
  k.mask = d_mask;
  k.vec = (k.nx % 4) == 0;
  k.cap_roi = pl->prm.max_rois;
  if ((s = flush_live(pl, st)) != NYX_OK) return s;
  if ((s = run_front(pl, k, st)) != NYX_OK) return s;
  if ((s = run_sort_setup(pl, k, st)) != NYX_OK) return s;
  NYX_CUDA(c, launch_debug_bins(k, d_bins, c->nsm, st));
  if ((s = run_reset(pl, k, st)) != NYX_OK) return s;
  return read_err(pl, st);
}

nyx_status nyx_backward(nyx_plan* pl, const void* d_img, const int32_t* d_mask, const double* d_grad_table,
                        float* d_grad_img, void* stream) {
  if (!pl || !d_grad_table || !d_grad_img) return NYX_ERR_ARG;
  nyx_status s = check_ptrs(pl, d_img, d_mask);
  if (s != NYX_OK) return s;
  if (!pl->have_saved) return fail(pl->ctx, NYX_ERR_STATE, "no forward pass saved for backward");
  cudaStream_t st = (cudaStream_t)stream;
  nyx_ctx* c = pl->ctx;
  NYX_CUDA(c, cudaSetDevice(c->device));
  KParams k = pl->kp;
  k.img = d_img;
  k.mask = d_mask;
  k.vec = (k.nx % 4) == 0;
  k.saved = pl->d_saved;
  k.cap_roi = pl->prm.max_rois;
  // the label -> ROI map of the saved forward pass is still in the table when
  // the image and mask are the same buffers; otherwise rebuild it
  if (!(pl->table_live && pl->live_img == d_img && pl->live_mask == d_mask)) {
    if ((s = flush_live(pl, st)) != NYX_OK) return s;
    if ((s = run_front(pl, k, st)) != NYX_OK) return s;
    if ((s = run_sort_setup(pl, k, st)) != NYX_OK) return s;
  }
  pl->table_live = false;
  cudaError_t e = launch_backward(k, d_grad_table, d_grad_img, c->nsm, st);
  if (e != cudaSuccess) return fail(c, NYX_ERR_CUDA, "backward launch failed: %s", cudaGetErrorString(e));
  return run_reset(pl, k, st);
}

}  // extern "C"
