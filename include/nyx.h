/*
 * nyx.h -- C ABI of the GB300 per-ROI feature-extraction library (libnyxgpu).
 *
 * The operation (arxiv 2603.12016, "Nyxus", section "Nyxus architecture" and
 * "Feature Control and Tunability"): given an intensity image and an integer
 * label mask of the same shape, separate the pixels of every labelled region
 * of interest (ROI) and compute, per ROI, a selected set of features --
 * first-order intensity statistics (Table S1 / S5), raw, central and
 * normalised geometric moments with Hu invariants (Table S2 rows 123-135,
 * Table S5 rows 368/370) and grey-level co-occurrence (GLCM) features (Table
 * S3 rows 140-174, Table S5 row 361) -- under hyperparameters chosen by the
 * caller (grey depth g, offsets s, histogram bins h of the O(m,h) and
 * O(m,g,s) cost model).  The result is one FP64 row per ROI.
 *
 * Conventions shared by every call:
 *   - Device pointers ("d_" prefix) are owned by the caller and must stay
 *     valid until the stream has passed the end of the call.  The library
 *     never frees or retains them.
 *   - Calls are stream-ordered on the `stream` argument (a cudaStream_t
 *     passed as void*; NULL = legacy default stream) and asynchronous unless
 *     stated otherwise.
 *   - Every call returns a nyx_status.  No C++ exception crosses the ABI.
 *     Errors found on the device (negative label, non-finite float pixel
 *     inside an ROI, capacity overflow) are recorded in a device error word
 *     and reported by nyx_sync_status() or by a call made with NYX_SYNC.
 *   - A context (nyx_ctx) and its plans may be used from one host thread at
 *     a time.
 */
#ifndef NYX_H_
#define NYX_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NYX_ABI_VERSION 1

typedef enum {
  NYX_OK = 0,
  NYX_ERR_ARG = 1,        /* null pointer, out-of-range parameter, misaligned pointer */
  NYX_ERR_DTYPE = 2,      /* unsupported pixel dtype */
  NYX_ERR_SHAPE = 3,      /* dims / batch inconsistent or too large */
  NYX_ERR_BAD_LABEL = 4,  /* a negative label in the mask */
  NYX_ERR_NONFINITE = 5,  /* NaN or Inf float pixel inside an ROI */
  NYX_ERR_CAPACITY = 6,   /* more ROIs than cap_roi / plan max_rois, or an ROI beyond the size limits */
  NYX_ERR_CUDA = 7,       /* a CUDA runtime call failed (message in nyx_last_error) */
  NYX_ERR_OOM = 8,        /* device allocation of the plan workspace failed */
  NYX_ERR_TIMEOUT = 9,    /* a bounded device wait ran out */
  NYX_ERR_STATE = 10      /* call out of order (e.g. backward without a saved forward) */
} nyx_status;

typedef enum { NYX_U16 = 0, NYX_I16 = 1, NYX_F32 = 2 } nyx_dtype;

/* Arithmetic of the per-pixel accumulations.  FP32_COMP: FP32 partial sums
 * merged with two-sum compensation, centred at a pass-1 reference, FP64 only
 * for per-ROI normalisation.  FP64_PLAIN: the same per-ROI algorithm with
 * FP64 accumulation throughout (the in-repo comparison path). */
typedef enum { NYX_PREC_FP32_COMP = 0, NYX_PREC_FP64_PLAIN = 1 } nyx_prec;

/* Flags of nyx_extract. */
#define NYX_SAVE_FOR_BACKWARD 1u /* keep per-ROI state (and the label -> ROI map) for nyx_backward */
#define NYX_SYNC 2u              /* synchronise the stream and return the device error word */

/* Hyperparameters of one plan.  POD; set struct_size = sizeof(nyx_params)
 * (ABI versioning).  Zero-initialise and fill; nyx_params_default() gives the
 * untargeted default profile. */
typedef struct {
  uint32_t struct_size;
  int32_t ndim;              /* 2 or 3 spatial dimensions */
  int64_t dims[3];           /* (x, y, z) extent of ONE image; z = 1 for 2D.  Row-major
                                [batch][z][y][x], dense (pitch = x) */
  int32_t batch;             /* images of identical shape stored back to back (>= 1) */
  int32_t dtype;             /* nyx_dtype */
  uint64_t feature_mask[4];  /* bit i selects feature id i (nyx_feature_id); all ones =
                                untargeted extraction, a subset = targeted */
  int32_t glcm_levels;       /* grey levels Ng of the GLCM quantisation, 2..256 (0 = no GLCM) */
  int32_t n_dist;            /* number of GLCM distances (1..8) */
  int32_t dists[8];          /* GLCM distances (Chebyshev), each 1..8 */
  int32_t glcm_per_offset_cols; /* 0: mean over directions per distance; 1: also one column
                                   per (distance, direction) */
  int32_t hist_bins;         /* bins of the entropy / uniformity histogram, 2..4096 */
  int32_t precision;         /* nyx_prec */
  int64_t max_rois;          /* upper bound on ROIs per call (sizes the workspace) */
} nyx_params;

typedef struct nyx_ctx nyx_ctx;
typedef struct nyx_plan nyx_plan;

/* Fill *p with the default untargeted profile for a 2D uint16 image of the
 * given extent: all features, Ng = 64, distance 1, 256 histogram bins,
 * FP32_COMP, max_rois = 65536.  Always succeeds for non-null p. */
nyx_status nyx_params_default(nyx_params* p, int64_t nx, int64_t ny);

/* Create a context bound to CUDA device `device`.  *out owns only library
 * state.  Errors: NYX_ERR_ARG (null out), NYX_ERR_CUDA (bad device). */
nyx_status nyx_create(nyx_ctx** out, int device);
void nyx_destroy(nyx_ctx* ctx);

/* Message of the last failing call on this context (static storage owned by
 * the context, valid until the next call on it). */
const char* nyx_last_error(const nyx_ctx* ctx);

/* Validate params and allocate the plan's device workspace (hash tables,
 * per-ROI state, accumulators), sized by dims, batch and max_rois.  The plan
 * owns its workspace and frees it in nyx_plan_destroy.
 * Errors: NYX_ERR_ARG / NYX_ERR_DTYPE / NYX_ERR_SHAPE (params), NYX_ERR_OOM. */
nyx_status nyx_plan_create(nyx_ctx* ctx, const nyx_params* params, nyx_plan** out);
void nyx_plan_destroy(nyx_plan* plan);

/* Number of FP64 columns of one output row, and the name of column `col`
 * (NUL-terminated, truncated to cap).  Column order: LABEL, IMAGE, AREA,
 * bounding box, centroid, then the selected features in feature-id order;
 * GLCM features expand to one column per distance (suffix _D<d>) and, when
 * glcm_per_offset_cols = 1, one per direction (_A<deg> in 2D, _O<k> in 3D). */
nyx_status nyx_num_columns(const nyx_plan* plan, int* n_col);
nyx_status nyx_column_name(const nyx_plan* plan, int col, char* buf, size_t cap);

/* Feature id of a feature name (e.g. "MEAN", "INT_HU", "GLCM_CONTRAST"), -1
 * if unknown.  Ids: 0..40 first-order statistics (Table S1 / S5), 41..50
 * moment families, one id each (INT_M, INT_MU, INT_ETA, INT_NU, INT_HU and
 * the BIN_ variants; Table S2 rows 123-135), 51..80 GLCM features (Table S3
 * rows 140-174), 81..85 edge intensity statistics (Table S1 rows 3-7,
 * Table S5): EDGE_INTEGRATED_INTENSITY, EDGE_MAX_INTENSITY,
 * EDGE_MIN_INTENSITY, EDGE_MEAN_INTENSITY, EDGE_STDDEV_INTENSITY over the
 * ROI's edge pixels, those with a face neighbour (4 in 2D, 6 in 3D) outside
 * the ROI or the image; the deviation is the unbiased one (0 for a single
 * edge pixel); 86..90 NGTDM features (Table S3 rows 246-250, need
 * glcm_levels > 0): NGTDM_COARSENESS, NGTDM_CONTRAST, NGTDM_BUSYNESS,
 * NGTDM_COMPLEXITY, NGTDM_STRENGTH on the GLCM grey levels, over the pixels
 * with at least one ROI pixel among their 8 (2D) / 26 (3D) neighbours;
 * 91..104 GLDM features (Table S3 rows 251-264, need glcm_levels > 0):
 * GLDM_SDE, GLDM_LDE, GLDM_GLN, GLDM_DN, GLDM_DNN, GLDM_GLV, GLDM_DV,
 * GLDM_DE, GLDM_LGLE, GLDM_HGLE, GLDM_SDLGLE, GLDM_SDHGLE, GLDM_LDLGLE,
 * GLDM_LDHGLE of the grey-level dependence matrix on the GLCM grey levels,
 * the dependence of a pixel being 1 + the number of its 8 / 26 neighbours
 * in the ROI at its own level. */
int nyx_feature_id(const char* name);

/* Run the label scan only and return the number of ROIs (distinct
 * (image, label > 0) pairs) in *n_roi.  Synchronises `stream` (reads 8 bytes
 * back).  d_img: dims x batch pixels of params.dtype; d_mask: int32, same
 * shape; both 16-byte aligned.  Errors: NYX_ERR_ARG, NYX_ERR_BAD_LABEL,
 * NYX_ERR_CAPACITY (more than max_rois), NYX_ERR_CUDA.
 * Staging (this call and every extraction): by default, when both row
 * pitches (x extent times the pixel size, and times 4 for the mask) are
 * multiples of 16 bytes, the scan stages rows of image and mask into shared
 * memory by 2D bulk tensor copies (TMA); otherwise, or after
 * nyx_set_scan_staging(plan, 1), it loads them into registers.  The results
 * are identical. */
nyx_status nyx_count_rois(nyx_plan* plan, const void* d_img, const int32_t* d_mask, int64_t* n_roi,
                          void* stream);

/* Extract the feature table.  Rows are the ROIs in ascending
 * (image, label) order.  d_table: caller-allocated FP64 [cap_roi x n_col],
 * row-major; rows >= n_roi are left untouched.  d_n_roi: device int64
 * receiving the ROI count (may be NULL).  flags: NYX_SAVE_FOR_BACKWARD,
 * NYX_SYNC.  Without NYX_SYNC the call is asynchronous and device-detected
 * errors surface at the next nyx_sync_status().
 * Errors: NYX_ERR_ARG (null/misaligned pointers, cap_roi < 0), NYX_ERR_STATE
 * (plan busy), NYX_ERR_CUDA; with NYX_SYNC also the device-detected codes. */
nyx_status nyx_extract(nyx_plan* plan, const void* d_img, const int32_t* d_mask, double* d_table, int64_t cap_roi,
                       int64_t* d_n_roi, uint32_t flags, void* stream);

/* CUDA graphs.  By default a plan captures its extraction launch sequence
 * (label scan, key sort, the size-class kernels, GLCM features, table reset)
 * into a CUDA graph the first time it sees a given set of arguments (device
 * pointers, cap_roi, flags, class limits) and replays it on later calls with
 * the same arguments; new arguments trigger a new capture.  Capture uses a
 * stream owned by the plan, so `stream` may be the legacy default stream; the
 * graph is launched on `stream`.  Calls with profiling enabled launch
 * directly.  nyx_use_graphs(plan, 0) switches to direct launches;
 * nyx_graph_captures reports how many captures the plan has made.  Not in
 * the paper.  Errors: NYX_ERR_ARG (null plan / n). */
nyx_status nyx_use_graphs(nyx_plan* plan, int enable);
nyx_status nyx_graph_captures(const nyx_plan* plan, int64_t* n);

/* Size classes (the paper, "Results, Scalability": how much the GPU helps
 * depends on ROI size and count, Fig. 3f/g).  Every ROI
 * goes to the first class whose pixel limit and padded bounding-box cell
 * capacity it fits: one warp per ROI (capacity 256 px / 1,024 cells), one
 * 128-thread block (1,024 / 4,096), one 256-thread block (4,096 / 8,192; two
 * blocks per SM), one 512-thread block (8,192 / 16,384; one block per SM),
 * else the multi-block path.  lim_pix[NYX_N_CLASSES] sets the pixel limits
 * of these block classes (0 disables a class; each at most its capacity).
 * nyx_autotune times the extraction of (d_img, d_mask) under a grid of
 * limits (warp 0/64/128/256, small 0/512/1024, medium 0/2048/4096, large
 * 0/8192), then times the label scan alone under its tile heights (8/16/32
 * rows per warp, tiles of 128 columns by 64/128/256 rows) and both stagings
 * of its rows (below); each candidate is timed
 * as the median of `reps` calls, every call preceded by a 256 MB write that
 * flushes the L2 cache (allocated and freed inside this call).  It keeps the
 * fastest setting in the plan and returns the limits in h_lim_pix (host
 * int32[NYX_N_CLASSES], may be NULL); nyx_get_tuning reads the tile height
 * too.
 * d_table / cap_roi as in nyx_extract.  Synchronises.  Results do not depend
 * on these settings beyond floating-point rounding.  Limits whose extraction
 * ends in NYX_ERR_CAPACITY (so many ROIs routed to the multi-block class
 * that its workspace overflows) are skipped as candidates.  Errors:
 * NYX_ERR_ARG, and those of nyx_extract.
 * nyx_set_tuning / nyx_get_tuning: t[0..NYX_N_CLASSES) the class pixel
 * limits as above, t[NYX_N_CLASSES] the scan's rows per warp (0: chosen from
 * the tile count; else 4, 8, 16 or 32); t is host int32[NYX_N_CLASSES + 1].
 * nyx_set_scan_staging / nyx_get_scan_staging: how the label scan reads its
 * rows, 0 = bulk tensor copies into shared memory where the row pitch
 * allows (the default), 1 = register loads; the autotuner times both with
 * each tile height.  Errors: NYX_ERR_ARG. */
#define NYX_N_CLASSES 4
nyx_status nyx_set_class_limits(nyx_plan* plan, const int32_t* lim_pix);
nyx_status nyx_set_tuning(nyx_plan* plan, const int32_t* t);
nyx_status nyx_get_tuning(const nyx_plan* plan, int32_t* t);
nyx_status nyx_set_scan_staging(nyx_plan* plan, int mode);
nyx_status nyx_get_scan_staging(const nyx_plan* plan, int* mode);
nyx_status nyx_autotune(nyx_plan* plan, const void* d_img, const int32_t* d_mask, double* d_table, int64_t cap_roi,
                        int reps, void* stream, int32_t* h_lim_pix);

/* Source of one tile of a mosaic for nyx_extract_tiles: fill h_img (w x h
 * pixels of the plan's dtype, row-major dense) and h_mask (int32, w x h) with
 * the tile whose top-left pixel is (x0, y0).  Both buffers are pinned host
 * memory owned by the library, valid during the call only.  Return 0 on
 * success; any other value aborts the extraction. */
typedef int (*nyx_tile_fn)(void* user, int64_t x0, int64_t y0, int64_t w, int64_t h, void* h_img, int32_t* h_mask);

/* Streamed extraction of a large 2D mosaic (the plan's dims; batch 1), the
 * whole-slide regime of "Results, Scalability" where host-to-device traffic
 * decides GPU benefit.  Tiles of tile_w x tile_h (edge tiles smaller) are
 * requested from `fn` in row-major tile order into two pinned staging
 * buffers, copied into d_img / d_mask (caller-allocated device buffers of
 * the whole mosaic, 16-byte aligned, filled by this call), and every band of
 * tile rows is label-scanned as soon as its tiles are in, while the host
 * produces the next tiles.  After the last band the per-ROI kernels run on
 * the device-resident mosaic, so ROIs crossing tile borders are merged in the
 * label table (counts, bounding boxes, intensity ranges) and processed whole.
 * Output as nyx_extract (d_table FP64 [cap_roi x n_col], rows in ascending
 * label order; d_n_roi device int64 or NULL).  flags: NYX_SYNC only.  The
 * call returns once every tile has been handed to the stream.  Plans above
 * 16,384 ROIs sort their keys with a multi-block merge sort.  Errors:
 * NYX_ERR_ARG (null fn/pointers, bad tile extent, the source failed),
 * NYX_ERR_SHAPE (plan not 2D or batch > 1), NYX_ERR_OOM (staging), and with
 * NYX_SYNC the device-detected codes. */
nyx_status nyx_extract_tiles(nyx_plan* plan, int64_t tile_w, int64_t tile_h, nyx_tile_fn fn, void* user, void* d_img,
                             int32_t* d_mask, double* d_table, int64_t cap_roi, int64_t* d_n_roi, uint32_t flags,
                             void* stream);

/* Synchronise `stream` and return the device error word of the plan's last
 * calls as a status (NYX_OK if clean); clears the word. */
nyx_status nyx_sync_status(nyx_plan* plan, void* stream);

/* Backward pass of the smooth intensity features (first-order statistics
 * except order statistics, weighted centroids, mass displacement, every
 * intensity-weighted moment, and the edge integrated intensity, mean and
 * deviation, differentiated on the fixed edge set) with respect to the pixel
 * intensities: given
 * dL/dF for every output cell (d_grad_table, FP64 [n_roi x n_col], same
 * layout as the last nyx_extract made with NYX_SAVE_FOR_BACKWARD), write
 * dL/dI for every pixel to d_grad_img (FP32, image shape; 0 outside ROIs).
 * Non-smooth columns (min/max, order statistics, histogram, GLCM, NGTDM,
 * GLDM, binary moments, geometry) contribute nothing.  Not in the paper: it
 * makes the features usable as a differentiable layer for the AI/ML use the
 * paper's introduction motivates.  When d_img / d_mask are the buffers of that
 * forward pass, its label -> ROI map is reused (the forward pass kept it);
 * otherwise the map is rebuilt by a label scan of d_mask.  Any other call on
 * the plan releases a kept map first.  Errors: NYX_ERR_STATE (no saved
 * forward), NYX_ERR_ARG, NYX_ERR_CUDA. */
nyx_status nyx_backward(nyx_plan* plan, const void* d_img, const int32_t* d_mask, const double* d_grad_table,
                        float* d_grad_img, void* stream);

/* Test hook: GLCM counts of ROI row `roi` (0-based, ascending key order) for
 * offset index `off` (distance index * n_directions + direction) as found by
 * the last nyx_extract, written densely to h_counts (host, uint32 [Ng x Ng],
 * symmetric).  Requires that nyx_debug_select(plan, roi) preceded that
 * extract.  Synchronises. */
nyx_status nyx_debug_select(nyx_plan* plan, int64_t roi);
nyx_status nyx_debug_glcm(nyx_plan* plan, int off, uint32_t* h_counts);

/* Test hook: per-pixel GLCM bin index (rule: b = floor(Ng (x - min)/(max - min)),
 * clamped to Ng-1, per-ROI min/max; 0xFFFF outside ROIs) of the last
 * extract's image, written to d_bins (device uint16, image shape). */
nyx_status nyx_debug_bins(nyx_plan* plan, const void* d_img, const int32_t* d_mask, uint16_t* d_bins,
                          void* stream);

/* Profiling hook (not in the paper): with `slots` > 0, every nyx_extract
 * records CUDA events on its stream between its phases into a ring of
 * `slots` event sets (slots = 0 turns recording off).  nyx_phase_times waits
 * for the events of the extract `back` calls ago (0 = the last one, up to
 * slots - 1) and writes up to NYX_N_PHASES durations in milliseconds:
 * [0] counters + label scan, [1] key sort + per-ROI setup, [2] ROI kernel of
 * the warp class (one warp per ROI), [3] of the small block class, [4] of the
 * medium block class, [5] of the large block class, [6] the multi-block
 * class (ROIs larger than a block stages; with GLRLM / GLSZM selected it
 * includes their kernels), [7] statistics, moments and GLCM features from the
 * per-ROI sums, [8] table reset.
 * Errors: NYX_ERR_ARG (null plan/ms, slots out of 0..1024, back out of
 * range), NYX_ERR_STATE (that extract was not recorded), NYX_ERR_CUDA. */
#define NYX_N_PHASES 9
nyx_status nyx_profile_enable(nyx_plan* plan, int slots);
nyx_status nyx_phase_times(nyx_plan* plan, int back, float* ms, int n);

/* Profiling hook (not in the paper) for the graph-replayed extraction: with
 * enable != 0 the captured graph of nyx_extract also records, as event
 * nodes, a begin and an end CUDA event around each phase, on the stream that
 * phase runs on (the size classes run as parallel branches).  Toggling drops
 * the cached graphs.  nyx_graph_phase_times waits for the most recent replay
 * and writes up to NYX_N_GPHASES durations in milliseconds, indexed by
 * NYX_GPH_*: label scan, key sort + setup, the warp / small / medium / large
 * block classes, the multi-block class, the GLCM feature kernel, the statistics
 * kernel, the table reset, the per-ROI stage (from before the size classes
 * fork to after they join: the four classes run as concurrent branches, so
 * each class's own span includes waiting for SMs that the others hold), and
 * the whole extraction, and the GLRLM / GLSZM kernels (block classes, then
 * multi-block ROIs: a branch of their own beside the size classes, inside
 * the per-ROI stage).  A class that receives no ROI reads as about 0.
 * Errors: NYX_ERR_ARG (null plan/ms), NYX_ERR_STATE (events off or graphs
 * off), NYX_ERR_CUDA. */
enum {
  NYX_GPH_SCAN = 0, NYX_GPH_SORT, NYX_GPH_WARP, NYX_GPH_SMALL, NYX_GPH_MED, NYX_GPH_LARGE, NYX_GPH_BIG, NYX_GPH_GLCMF,
  NYX_GPH_STATSF, NYX_GPH_RESET, NYX_GPH_ROI, NYX_GPH_ALL, NYX_GPH_RZ, NYX_N_GPHASES
};
nyx_status nyx_graph_phase_events(nyx_plan* plan, int enable);
nyx_status nyx_graph_phase_times(nyx_plan* plan, float* ms, int n);

/* Allocation-free ROI count (the paper has no counterpart; this is a service
 * for callers that may not allocate device memory).  Some hosts cannot let a
 * library call cudaMalloc: applications that hand all device memory to their
 * own pool allocator and forbid plug-ins from allocating, programs running
 * under a fixed device-memory quota on a shared node or an acquisition
 * workstation, and code paths that cannot afford cudaMalloc's implicit
 * device synchronisation.  This call counts the ROIs of an image exactly like
 * nyx_count_rois, with no context, no plan and no allocation: its label table
 * lives in a fixed array inside the library, of about 2 MB per GPU, which
 * every GPU that loads the library holds until the process exits.
 *   params : dims, batch, dtype and ndim are read (other fields ignored);
 *            struct_size must be sizeof(nyx_params)
 *   d_img, d_mask : device pointers as for nyx_count_rois, 16-byte aligned
 *   n_roi  : host int64 receiving the count
 * Limits: at most NYX_NOALLOC_MAX_LABELS distinct (image, label) pairs and a
 * batch of at most NYX_NOALLOC_MAX_BATCH images; beyond either the call
 * returns NYX_ERR_CAPACITY.  The first call on a device resolves the array's
 * device address (cudaGetSymbolAddress) with that device current, so make it
 * before any stream capture.  All calls share the one array: calls whose work
 * overlaps on the GPU (other streams, other host threads) race and must be
 * serialised by the caller.  The call synchronises `stream`.
 * Errors: NYX_ERR_ARG, NYX_ERR_SHAPE, NYX_ERR_DTYPE, NYX_ERR_BAD_LABEL,
 * NYX_ERR_NONFINITE, NYX_ERR_CAPACITY, NYX_ERR_CUDA. */
#define NYX_NOALLOC_MAX_LABELS 16384
#define NYX_NOALLOC_MAX_BATCH 1024
nyx_status nyx_count_rois_noalloc(const nyx_params* params, const void* d_img, const int32_t* d_mask,
                                  int64_t* n_roi, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* NYX_H_ */
