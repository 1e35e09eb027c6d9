/*
 * nyx_oracle.c -- plain, slow FP64 CPU oracle for batched per-ROI feature
 * extraction (image + integer label mask in, one feature row per ROI out).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg use it.  It shares no code, header, table or
 * constant with the CUDA library.
 *
 * Sources (arxiv 2603.12016, "Nyxus"):
 *   - problem statement: intensity image + label mask in, per-ROI feature
 *     table out; ROI separation into per-ROI pixel sets ("Nyxus architecture"
 *     section, pixel-cloud paragraph);
 *   - feature inventory: Table S1 (2D intensity), Table S2 (shape/geometric
 *     and intensity moments, rows 123-135), Table S3 (GLCM rows 140-174,
 *     NGTDM rows 246-250, GLDM rows 251-264; GLRLM rows from 193 with the
 *     acronyms of its note, GLSZM rows 228-245, both on request),
 *     Table S5 (3D intensity, 3D GLCM row 361, 3D raw/central moments rows
 *     368/370);
 *   - the paper states IBSI compliance ("IBSI profile", Fig. 5) and defers
 *     formulas to external documentation, so every feature below is the
 *     textbook / IBSI definition written out literally;
 *   - cost structure O(m), O(m,h), O(m,g,s) (section "Feature Control and
 *     Tunability") names the histogram bin count h, grey depth g and spatial
 *     offset s used here as hist_bins, ng and dist[].
 *
 * Everything is computed literally: two-pass statistics, dense Ng x Ng GLCM
 * matrices per offset, every GLCM double sum written out in full.  Readings
 * where the paper is silent are listed in the repository design notes and
 * repeated at the point of use.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define ORC_U16 0
#define ORC_I16 1
#define ORC_F32 2
#define ORC_F64 3 /* oracle-only: used by finite-difference gradient checks */

#define ORC_MAX_DIST 8
#define ORC_MAX_DIR 13
#define ORC_NGLCM 30
#define ORC_NAME 48

typedef struct {
  int ndim;              /* 2 or 3 */
  int64_t nx, ny, nz;    /* extent of one image; nz = 1 for 2D */
  int batch;             /* number of images stored back to back */
  int dtype;             /* ORC_U16 / ORC_I16 / ORC_F32 / ORC_F64 */
  int ng;                /* GLCM grey levels */
  int n_dist;            /* number of GLCM distances */
  int dist[ORC_MAX_DIST];
  int hist_bins;         /* bins of the entropy / uniformity histogram */
  int families;          /* optional texture families: 1 = GLRLM, 2 = GLSZM (0 = neither) */
} orc_cfg;

/* ------------------------------------------------------------------------ */
/* GLCM offsets.  2D: angle 0 = (+1,0), 45 = (+1,-1),
 * 90 = (0,-1), 135 = (-1,-1) in (dx,dy) with the row index growing
 * downward.  3D: the 13 vectors of {-1,0,1}^3 whose first
 * nonzero component, read in the order (dz, dy, dx), is positive, enumerated
 * with dz outermost and dx fastest.  Distance d scales the unit vector. */
static int n_dirs(const orc_cfg* c) { return c->ndim == 3 ? 13 : 4; }

static void unit_dir(const orc_cfg* c, int k, int* dx, int* dy, int* dz) {
  if (c->ndim != 3) {
    static const int d2[4][2] = {{1, 0}, {1, -1}, {0, -1}, {-1, -1}};
    *dx = d2[k][0];
    *dy = d2[k][1];
    *dz = 0;
    return;
  }
  int idx = 0;
  for (int z = -1; z <= 1; ++z)
    for (int y = -1; y <= 1; ++y)
      for (int x = -1; x <= 1; ++x) {
        int first = z != 0 ? z : (y != 0 ? y : x);
        if (first <= 0) continue;
        if (idx == k) {
          *dx = x;
          *dy = y;
          *dz = z;
          return;
        }
        ++idx;
      }
}

/* ------------------------------------------------------------------------ */
/* pixel access */
static double pixel(const orc_cfg* c, const void* img, int64_t gidx) {
  switch (c->dtype) {
    case ORC_U16: return (double)((const uint16_t*)img)[gidx];
    case ORC_I16: return (double)((const int16_t*)img)[gidx];
    case ORC_F32: return (double)((const float*)img)[gidx];
    default: return ((const double*)img)[gidx];
  }
}

/* Intensity binning, the IBSI fixed-bin-number rule: 0-based,
 * per-ROI min/max.  Integer inputs: b = floor(n (x - min) / (max - min)) in
 * 64-bit integers.  Float inputs: the same expression in FP64 with every
 * operation rounded separately (this file is compiled without FMA
 * contraction).  b is clamped to n-1; max == min gives b = 0. */
static int bin_of(const orc_cfg* c, double x, double mn, double mx, int n) {
  if (mx == mn) return 0;
  int64_t b;
  if (c->dtype == ORC_U16 || c->dtype == ORC_I16) {
    int64_t xi = (int64_t)x, lo = (int64_t)mn, hi = (int64_t)mx;
    b = ((int64_t)n * (xi - lo)) / (hi - lo);
  } else {
    volatile double num = (double)n * (x - mn);
    volatile double den = mx - mn;
    volatile double q = num / den;
    b = (int64_t)floor(q);
  }
  if (b > n - 1) b = n - 1;
  if (b < 0) b = 0;
  return (int)b;
}

/* ------------------------------------------------------------------------ */
/* ROI separation: gather, per (image, label), the ascending list of linear
 * pixel indices.  Label 0 is background. */
typedef struct {
  int64_t b;       /* image index in the batch */
  int32_t label;
  int64_t n;       /* pixel count */
  int64_t* lin;    /* linear index inside image b, ascending */
} roi_t;

typedef struct {
  int64_t key;
  int64_t lin;
} keyed_t;

static int cmp_keyed(const void* a, const void* b) {
  const keyed_t* x = (const keyed_t*)a;
  const keyed_t* y = (const keyed_t*)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  if (x->lin != y->lin) return x->lin < y->lin ? -1 : 1;
  return 0;
}

static int cmp_i64(const void* a, const void* b) {
  int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}

static int64_t roi_key(int64_t b, int32_t label) { return (b << 32) | (int64_t)(uint32_t)label; }

/* subset: sorted keys to keep (NULL = all).  Returns the number of ROIs, or
 * -1 on a negative label, -2 on allocation failure. */
static int64_t separate(const orc_cfg* c, const int32_t* mask, const int64_t* subset, int64_t n_subset,
                        roi_t** out) {
  const int64_t per = c->nx * c->ny * c->nz;
  const int64_t total = per * c->batch;
  int64_t m = 0;
  for (int64_t i = 0; i < total; ++i) {
    if (mask[i] < 0) return -1;
    if (mask[i] > 0) ++m;
  }
  keyed_t* kv = (keyed_t*)malloc(sizeof(keyed_t) * (size_t)(m > 0 ? m : 1));
  if (!kv) return -2;
  int64_t k = 0;
  for (int64_t i = 0; i < total; ++i) {
    if (mask[i] <= 0) continue;
    int64_t key = roi_key(i / per, mask[i]);
    if (subset && !bsearch(&key, subset, (size_t)n_subset, sizeof(int64_t), cmp_i64)) continue;
    kv[k].key = key;
    kv[k].lin = i % per;
    ++k;
  }
  qsort(kv, (size_t)k, sizeof(keyed_t), cmp_keyed);
  int64_t nr = 0;
  for (int64_t i = 0; i < k; ++i)
    if (i == 0 || kv[i].key != kv[i - 1].key) ++nr;
  roi_t* r = (roi_t*)calloc((size_t)(nr > 0 ? nr : 1), sizeof(roi_t));
  if (!r) {
    free(kv);
    return -2;
  }
  int64_t j = -1;
  for (int64_t i = 0; i < k; ++i) {
    if (i == 0 || kv[i].key != kv[i - 1].key) {
      ++j;
      r[j].b = kv[i].key >> 32;
      r[j].label = (int32_t)(kv[i].key & 0xffffffff);
      r[j].n = 0;
    }
    r[j].n++;
  }
  int64_t pos = 0;
  for (int64_t i = 0; i < nr; ++i) {
    r[i].lin = (int64_t*)malloc(sizeof(int64_t) * (size_t)r[i].n);
    if (!r[i].lin) {
      free(kv);
      return -2;
    }
    for (int64_t q = 0; q < r[i].n; ++q) r[i].lin[q] = kv[pos + q].lin;
    pos += r[i].n;
  }
  free(kv);
  *out = r;
  return nr;
}

static void free_rois(roi_t* r, int64_t n) {
  for (int64_t i = 0; i < n; ++i) free(r[i].lin);
  free(r);
}

/* ------------------------------------------------------------------------ */
/* Feature record.  Filled by compute_roi(), written out by emit_all() which
 * also produces the column names in the same order. */
typedef struct {
  double label, image, area;
  double bbox_min[3], bbox_ext[3], centroid[3];
  /* Table S1 / S5 intensity features */
  double mean, min, max, range, var, var_b, std, std_b, skew, kurt, exkurt, hskew, hflat;
  double energy, rms, se, mad, medad, ii, wc[3], md, cov, covered, piu;
  double median, p01, p10, p25, p75, p90, p99, iqr, qcod, rmean, rmad, mode, mode_prob;
  double entropy, uniformity;
  /* Table S2 rows 123-135 (2D) and Table S5 rows 368/370 (3D).  Index 0 =
   * intensity weighting, 1 = binary (shape) weighting. */
  double M[2][20], MU[2][20], ETA[2][20], NU[2][20], HU[2][7];
  /* Table S3 rows 140-174 (GLCM), per offset and mean per distance */
  double glcm_off[ORC_MAX_DIST][ORC_MAX_DIR][ORC_NGLCM];
  double glcm_mean[ORC_MAX_DIST][ORC_NGLCM];
  /* Table S1 rows 3-7 / Table S5 IIE, Max IE, Min IE, Mean IE, std IE:
   * intensity statistics over the ROI's edge pixels (edge test below) */
  double edge_ii, edge_max, edge_min, edge_mean, edge_std;
  /* Table S3 rows 246-250 (NGTDM): coarseness, contrast, busyness,
   * complexity, strength */
  double ngtdm[5];
  /* Table S3 rows 251-264 (GLDM) */
  double gldm[14];
  /* GLRLM (Table S3 rows from 193, acronyms of its note) and GLSZM (rows
   * 228-245), readings c19 / c20, in the order of SZ_NAMES below */
  double glrlm[16];
  double glszm[18];
} feat_t;

static const char* GLCM_NAMES[ORC_NGLCM] = {
    "ASM",       "ACOR",      "CLUPROM", "CLUSHADE", "CLUTEND", "CONTRAST", "CORR",   "DIFAVE",
    "DIFENTRO",  "DIFVAR",    "DIS",     "ENERGY",   "ENTROPY", "HOM1",     "HOM2",   "IDM",
    "INFOMEAS1", "INFOMEAS2", "IDMN",    "ID",       "IDN",     "IV",       "JAVE",   "JE",
    "JMAX",      "SUMAVE",    "SUMENT",  "JVAR",     "SUMVAR",  "VARIANCE"};

/* moment exponent lists: 2D (p,q) with p+q <= 3, 3D (p,q,r) with p+q+r <= 3 */
static int n_moments(const orc_cfg* c) { return c->ndim == 3 ? 20 : 10; }

static void moment_exp(const orc_cfg* c, int k, int* p, int* q, int* r) {
  int idx = 0;
  if (c->ndim == 3) {
    for (int a = 0; a <= 3; ++a)
      for (int b = 0; a + b <= 3; ++b)
        for (int d = 0; a + b + d <= 3; ++d) {
          if (idx == k) {
            *p = a;
            *q = b;
            *r = d;
            return;
          }
          ++idx;
        }
  } else {
    for (int a = 0; a <= 3; ++a)
      for (int b = 0; a + b <= 3; ++b) {
        if (idx == k) {
          *p = a;
          *q = b;
          *r = 0;
          return;
        }
        ++idx;
      }
  }
}

static int moment_index(const orc_cfg* c, int p, int q, int r) {
  for (int k = 0; k < n_moments(c); ++k) {
    int a, b, d;
    moment_exp(c, k, &a, &b, &d);
    if (a == p && b == q && d == r) return k;
  }
  return -1;
}

typedef struct {
  double* row;
  char (*names)[ORC_NAME];
  int k;
} emitter;

static void emit(emitter* e, double v, const char* fmt, ...) __attribute__((format(printf, 3, 4)));
#include <stdarg.h>
static void emit(emitter* e, double v, const char* fmt, ...) {
  if (e->names) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(e->names[e->k], ORC_NAME, fmt, ap);
    va_end(ap);
  }
  if (e->row) e->row[e->k] = v;
  e->k++;
}

static void emit_all(const orc_cfg* c, const feat_t* f, emitter* e) {
  const int d3 = c->ndim == 3;
  const char* ax[3] = {"X", "Y", "Z"};
  const int nax = d3 ? 3 : 2;
  emit(e, f->label, "LABEL");
  emit(e, f->image, "IMAGE");
  emit(e, f->area, "AREA");
  for (int a = 0; a < nax; ++a) emit(e, f->bbox_min[a], "BBOX_%sMIN", ax[a]);
  emit(e, f->bbox_ext[0], "BBOX_WIDTH");
  emit(e, f->bbox_ext[1], "BBOX_HEIGHT");
  if (d3) emit(e, f->bbox_ext[2], "BBOX_DEPTH");
  for (int a = 0; a < nax; ++a) emit(e, f->centroid[a], "CENTROID_%s", ax[a]);

  emit(e, f->mean, "MEAN");
  emit(e, f->min, "MIN");
  emit(e, f->max, "MAX");
  emit(e, f->range, "RANGE");
  emit(e, f->var, "VARIANCE");
  emit(e, f->var_b, "VARIANCE_BIASED");
  emit(e, f->std, "STDDEV");
  emit(e, f->std_b, "STDDEV_BIASED");
  emit(e, f->skew, "SKEWNESS");
  emit(e, f->kurt, "KURTOSIS");
  emit(e, f->exkurt, "EXCESS_KURTOSIS");
  emit(e, f->hskew, "HYPERSKEWNESS");
  emit(e, f->hflat, "HYPERFLATNESS");
  emit(e, f->energy, "ENERGY");
  emit(e, f->rms, "ROOT_MEAN_SQUARED");
  emit(e, f->se, "STANDARD_ERROR");
  emit(e, f->mad, "MEAN_ABSOLUTE_DEVIATION");
  emit(e, f->medad, "MEDIAN_ABSOLUTE_DEVIATION");
  emit(e, f->ii, "INTEGRATED_INTENSITY");
  for (int a = 0; a < nax; ++a) emit(e, f->wc[a], "WEIGHTED_CENTROID_%s", ax[a]);
  emit(e, f->md, "MASS_DISPLACEMENT");
  emit(e, f->cov, "COV");
  emit(e, f->covered, "COVERED_IMAGE_INTENSITY_RANGE");
  emit(e, f->piu, "UNIFORMITY_PIU");
  emit(e, f->median, "MEDIAN");
  emit(e, f->p01, "P01");
  emit(e, f->p10, "P10");
  emit(e, f->p25, "P25");
  emit(e, f->p75, "P75");
  emit(e, f->p90, "P90");
  emit(e, f->p99, "P99");
  emit(e, f->iqr, "INTERQUARTILE_RANGE");
  emit(e, f->qcod, "QCOD");
  emit(e, f->rmean, "ROBUST_MEAN");
  emit(e, f->rmad, "ROBUST_MEAN_ABSOLUTE_DEVIATION");
  emit(e, f->mode, "MODE");
  emit(e, f->mode_prob, "MODE_PROBABILITY");
  emit(e, f->entropy, "ENTROPY");
  emit(e, f->uniformity, "UNIFORMITY");

  const char* wname[2] = {"INT", "BIN"};
  for (int w = 0; w < 2; ++w) {
    char s[16];
    for (int k = 0; k < n_moments(c); ++k) {
      int p, q, r;
      moment_exp(c, k, &p, &q, &r);
      if (d3) snprintf(s, sizeof s, "%d%d%d", p, q, r);
      else snprintf(s, sizeof s, "%d%d", p, q);
      emit(e, f->M[w][k], "%s_M%s", wname[w], s);
    }
    for (int k = 0; k < n_moments(c); ++k) {
      int p, q, r;
      moment_exp(c, k, &p, &q, &r);
      if (d3) snprintf(s, sizeof s, "%d%d%d", p, q, r);
      else snprintf(s, sizeof s, "%d%d", p, q);
      emit(e, f->MU[w][k], "%s_MU%s", wname[w], s);
    }
    for (int k = 0; k < n_moments(c); ++k) {
      int p, q, r;
      moment_exp(c, k, &p, &q, &r);
      if (p + q + r < 2) continue;
      if (d3) snprintf(s, sizeof s, "%d%d%d", p, q, r);
      else snprintf(s, sizeof s, "%d%d", p, q);
      emit(e, f->ETA[w][k], "%s_ETA%s", wname[w], s);
    }
    if (!d3) {
      for (int k = 0; k < n_moments(c); ++k) {
        int p, q, r;
        moment_exp(c, k, &p, &q, &r);
        snprintf(s, sizeof s, "%d%d", p, q);
        emit(e, f->NU[w][k], "%s_NU%s", wname[w], s);
      }
      for (int h = 0; h < 7; ++h) emit(e, f->HU[w][h], "%s_HU%d", wname[w], h + 1);
    }
  }

  for (int di = 0; di < c->n_dist; ++di)
    for (int g = 0; g < ORC_NGLCM; ++g) emit(e, f->glcm_mean[di][g], "GLCM_%s_D%d", GLCM_NAMES[g], c->dist[di]);
  for (int di = 0; di < c->n_dist; ++di)
    for (int o = 0; o < n_dirs(c); ++o)
      for (int g = 0; g < ORC_NGLCM; ++g) {
        if (d3) emit(e, f->glcm_off[di][o][g], "GLCM_%s_D%d_O%d", GLCM_NAMES[g], c->dist[di], o);
        else emit(e, f->glcm_off[di][o][g], "GLCM_%s_D%d_A%d", GLCM_NAMES[g], c->dist[di], 45 * o);
      }

  if (c->ng > 0) {
    static const char* NG_NAMES[5] = {"COARSENESS", "CONTRAST", "BUSYNESS", "COMPLEXITY", "STRENGTH"};
    for (int q = 0; q < 5; ++q) emit(e, f->ngtdm[q], "NGTDM_%s", NG_NAMES[q]);
    static const char* GD_NAMES[14] = {"SDE", "LDE", "GLN", "DN", "DNN", "GLV", "DV",
                                       "DE", "LGLE", "HGLE", "SDLGLE", "SDHGLE", "LDLGLE", "LDHGLE"};
    for (int q = 0; q < 14; ++q) emit(e, f->gldm[q], "GLDM_%s", GD_NAMES[q]);
    static const char* RL_NAMES[16] = {"SRE", "LRE", "GLNU", "GLNUN", "RLNU", "RLNUN", "RP", "GLV",
                                       "RV", "RE", "LGLRE", "HGLRE", "SRLGLE", "SRHGLE", "LRLGLE", "LRHGLE"};
    static const char* SZ_NAMES[18] = {"SAE", "LAE", "GLNU", "GLNUN", "SZNU", "SZNUN", "ZP", "GLV", "ZV",
                                       "ZE", "LGLZE", "HGLZE", "SALGLE", "SAHGLE", "LALGLE", "LAHGLE", "GLM", "ZSM"};
    if (c->families & 1)
      for (int q = 0; q < 16; ++q) emit(e, f->glrlm[q], "GLRLM_%s", RL_NAMES[q]);
    if (c->families & 2)
      for (int q = 0; q < 18; ++q) emit(e, f->glszm[q], "GLSZM_%s", SZ_NAMES[q]);
  }
  emit(e, f->edge_ii, "EDGE_INTEGRATED_INTENSITY");
  emit(e, f->edge_max, "EDGE_MAX_INTENSITY");
  emit(e, f->edge_min, "EDGE_MIN_INTENSITY");
  emit(e, f->edge_mean, "EDGE_MEAN_INTENSITY");
  emit(e, f->edge_std, "EDGE_STDDEV_INTENSITY");
}

/* ------------------------------------------------------------------------ */
/* GLCM features of one dense Ng x Ng count matrix (Table S3 rows 140-174,
 * IBSI definitions, 1-based grey levels, log base 2).  Zero total -> every
 * feature NaN. */
static void glcm_features(int ng, const double* P, double* out) {
  double tot = 0;
  for (int i = 0; i < ng * ng; ++i) tot += P[i];
  if (tot == 0) {
    for (int g = 0; g < ORC_NGLCM; ++g) out[g] = NAN;
    return;
  }
  double* p = (double*)malloc(sizeof(double) * (size_t)ng * ng);
  double* px = (double*)calloc((size_t)ng, sizeof(double));
  double* py = (double*)calloc((size_t)ng, sizeof(double));
  double* pxpy = (double*)calloc((size_t)(2 * ng + 1), sizeof(double)); /* index k = i + j, 2..2ng */
  double* pxmy = (double*)calloc((size_t)ng, sizeof(double));           /* index k = |i - j|, 0..ng-1 */
  for (int a = 0; a < ng * ng; ++a) p[a] = P[a] / tot;
  for (int i = 1; i <= ng; ++i)
    for (int j = 1; j <= ng; ++j) {
      double v = p[(i - 1) * ng + (j - 1)];
      px[i - 1] += v;
      py[j - 1] += v;
      pxpy[i + j] += v;
      pxmy[abs(i - j)] += v;
    }
  double mux = 0, muy = 0;
  for (int i = 1; i <= ng; ++i) {
    mux += i * px[i - 1];
    muy += i * py[i - 1];
  }
  double sx2 = 0, sy2 = 0;
  for (int i = 1; i <= ng; ++i) {
    sx2 += (i - mux) * (i - mux) * px[i - 1];
    sy2 += (i - muy) * (i - muy) * py[i - 1];
  }
  double asm_ = 0, acor = 0, cprom = 0, cshade = 0, ctend = 0, contrast = 0, dis = 0, je = 0;
  double hom1 = 0, hom2 = 0, idmn = 0, idn = 0, jave = 0, jmax = 0, jvar = 0;
  for (int i = 1; i <= ng; ++i)
    for (int j = 1; j <= ng; ++j) {
      double v = p[(i - 1) * ng + (j - 1)];
      double s = i + j - mux - muy;
      asm_ += v * v;
      acor += (double)i * j * v;
      cprom += s * s * s * s * v;
      cshade += s * s * s * v;
      ctend += s * s * v;
      contrast += (double)(i - j) * (i - j) * v;
      dis += fabs((double)(i - j)) * v;
      if (v > 0) je -= v * log2(v);
      hom1 += v / (1.0 + fabs((double)(i - j)));
      hom2 += v / (1.0 + (double)(i - j) * (i - j));
      idmn += v / (1.0 + (double)(i - j) * (i - j) / ((double)ng * ng));
      idn += v / (1.0 + fabs((double)(i - j)) / ng);
      jave += i * v;
      if (v > jmax) jmax = v;
      jvar += (i - mux) * (i - mux) * v;
    }
  double corr = (sx2 == 0 || sy2 == 0) ? 1.0 : (acor - mux * muy) / sqrt(sx2 * sy2);
  double difave = 0, difvar = 0, difent = 0, iv = 0;
  for (int k = 0; k < ng; ++k) difave += k * pxmy[k];
  for (int k = 0; k < ng; ++k) {
    difvar += (k - difave) * (k - difave) * pxmy[k];
    if (pxmy[k] > 0) difent -= pxmy[k] * log2(pxmy[k]);
    if (k >= 1) iv += pxmy[k] / ((double)k * k);
  }
  double sumave = 0, sumvar = 0, sument = 0;
  for (int k = 2; k <= 2 * ng; ++k) sumave += k * pxpy[k];
  for (int k = 2; k <= 2 * ng; ++k) {
    sumvar += (k - sumave) * (k - sumave) * pxpy[k];
    if (pxpy[k] > 0) sument -= pxpy[k] * log2(pxpy[k]);
  }
  double hx = 0, hy = 0;
  for (int i = 0; i < ng; ++i) {
    if (px[i] > 0) hx -= px[i] * log2(px[i]);
    if (py[i] > 0) hy -= py[i] * log2(py[i]);
  }
  double hxy = je, hxy1 = 0, hxy2 = 0;
  for (int i = 0; i < ng; ++i)
    for (int j = 0; j < ng; ++j) {
      double v = p[i * ng + j];
      double pp = px[i] * py[j];
      if (v > 0) hxy1 -= v * log2(pp);
      if (pp > 0) hxy2 -= pp * log2(pp);
    }
  double hmax = hx > hy ? hx : hy;
  double im1 = hmax == 0 ? 0.0 : (hxy - hxy1) / hmax;
  double arg = 1.0 - exp(-2.0 * (hxy2 - hxy));
  double im2 = sqrt(arg > 0 ? arg : 0.0);

  double v[ORC_NGLCM] = {asm_,   acor, cprom, cshade, ctend, contrast, corr, difave, difent,   difvar,
                         dis,    sqrt(asm_), je, hom1, hom2,    hom2,     im1,  im2,    idmn,     hom1,
                         idn,    iv,   jave,  je,     jmax,  sumave,   sument, jvar,  sumvar,   jvar};
  memcpy(out, v, sizeof v);
  free(p);
  free(px);
  free(py);
  free(pxpy);
  free(pxmy);
}

/* Dense GLCM of one ROI for unit direction k at distance d: for every ROI
 * pixel q and its neighbour q + d*dir inside the same ROI, P[b_q][b_n] += 1
 * and P[b_n][b_q] += 1 (symmetric).  Bins come from the fixed-bin-number rule with
 * n = ng on the ROI's own min/max. */
static void roi_glcm(const orc_cfg* c, const void* img, const int32_t* mask, const roi_t* r, double mn, double mx,
                     int dir, int d, double* P) {
  const int64_t per = c->nx * c->ny * c->nz;
  const int64_t base = r->b * per;
  int dx, dy, dz;
  unit_dir(c, dir, &dx, &dy, &dz);
  dx *= d;
  dy *= d;
  dz *= d;
  memset(P, 0, sizeof(double) * (size_t)c->ng * c->ng);
  for (int64_t k = 0; k < r->n; ++k) {
    int64_t lin = r->lin[k];
    int64_t x = lin % c->nx, y = (lin / c->nx) % c->ny, z = lin / (c->nx * c->ny);
    int64_t X = x + dx, Y = y + dy, Z = z + dz;
    if (X < 0 || Y < 0 || Z < 0 || X >= c->nx || Y >= c->ny || Z >= c->nz) continue;
    int64_t nlin = (Z * c->ny + Y) * c->nx + X;
    if (mask[base + nlin] != r->label) continue;
    int a = bin_of(c, pixel(c, img, base + lin), mn, mx, c->ng);
    int b = bin_of(c, pixel(c, img, base + nlin), mn, mx, c->ng);
    P[a * c->ng + b] += 1;
    P[b * c->ng + a] += 1;
  }
}

static double percentile(const double* v, int64_t n, double q) {
  /* linear interpolation at h = (n-1) q ("type 7") */
  double h = (double)(n - 1) * q;
  int64_t lo = (int64_t)floor(h);
  if (lo >= n - 1) return v[n - 1];
  return v[lo] + (h - (double)lo) * (v[lo + 1] - v[lo]);
}

static int cmp_double(const void* a, const void* b) {
  double x = *(const double*)a, y = *(const double*)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}

/* Hu's seven invariants from normalised central moments (Hu 1962). */
static void hu7(double n20, double n02, double n11, double n30, double n21, double n12, double n03, double* h) {
  double a = n30 - 3 * n12, b = 3 * n21 - n03, s = n30 + n12, t = n21 + n03;
  h[0] = n20 + n02;
  h[1] = (n20 - n02) * (n20 - n02) + 4 * n11 * n11;
  h[2] = a * a + b * b;
  h[3] = s * s + t * t;
  h[4] = a * s * (s * s - 3 * t * t) + b * t * (3 * s * s - t * t);
  h[5] = (n20 - n02) * (s * s - t * t) + 4 * n11 * s * t;
  h[6] = b * s * (s * s - 3 * t * t) - a * t * (3 * s * s - t * t);
}

static double ipow(double x, int k) {
  double r = 1;
  for (int i = 0; i < k; ++i) r *= x;
  return r;
}

/* All features of one ROI. */
/* Edge test: pixel (x, y, z) of ROI `label` in image `base`
 * has a face neighbour (4 in 2D, 6 in 3D) outside the image or under
 * another label. */
static int is_edge(const orc_cfg* c, const int32_t* mask, int64_t base, const int64_t* X, int32_t label) {
  static const int nb[6][3] = {{1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
  const int nnb = c->ndim == 3 ? 6 : 4;
  for (int q = 0; q < nnb; ++q) {
    const int64_t x = X[0] + nb[q][0], y = X[1] + nb[q][1], z = X[2] + nb[q][2];
    if (x < 0 || y < 0 || z < 0 || x >= c->nx || y >= c->ny || z >= c->nz) return 1;
    if (mask[base + (z * c->ny + y) * c->nx + x] != label) return 1;
  }
  return 0;
}

/* ---- run-length and size-zone matrices ----
 * Both matrices count items (runs or zones) by grey level i (1-based GLCM
 * bin) and size s (run length or zone area).  With M items over Np ROI
 * pixels, p = count(i, s) / M, and sums over the items:
 *   [0] small emphasis  sum 1/s^2 / M      [1] large emphasis  sum s^2 / M
 *   [2] grey-level non-uniformity  sum_i n_i^2 / M,  [3] the same / M
 *   [4] size non-uniformity  sum_s n_s^2 / M,        [5] the same / M
 *   [6] percentage M / Np
 *   [7] grey-level variance  sum p (i - mu_i)^2,  [8] size variance  sum p (s - mu_s)^2
 *   [9] entropy -sum p log2 p over the non-empty (i, s) cells
 *   [10] low grey  sum 1/i^2 / M   [11] high grey  sum i^2 / M
 *   [12] small-low  sum 1/(i^2 s^2) / M   [13] small-high  sum i^2/s^2 / M
 *   [14] large-low  sum s^2/i^2 / M       [15] large-high  sum i^2 s^2 / M
 *   [16] grey-level mean mu_i             [17] size mean mu_s
 * n_i = items of level i, n_s = items of size s. */
typedef struct {
  int64_t i, s;
} item_t;

static int cmp_item(const void* a, const void* b) {
  const item_t* x = (const item_t*)a;
  const item_t* y = (const item_t*)b;
  if (x->i != y->i) return x->i < y->i ? -1 : 1;
  if (x->s != y->s) return x->s < y->s ? -1 : 1;
  return 0;
}

static void size_matrix_features(item_t* it, int64_t M, int ng, int64_t smax, int64_t Np, double* o) {
  for (int q = 0; q < 18; ++q) o[q] = 0;
  const double Md = (double)M;
  double* ni = (double*)calloc((size_t)ng + 1, sizeof(double));
  double* ns = (double*)calloc((size_t)smax + 1, sizeof(double));
  double mui = 0, mus = 0;
  for (int64_t k = 0; k < M; ++k) {
    const double i = (double)it[k].i, sz = (double)it[k].s, i2 = i * i, s2 = sz * sz;
    ni[it[k].i] += 1;
    ns[it[k].s] += 1;
    o[0] += 1 / s2;
    o[1] += s2;
    o[10] += 1 / i2;
    o[11] += i2;
    o[12] += 1 / (i2 * s2);
    o[13] += i2 / s2;
    o[14] += s2 / i2;
    o[15] += i2 * s2;
    mui += i;
    mus += sz;
  }
  mui /= Md;
  mus /= Md;
  for (int64_t k = 0; k < M; ++k) {
    o[7] += ((double)it[k].i - mui) * ((double)it[k].i - mui);
    o[8] += ((double)it[k].s - mus) * ((double)it[k].s - mus);
  }
  for (int a = 0; a <= ng; ++a) o[2] += ni[a] * ni[a];
  for (int64_t a = 0; a <= smax; ++a) o[4] += ns[a] * ns[a];
  qsort(it, (size_t)M, sizeof(item_t), cmp_item);
  for (int64_t k = 0; k < M;) {
    int64_t e = k;
    while (e < M && it[e].i == it[k].i && it[e].s == it[k].s) ++e;
    const double pc = (double)(e - k) / Md;
    o[9] -= pc * log2(pc);
    k = e;
  }
  const int per_m[18] = {1, 1, 1, 0, 1, 0, 0, 1, 1, 0, 1, 1, 1, 1, 1, 1, 0, 0};
  for (int q = 0; q < 18; ++q)
    if (per_m[q]) o[q] /= Md;
  o[3] = o[2] / Md;
  o[5] = o[4] / Md;
  o[6] = Md / (double)Np;
  o[16] = mui;
  o[17] = mus;
  free(ni);
  free(ns);
}

/* GLRLM and GLSZM of one ROI.  lev[] holds the
 * 1-based level of each cell of the ROI's bounding box (W x H x D, x
 * fastest), 0 outside the ROI; Np is the ROI's pixel count.  GLRLM: for
 * each GLCM unit direction v, a run is a maximal chain p, p + v, ... of
 * ROI cells with one level; the 16 features of each direction's matrix are
 * averaged over the directions.  GLSZM: a zone is a maximal set of ROI
 * cells of one level connected through their 8 (2D) / 26 (3D) Chebyshev-1
 * neighbours. */
static void run_zone_features(const orc_cfg* c, const int* lev, int64_t W, int64_t H, int64_t D, int64_t Np,
                              feat_t* f) {
  const int64_t cells = W * H * D;
  int64_t smax = W > H ? W : H;
  if (D > smax) smax = D;
  if (c->families & 1) {
    item_t* it = (item_t*)malloc(sizeof(item_t) * (size_t)Np);
    double acc[18] = {0}, o[18];
    const int nd = n_dirs(c);
    for (int k = 0; k < nd; ++k) {
      int dx, dy, dz;
      unit_dir(c, k, &dx, &dy, &dz);
      int64_t M = 0;
      for (int64_t z = 0; z < D; ++z)
        for (int64_t y = 0; y < H; ++y)
          for (int64_t x = 0; x < W; ++x) {
            const int L = lev[(z * H + y) * W + x];
            if (!L) continue;
            /* a run starts here when the cell before it is not of level L */
            const int64_t px = x - dx, py = y - dy, pz = z - dz;
            if (px >= 0 && py >= 0 && pz >= 0 && px < W && py < H && pz < D && lev[(pz * H + py) * W + px] == L)
              continue;
            int64_t len = 0, qx = x, qy = y, qz = z;
            while (qx >= 0 && qy >= 0 && qz >= 0 && qx < W && qy < H && qz < D && lev[(qz * H + qy) * W + qx] == L) {
              ++len;
              qx += dx;
              qy += dy;
              qz += dz;
            }
            it[M].i = L;
            it[M].s = len;
            ++M;
          }
      size_matrix_features(it, M, c->ng, smax, Np, o);
      for (int q = 0; q < 16; ++q) acc[q] += o[q];
    }
    for (int q = 0; q < 16; ++q) f->glrlm[q] = acc[q] / nd;
    free(it);
  }
  if (c->families & 2) {
    item_t* it = (item_t*)malloc(sizeof(item_t) * (size_t)Np);
    char* seen = (char*)calloc((size_t)cells, 1);
    int64_t* stack = (int64_t*)malloc(sizeof(int64_t) * (size_t)Np);
    int64_t M = 0;
    const int d3 = c->ndim == 3;
    for (int64_t start = 0; start < cells; ++start) {
      if (!lev[start] || seen[start]) continue;
      const int L = lev[start];
      int64_t top = 0, size = 0;
      stack[top++] = start;
      seen[start] = 1;
      while (top > 0) {
        const int64_t q = stack[--top];
        ++size;
        const int64_t x = q % W, y = (q / W) % H, z = q / (W * H);
        for (int ez = -1; ez <= 1; ++ez)
          for (int ey = -1; ey <= 1; ++ey)
            for (int ex = -1; ex <= 1; ++ex) {
              if (!d3 && ez != 0) continue;
              const int64_t nx = x + ex, ny = y + ey, nz = z + ez;
              if (nx < 0 || ny < 0 || nz < 0 || nx >= W || ny >= H || nz >= D) continue;
              const int64_t nb = (nz * H + ny) * W + nx;
              if (seen[nb] || lev[nb] != L) continue;
              seen[nb] = 1;
              stack[top++] = nb;
            }
      }
      it[M].i = L;
      it[M].s = size;
      ++M;
    }
    size_matrix_features(it, M, c->ng, Np, Np, f->glszm);
    free(seen);
    free(stack);
    free(it);
  }
}

static void compute_roi(const orc_cfg* c, const void* img, const int32_t* mask, const roi_t* r, double img_min,
                        double img_max, feat_t* f) {
  const int64_t per = c->nx * c->ny * c->nz;
  const int64_t base = r->b * per;
  const int64_t N = r->n;
  const int d3 = c->ndim == 3;
  memset(f, 0, sizeof *f);
  f->label = r->label;
  f->image = (double)r->b;
  f->area = (double)N;

  double* I = (double*)malloc(sizeof(double) * (size_t)N);
  int64_t(*X)[3] = malloc(sizeof(int64_t[3]) * (size_t)N);
  int64_t lo[3] = {INT64_MAX, INT64_MAX, INT64_MAX}, hi[3] = {INT64_MIN, INT64_MIN, INT64_MIN};
  for (int64_t k = 0; k < N; ++k) {
    int64_t lin = r->lin[k];
    X[k][0] = lin % c->nx;
    X[k][1] = (lin / c->nx) % c->ny;
    X[k][2] = lin / (c->nx * c->ny);
    I[k] = pixel(c, img, base + lin);
    for (int a = 0; a < 3; ++a) {
      if (X[k][a] < lo[a]) lo[a] = X[k][a];
      if (X[k][a] > hi[a]) hi[a] = X[k][a];
    }
  }
  for (int a = 0; a < 3; ++a) {
    f->bbox_min[a] = (double)lo[a];
    f->bbox_ext[a] = (double)(hi[a] - lo[a] + 1);
  }
  /* binary centroid in image coordinates (Table S2 rows 48-49) */
  for (int a = 0; a < 3; ++a) {
    double s = 0;
    for (int64_t k = 0; k < N; ++k) s += (double)X[k][a];
    f->centroid[a] = s / N;
  }

  /* ---- first-order statistics, Table S1 (two-pass) ---- */
  double sum = 0, mn = I[0], mx = I[0], energy = 0;
  for (int64_t k = 0; k < N; ++k) {
    sum += I[k];
    energy += I[k] * I[k];
    if (I[k] < mn) mn = I[k];
    if (I[k] > mx) mx = I[k];
  }
  const double mean = sum / N;
  double m[7] = {0}, absdev = 0;
  for (int64_t k = 0; k < N; ++k) {
    double d = I[k] - mean;
    for (int j = 2; j <= 6; ++j) m[j] += ipow(d, j);
    absdev += fabs(d);
  }
  for (int j = 2; j <= 6; ++j) m[j] /= N;
  f->mean = mean;
  f->min = mn;
  f->max = mx;
  f->range = mx - mn;
  f->var = N > 1 ? m[2] * N / (N - 1) : 0.0;
  f->var_b = m[2];
  f->std = sqrt(f->var);
  f->std_b = sqrt(m[2]);
  if (m[2] > 0) {
    f->skew = m[3] / pow(m[2], 1.5);
    f->kurt = m[4] / (m[2] * m[2]);
    f->exkurt = f->kurt - 3.0;
    f->hskew = m[5] / pow(m[2], 2.5);
    f->hflat = m[6] / (m[2] * m[2] * m[2]);
  } /* else all zero (no spread: the degenerate case) */
  f->energy = energy;
  f->rms = sqrt(energy / N);
  f->se = f->std / sqrt((double)N);
  f->mad = absdev / N;
  f->ii = sum;
  const int nax = d3 ? 3 : 2;
  for (int a = 0; a < nax; ++a) {
    double s = 0;
    for (int64_t k = 0; k < N; ++k) s += (double)X[k][a] * I[k];
    f->wc[a] = sum != 0 ? s / sum : NAN;
  }
  {
    double s = 0;
    for (int a = 0; a < nax; ++a) s += (f->wc[a] - f->centroid[a]) * (f->wc[a] - f->centroid[a]);
    f->md = sqrt(s);
  }
  f->cov = mean != 0 ? f->std / mean : NAN;
  f->covered = img_max != img_min ? (mx - mn) / (img_max - img_min) : NAN;
  f->piu = (mx + mn) != 0 ? 100.0 * (1.0 - (mx - mn) / (mx + mn)) : NAN;

  /* edge intensity statistics (Table S1 rows 3-7, Table S5): a pixel of the
   * ROI is an edge pixel when one of its 4 (2D) / 6 (3D) face neighbours is
   * outside the image or carries another label.  Two-pass
   * mean and unbiased standard deviation over the edge pixels. */
  {
    int64_t ne = 0;
    double es = 0, emn = INFINITY, emx = -INFINITY;
    char* edge = (char*)calloc((size_t)N, 1);
    for (int64_t k = 0; k < N; ++k) {
      edge[k] = (char)is_edge(c, mask, base, X[k], r->label);
      if (!edge[k]) continue;
      ++ne;
      es += I[k];
      if (I[k] < emn) emn = I[k];
      if (I[k] > emx) emx = I[k];
    }
    const double em = es / ne;  /* every finite ROI has an edge pixel */
    double ev = 0;
    for (int64_t k = 0; k < N; ++k)
      if (edge[k]) ev += (I[k] - em) * (I[k] - em);
    free(edge);
    f->edge_ii = es;
    f->edge_max = emx;
    f->edge_min = emn;
    f->edge_mean = em;
    f->edge_std = ne > 1 ? sqrt(ev / (ne - 1)) : 0.0;
  }

  /* order statistics on the sorted values */
  double* v = (double*)malloc(sizeof(double) * (size_t)N);
  memcpy(v, I, sizeof(double) * (size_t)N);
  qsort(v, (size_t)N, sizeof(double), cmp_double);
  f->median = percentile(v, N, 0.50);
  f->p01 = percentile(v, N, 0.01);
  f->p10 = percentile(v, N, 0.10);
  f->p25 = percentile(v, N, 0.25);
  f->p75 = percentile(v, N, 0.75);
  f->p90 = percentile(v, N, 0.90);
  f->p99 = percentile(v, N, 0.99);
  f->iqr = f->p75 - f->p25;
  f->qcod = (f->p75 + f->p25) != 0 ? (f->p75 - f->p25) / (f->p75 + f->p25) : NAN;
  {
    double s = 0;
    int64_t cnt = 0;
    for (int64_t k = 0; k < N; ++k)
      if (v[k] >= f->p10 && v[k] <= f->p90) {
        s += v[k];
        ++cnt;
      }
    f->rmean = s / cnt;
    double t = 0;
    for (int64_t k = 0; k < N; ++k)
      if (v[k] >= f->p10 && v[k] <= f->p90) t += fabs(v[k] - f->rmean);
    f->rmad = t / cnt;
  }
  {
    double s = 0;
    for (int64_t k = 0; k < N; ++k) s += fabs(v[k] - f->median);
    f->medad = s / N;
  }
  {
    /* mode: most frequent raw value, ties -> smallest */
    double best = v[0];
    int64_t bestc = 0, run = 0;
    for (int64_t k = 0; k < N; ++k) {
      run = (k > 0 && v[k] == v[k - 1]) ? run + 1 : 1;
      if (run > bestc) {
        bestc = run;
        best = v[k];
      }
    }
    f->mode = best;
    f->mode_prob = (double)bestc / N;
  }
  {
    /* histogram features (Table S1 rows 9, 35): fixed-bin-number bins with
     * n = hist_bins on the ROI's min/max */
    int64_t* h = (int64_t*)calloc((size_t)c->hist_bins, sizeof(int64_t));
    for (int64_t k = 0; k < N; ++k) h[bin_of(c, I[k], mn, mx, c->hist_bins)]++;
    double ent = 0, uni = 0;
    for (int b = 0; b < c->hist_bins; ++b) {
      if (h[b] == 0) continue;
      double p = (double)h[b] / N;
      ent -= p * log2(p);
      uni += p * p;
    }
    f->entropy = ent;
    f->uniformity = uni;
    free(h);
  }
  free(v);

  /* ---- geometric moments, Table S2 rows 123-135 / Table S5 rows 368, 370 ---
   * ROI-local coordinates with origin at the bounding-box corner and pixel
   * centres at integers; central moments are computed directly
   * about the centroid (two-pass), not by binomial expansion. */
  const int nm = n_moments(c);
  for (int w = 0; w < 2; ++w) {
    for (int k = 0; k < nm; ++k) {
      int p, q, rr;
      moment_exp(c, k, &p, &q, &rr);
      double s = 0;
      for (int64_t i = 0; i < N; ++i) {
        double wt = w == 0 ? I[i] : 1.0;
        s += ipow((double)(X[i][0] - lo[0]), p) * ipow((double)(X[i][1] - lo[1]), q) *
             ipow((double)(X[i][2] - lo[2]), rr) * wt;
      }
      f->M[w][k] = s;
    }
    const double M00 = f->M[w][moment_index(c, 0, 0, 0)];
    double cen[3] = {f->M[w][moment_index(c, 1, 0, 0)] / M00, f->M[w][moment_index(c, 0, 1, 0)] / M00,
                     d3 ? f->M[w][moment_index(c, 0, 0, 1)] / M00 : 0.0};
    for (int k = 0; k < nm; ++k) {
      int p, q, rr;
      moment_exp(c, k, &p, &q, &rr);
      double s = 0;
      for (int64_t i = 0; i < N; ++i) {
        double wt = w == 0 ? I[i] : 1.0;
        s += ipow((double)(X[i][0] - lo[0]) - cen[0], p) * ipow((double)(X[i][1] - lo[1]) - cen[1], q) *
             ipow(d3 ? (double)(X[i][2] - lo[2]) - cen[2] : 0.0, rr) * wt;
      }
      f->MU[w][k] = M00 != 0 ? s : NAN;
    }
    const double mu00 = f->MU[w][moment_index(c, 0, 0, 0)];
    for (int k = 0; k < nm; ++k) {
      int p, q, rr;
      moment_exp(c, k, &p, &q, &rr);
      int o = p + q + rr;
      double gam = d3 ? 1.0 + o / 3.0 : 1.0 + o / 2.0;
      f->ETA[w][k] = (o >= 2 && M00 != 0) ? f->MU[w][k] / pow(mu00, gam) : (o >= 2 ? NAN : 0.0);
      f->NU[w][k] = M00 != 0 ? f->M[w][k] / pow(M00, gam) : NAN;
    }
    if (!d3) {
      hu7(f->ETA[w][moment_index(c, 2, 0, 0)], f->ETA[w][moment_index(c, 0, 2, 0)],
          f->ETA[w][moment_index(c, 1, 1, 0)], f->ETA[w][moment_index(c, 3, 0, 0)],
          f->ETA[w][moment_index(c, 2, 1, 0)], f->ETA[w][moment_index(c, 1, 2, 0)],
          f->ETA[w][moment_index(c, 0, 3, 0)], f->HU[w]);
    }
  }

  /* ---- GLCM, Table S3 rows 140-174; per offset, then the arithmetic mean
   * over the directions of each distance that have at least one pair
   * (readings c5, c8) ---- */
  if (c->ng > 0) {
    double* P = (double*)malloc(sizeof(double) * (size_t)c->ng * c->ng);
    for (int di = 0; di < c->n_dist; ++di) {
      double acc[ORC_NGLCM] = {0};
      int used = 0;
      for (int o = 0; o < n_dirs(c); ++o) {
        roi_glcm(c, img, mask, r, mn, mx, o, c->dist[di], P);
        glcm_features(c->ng, P, f->glcm_off[di][o]);
        if (!isnan(f->glcm_off[di][o][0])) {
          ++used;
          for (int g = 0; g < ORC_NGLCM; ++g) acc[g] += f->glcm_off[di][o][g];
        }
      }
      for (int g = 0; g < ORC_NGLCM; ++g) f->glcm_mean[di][g] = used ? acc[g] / used : NAN;
    }
    free(P);
  }

  /* ---- NGTDM, Table S3 rows 246-250: for every ROI pixel
   * with grey level L (1-based GLCM bin) and at least one neighbour in the
   * ROI among its 8 (2D) / 26 (3D) Chebyshev-1 neighbours, the mean level
   * A of those neighbours; n_L counts such pixels and s_L sums |L - A|.
   * With p_L = n_L / N (N = number of such pixels) and the sums over the
   * levels with p_L > 0: coarseness 1 / sum p s; contrast
   * [sum_i sum_j p_i p_j (i-j)^2 / (G (G-1))] [sum s / N] (G levels present);
   * busyness sum p s / sum_i sum_j |i p_i - j p_j|; complexity
   * (1/N) sum_i sum_j |i - j| (p_i s_i + p_j s_j) / (p_i + p_j); strength
   * sum_i sum_j (p_i + p_j) (i-j)^2 / sum s. ---- */
  if (c->ng > 0) {
    double* nL = (double*)calloc((size_t)c->ng, sizeof(double));
    double* sL = (double*)calloc((size_t)c->ng, sizeof(double));
    for (int64_t k = 0; k < N; ++k) {
      const int L = bin_of(c, I[k], mn, mx, c->ng) + 1;
      double sum = 0;
      int cnt = 0;
      for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            if (dx == 0 && dy == 0 && dz == 0) continue;
            if (!d3 && dz != 0) continue;
            const int64_t x = X[k][0] + dx, y = X[k][1] + dy, z = X[k][2] + dz;
            if (x < 0 || y < 0 || z < 0 || x >= c->nx || y >= c->ny || z >= c->nz) continue;
            const int64_t nl = (z * c->ny + y) * c->nx + x;
            if (mask[base + nl] != r->label) continue;
            sum += bin_of(c, pixel(c, img, base + nl), mn, mx, c->ng) + 1;
            ++cnt;
          }
      if (cnt == 0) continue;
      nL[L - 1] += 1;
      sL[L - 1] += fabs(L - sum / cnt);
    }
    double Nv = 0;
    for (int i = 0; i < c->ng; ++i) Nv += nL[i];
    for (int q = 0; q < 5; ++q) f->ngtdm[q] = NAN;
    if (Nv > 0) {
      double ps = 0, ssum = 0, G = 0;
      for (int i = 0; i < c->ng; ++i) {
        if (nL[i] == 0) continue;
        ps += nL[i] / Nv * sL[i];
        ssum += sL[i];
        G += 1;
      }
      double pair_c = 0, busy_den = 0, cplx = 0, str_num = 0;
      for (int i = 0; i < c->ng; ++i) {
        if (nL[i] == 0) continue;
        const double pi = nL[i] / Nv, li = i + 1;
        for (int j = 0; j < c->ng; ++j) {
          if (nL[j] == 0) continue;
          const double pj = nL[j] / Nv, lj = j + 1;
          pair_c += pi * pj * (li - lj) * (li - lj);
          busy_den += fabs(li * pi - lj * pj);
          cplx += fabs(li - lj) * (pi * sL[i] + pj * sL[j]) / (pi + pj);
          str_num += (pi + pj) * (li - lj) * (li - lj);
        }
      }
      f->ngtdm[0] = ps > 0 ? 1.0 / ps : NAN;
      f->ngtdm[1] = G > 1 ? pair_c / (G * (G - 1)) * (ssum / Nv) : 0.0;
      f->ngtdm[2] = busy_den > 0 ? ps / busy_den : 0.0;
      f->ngtdm[3] = cplx / Nv;
      f->ngtdm[4] = ssum > 0 ? str_num / ssum : 0.0;
    }
    free(nL);
    free(sL);
  }

  /* ---- GLDM, Table S3 rows 251-264: the dependence of a
   * pixel of grey level i (1-based GLCM bin) is j = 1 + the number of its 8
   * (2D) / 26 (3D) Chebyshev-1 neighbours in the ROI with the same level;
   * P(i, j) counts the pixels, N = sum P = the ROI's pixel count, p = P / N.
   * SDE sum P / j^2 / N, LDE sum P j^2 / N, GLN sum_i (sum_j P)^2 / N, DN
   * sum_j (sum_i P)^2 / N, DNN DN / N, GLV sum p (i - mu_i)^2, DV
   * sum p (j - mu_j)^2, DE -sum p log2 p (cells with P > 0), LGLE
   * sum P / i^2 / N, HGLE sum P i^2 / N, SDLGLE sum P / (i^2 j^2) / N,
   * SDHGLE sum P i^2 / j^2 / N, LDLGLE sum P j^2 / i^2 / N, LDHGLE
   * sum P i^2 j^2 / N. ---- */
  if (c->ng > 0) {
    const int nj = d3 ? 27 : 9;
    double* P = (double*)calloc((size_t)c->ng * nj, sizeof(double));
    for (int64_t k = 0; k < N; ++k) {
      const int L = bin_of(c, I[k], mn, mx, c->ng);
      int dep = 1;
      for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            if (dx == 0 && dy == 0 && dz == 0) continue;
            if (!d3 && dz != 0) continue;
            const int64_t x = X[k][0] + dx, y = X[k][1] + dy, z = X[k][2] + dz;
            if (x < 0 || y < 0 || z < 0 || x >= c->nx || y >= c->ny || z >= c->nz) continue;
            const int64_t nl = (z * c->ny + y) * c->nx + x;
            if (mask[base + nl] != r->label) continue;
            if (bin_of(c, pixel(c, img, base + nl), mn, mx, c->ng) == L) ++dep;
          }
      P[L * nj + (dep - 1)] += 1;
    }
    const double Nz = (double)N;
    double g[14] = {0};
    double mui = 0, muj = 0;
    for (int i = 0; i < c->ng; ++i)
      for (int j = 0; j < nj; ++j) {
        const double pij = P[i * nj + j] / Nz;
        mui += pij * (i + 1);
        muj += pij * (j + 1);
      }
    for (int i = 0; i < c->ng; ++i) {
      double rowsum = 0;
      const double ii = i + 1.0, i2 = ii * ii;
      for (int j = 0; j < nj; ++j) {
        const double v = P[i * nj + j];
        rowsum += v;
        if (v == 0) continue;
        const double jj = j + 1.0, j2 = jj * jj, pij = v / Nz;
        g[0] += v / j2;
        g[1] += v * j2;
        g[5] += pij * (ii - mui) * (ii - mui);
        g[6] += pij * (jj - muj) * (jj - muj);
        g[7] -= pij * log2(pij);
        g[8] += v / i2;
        g[9] += v * i2;
        g[10] += v / (i2 * j2);
        g[11] += v * i2 / j2;
        g[12] += v * j2 / i2;
        g[13] += v * i2 * j2;
      }
      g[2] += rowsum * rowsum;
    }
    for (int j = 0; j < nj; ++j) {
      double colsum = 0;
      for (int i = 0; i < c->ng; ++i) colsum += P[i * nj + j];
      g[3] += colsum * colsum;
    }
    const int per_n[14] = {1, 1, 1, 1, 0, 0, 0, 0, 1, 1, 1, 1, 1, 1};
    for (int q = 0; q < 14; ++q) f->gldm[q] = per_n[q] ? g[q] / Nz : g[q];
    f->gldm[4] = g[3] / (Nz * Nz);
    free(P);
  }

  /* ---- GLRLM / GLSZM, when asked for ---- */
  if (c->ng > 0 && c->families) {
    const int64_t W = hi[0] - lo[0] + 1, H = hi[1] - lo[1] + 1, D = hi[2] - lo[2] + 1;
    int* lev = (int*)calloc((size_t)(W * H * D), sizeof(int));
    for (int64_t k = 0; k < N; ++k)
      lev[((X[k][2] - lo[2]) * H + (X[k][1] - lo[1])) * W + (X[k][0] - lo[0])] = bin_of(c, I[k], mn, mx, c->ng) + 1;
    run_zone_features(c, lev, W, H, D, N, f);
    free(lev);
  }
  free(I);
  free(X);
}

/* ======================================================================== */
/* exported API (used through ctypes by the tests and the benchmark) */

int orc_n_features(const orc_cfg* c) {
  feat_t* f = (feat_t*)calloc(1, sizeof(feat_t));
  emitter e = {NULL, NULL, 0};
  emit_all(c, f, &e);
  free(f);
  return e.k;
}

/* names: caller buffer of n_features * 48 chars */
int orc_feature_names(const orc_cfg* c, char* names) {
  feat_t* f = (feat_t*)calloc(1, sizeof(feat_t));
  emitter e = {NULL, (char(*)[ORC_NAME])names, 0};
  emit_all(c, f, &e);
  free(f);
  return e.k;
}

static void image_range(const orc_cfg* c, const void* img, int64_t b, double* mn, double* mx) {
  const int64_t per = c->nx * c->ny * c->nz;
  *mn = INFINITY;
  *mx = -INFINITY;
  for (int64_t i = 0; i < per; ++i) {
    double v = pixel(c, img, b * per + i);
    if (v < *mn) *mn = v;
    if (v > *mx) *mx = v;
  }
}

/* Count ROIs (distinct (image,label) pairs with label > 0); -1 on a
 * negative label. */
int64_t orc_count_rois(const orc_cfg* c, const int32_t* mask) {
  roi_t* r = NULL;
  int64_t n = separate(c, mask, NULL, 0, &r);
  if (n > 0) free_rois(r, n);
  return n;
}

/* Extract every ROI (subset == NULL) or only the listed (image << 32 | label)
 * keys, in ascending key order.  out: [n_roi x n_features] FP64 row-major.
 * Returns the number of rows written, or a negative error. */
int64_t orc_extract(const orc_cfg* c, const void* img, const int32_t* mask, const int64_t* subset, int64_t n_subset,
                    int64_t cap, double* out, int threads) {
  int64_t* sk = NULL;
  if (subset) {
    sk = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_subset > 0 ? n_subset : 1));
    memcpy(sk, subset, sizeof(int64_t) * (size_t)n_subset);
    qsort(sk, (size_t)n_subset, sizeof(int64_t), cmp_i64);
  }
  roi_t* r = NULL;
  int64_t n = separate(c, mask, sk, n_subset, &r);
  free(sk);
  if (n < 0) return n;
  if (n > cap) {
    free_rois(r, n);
    return -3;
  }
  const int nf = orc_n_features(c);
  double* imn = (double*)malloc(sizeof(double) * (size_t)c->batch);
  double* imx = (double*)malloc(sizeof(double) * (size_t)c->batch);
  for (int b = 0; b < c->batch; ++b) image_range(c, img, b, &imn[b], &imx[b]);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads > 0 ? threads : 1)
#endif
  for (int64_t i = 0; i < n; ++i) {
    feat_t* f = (feat_t*)malloc(sizeof(feat_t));
    compute_roi(c, img, mask, &r[i], imn[r[i].b], imx[r[i].b], f);
    emitter e = {out + i * nf, NULL, 0};
    emit_all(c, f, &e);
    free(f);
  }
  (void)threads;
  free(imn);
  free(imx);
  free_rois(r, n);
  return n;
}

/* Bin index (fixed bin number rule, n bins) of every pixel of the ROI with the given
 * key, in ascending linear-index order.  Returns the pixel count. */
int64_t orc_roi_bins(const orc_cfg* c, const void* img, const int32_t* mask, int64_t key, int nbins, int32_t* out,
                     int64_t cap) {
  roi_t* r = NULL;
  int64_t n = separate(c, mask, &key, 1, &r);
  if (n != 1) {
    if (n > 0) free_rois(r, n);
    return -1;
  }
  const int64_t per = c->nx * c->ny * c->nz;
  double mn = INFINITY, mx = -INFINITY;
  for (int64_t k = 0; k < r->n; ++k) {
    double v = pixel(c, img, r->b * per + r->lin[k]);
    if (v < mn) mn = v;
    if (v > mx) mx = v;
  }
  int64_t m = r->n;
  for (int64_t k = 0; k < m && k < cap; ++k) out[k] = bin_of(c, pixel(c, img, r->b * per + r->lin[k]), mn, mx, nbins);
  free_rois(r, 1);
  return m;
}

/* Dense symmetric GLCM counts (ng x ng, FP64) of one ROI for direction
 * index dir at distance d. */
int orc_roi_glcm(const orc_cfg* c, const void* img, const int32_t* mask, int64_t key, int dir, int d, double* out) {
  roi_t* r = NULL;
  int64_t n = separate(c, mask, &key, 1, &r);
  if (n != 1) {
    if (n > 0) free_rois(r, n);
    return -1;
  }
  const int64_t per = c->nx * c->ny * c->nz;
  double mn = INFINITY, mx = -INFINITY;
  for (int64_t k = 0; k < r->n; ++k) {
    double v = pixel(c, img, r->b * per + r->lin[k]);
    if (v < mn) mn = v;
    if (v > mx) mx = v;
  }
  roi_glcm(c, img, mask, r, mn, mx, dir, d, out);
  free_rois(r, 1);
  return 0;
}

/* GLCM features of a caller-supplied dense ng x ng count matrix. */
void orc_glcm_features(int ng, const double* P, double* out) { glcm_features(ng, P, out); }

void orc_unit_dir(const orc_cfg* c, int k, int* d) { unit_dir(c, k, &d[0], &d[1], &d[2]); }

/* ======================================================================== */
/* Analytic gradient of the smooth features with respect to pixel
 * intensities (the differentiable layer use the paper motivates in its
 * introduction: features feeding AI/ML pipelines).  Each derivative below is
 * obtained by hand with the chain rule through N, the mean, the centred sums
 * m_j, the centroid and the normalisations; non-smooth features (min, max,
 * order statistics, mode, histogram, GLCM, binary moments, geometry) have a
 * zero gradient.
 *
 *   d mean / dI_k        = 1/N
 *   d m_j / dI_k         = (j/N) (d_k^(j-1) - m_(j-1)),   d_k = I_k - mean,
 *                          m_0 = 1, m_1 = 0
 *   d MAD / dI_k         = (1/N) (sgn d_k - (1/N) sum_i sgn d_i)
 *   d WC_a / dI_k        = (x_k,a - WC_a) / sum I
 *   d M_pq / dI_k        = x_k^p y_k^q                    (ROI-local coords)
 *   d mu_pq / dI_k       = u^p v^q - p mu_(p-1,q) u / M00 - q mu_(p,q-1) v / M00
 *                          (u = x_k - xbar, v = y_k - ybar; 3D likewise)
 *   d eta / dI_k         = d mu / mu00^g - g eta / mu00     (d mu00 / dI = 1)
 *   d nu  / dI_k         = d M / M00^g  - g nu / M00
 *   Hu: partial derivatives of the seven polynomials in eta (see hu7_grad).
 */
static void hu7_grad(double n20, double n02, double n11, double n30, double n21, double n12, double n03,
                     double dh[7][7] /* [invariant][n20,n02,n11,n30,n21,n12,n03] */) {
  double a = n30 - 3 * n12, b = 3 * n21 - n03, s = n30 + n12, t = n21 + n03;
  memset(dh, 0, sizeof(double) * 49);
  /* helpers: derivative w.r.t. (a, b, s, t, n20, n02, n11) then mapped */
  double g[7][7]; /* [inv][a,b,s,t,n20,n02,n11] */
  memset(g, 0, sizeof g);
  g[0][4] = 1;
  g[0][5] = 1;
  g[1][4] = 2 * (n20 - n02);
  g[1][5] = -2 * (n20 - n02);
  g[1][6] = 8 * n11;
  g[2][0] = 2 * a;
  g[2][1] = 2 * b;
  g[3][2] = 2 * s;
  g[3][3] = 2 * t;
  g[4][0] = s * (s * s - 3 * t * t);
  g[4][1] = t * (3 * s * s - t * t);
  g[4][2] = a * (3 * s * s - 3 * t * t) + 6 * b * s * t;
  g[4][3] = -6 * a * s * t + b * (3 * s * s - 3 * t * t);
  g[5][4] = s * s - t * t;
  g[5][5] = -(s * s - t * t);
  g[5][6] = 4 * s * t;
  g[5][2] = 2 * s * (n20 - n02) + 4 * n11 * t;
  g[5][3] = -2 * t * (n20 - n02) + 4 * n11 * s;
  g[6][1] = s * s * s - 3 * s * t * t;
  g[6][0] = -(3 * s * s * t - t * t * t);
  g[6][2] = b * (3 * s * s - 3 * t * t) - 6 * a * s * t;
  g[6][3] = -6 * b * s * t - a * (3 * s * s - 3 * t * t);
  for (int h = 0; h < 7; ++h) {
    /* a = n30 - 3 n12, b = 3 n21 - n03, s = n30 + n12, t = n21 + n03 */
    dh[h][0] = g[h][4];
    dh[h][1] = g[h][5];
    dh[h][2] = g[h][6];
    dh[h][3] = g[h][0] + g[h][2];
    dh[h][4] = 3 * g[h][1] + g[h][3];
    dh[h][5] = -3 * g[h][0] + g[h][2];
    dh[h][6] = -g[h][1] + g[h][3];
  }
}

static int find_name(char (*names)[ORC_NAME], int nf, const char* s) {
  for (int i = 0; i < nf; ++i)
    if (strcmp(names[i], s) == 0) return i;
  return -1;
}

/* gtab: [n_roi x n_features] upstream gradient rows in the order of
 * orc_extract (ascending (image, label) key).  grad: image-shaped FP64
 * output (zero outside ROIs).  Returns the ROI count or a negative error. */
/* number of edge pixels of ROI R (face neighbour outside the image or the ROI) */
static int64_t edge_count(const orc_cfg* c, const int32_t* mask, const roi_t* R, int64_t per) {
  int64_t ne = 0;
  for (int64_t k = 0; k < R->n; ++k) {
    const int64_t lin = R->lin[k];
    const int64_t xi[3] = {lin % c->nx, (lin / c->nx) % c->ny, lin / (c->nx * c->ny)};
    ne += is_edge(c, mask, R->b * per, xi, R->label);
  }
  return ne;
}

int64_t orc_grad(const orc_cfg* c, const void* img, const int32_t* mask, const double* gtab, double* grad) {
  roi_t* r = NULL;
  int64_t n = separate(c, mask, NULL, 0, &r);
  if (n < 0) return n;
  const int nf = orc_n_features(c);
  char(*names)[ORC_NAME] = malloc(sizeof(char[ORC_NAME]) * (size_t)nf);
  orc_feature_names(c, (char*)names);
  const int64_t per = c->nx * c->ny * c->nz;
  const int d3 = c->ndim == 3;
  const int nax = d3 ? 3 : 2;
  const int nm = n_moments(c);
  memset(grad, 0, sizeof(double) * (size_t)(per * c->batch));
  const char* ax[3] = {"X", "Y", "Z"};
  for (int64_t ri = 0; ri < n; ++ri) {
    const roi_t* R = &r[ri];
    const double* g = gtab + ri * nf;
#define G(name) (find_name(names, nf, name) >= 0 ? g[find_name(names, nf, name)] : 0.0)
    feat_t* f = (feat_t*)malloc(sizeof(feat_t));
    compute_roi(c, img, mask, R, 0.0, 1.0, f);
    const int64_t N = R->n;
    const double mean = f->mean;
    double m[7] = {1, 0, 0, 0, 0, 0, 0};
    double sgn = 0;
    int64_t lo[3] = {(int64_t)f->bbox_min[0], (int64_t)f->bbox_min[1], (int64_t)f->bbox_min[2]};
    for (int64_t k = 0; k < N; ++k) {
      double d = pixel(c, img, R->b * per + R->lin[k]) - mean;
      for (int j = 2; j <= 6; ++j) m[j] += ipow(d, j) / N;
      sgn += d > 0 ? 1 : (d < 0 ? -1 : 0);
    }
    const double m2 = m[2];
    const double gmean = G("MEAN"), gii = G("INTEGRATED_INTENSITY"), gvar = G("VARIANCE"),
                 gvarb = G("VARIANCE_BIASED"), gstd = G("STDDEV"), gstdb = G("STDDEV_BIASED"),
                 gskew = G("SKEWNESS"), gkurt = G("KURTOSIS") + G("EXCESS_KURTOSIS"), ghs = G("HYPERSKEWNESS"),
                 ghf = G("HYPERFLATNESS"), gen = G("ENERGY"), grms = G("ROOT_MEAN_SQUARED"),
                 gse = G("STANDARD_ERROR"), gmad = G("MEAN_ABSOLUTE_DEVIATION"), gcov = G("COV"),
                 gmd = G("MASS_DISPLACEMENT");
    /* edge statistics over the fixed edge set E: d II_E = 1,
     * d mean_E = 1/n_E, d std_E = (I - mean_E) / ((n_E - 1) std_E) on E */
    const double geii = G("EDGE_INTEGRATED_INTENSITY"), gemean = G("EDGE_MEAN_INTENSITY"),
                 gestd = G("EDGE_STDDEV_INTENSITY");
    const int64_t ne_e = (geii != 0 || gemean != 0 || gestd != 0) ? edge_count(c, mask, R, per) : 0;
    double gwc[3];
    for (int a = 0; a < 3; ++a) {
      char s[48];
      snprintf(s, sizeof s, "WEIGHTED_CENTROID_%s", ax[a]);
      gwc[a] = a < nax ? G(s) : 0.0;
    }
    /* intensity moment gradients: look up names */
    double gM[20], gMU[20], gETA[20], gNU[20], gHU[7];
    for (int k = 0; k < nm; ++k) {
      int p, q, rr;
      moment_exp(c, k, &p, &q, &rr);
      char s[48], e[16];
      if (d3) snprintf(e, sizeof e, "%d%d%d", p, q, rr);
      else snprintf(e, sizeof e, "%d%d", p, q);
      snprintf(s, sizeof s, "INT_M%s", e);
      gM[k] = G(s);
      snprintf(s, sizeof s, "INT_MU%s", e);
      gMU[k] = G(s);
      snprintf(s, sizeof s, "INT_ETA%s", e);
      gETA[k] = G(s);
      snprintf(s, sizeof s, "INT_NU%s", e);
      gNU[k] = d3 ? 0.0 : G(s);
    }
    for (int h = 0; h < 7; ++h) {
      char s[48];
      snprintf(s, sizeof s, "INT_HU%d", h + 1);
      gHU[h] = d3 ? 0.0 : G(s);
    }
#undef G
    /* fold Hu into eta */
    if (!d3) {
      double dh[7][7];
      const int i20 = moment_index(c, 2, 0, 0), i02 = moment_index(c, 0, 2, 0), i11 = moment_index(c, 1, 1, 0),
                i30 = moment_index(c, 3, 0, 0), i21 = moment_index(c, 2, 1, 0), i12 = moment_index(c, 1, 2, 0),
                i03 = moment_index(c, 0, 3, 0);
      hu7_grad(f->ETA[0][i20], f->ETA[0][i02], f->ETA[0][i11], f->ETA[0][i30], f->ETA[0][i21], f->ETA[0][i12],
               f->ETA[0][i03], dh);
      const int idx[7] = {i20, i02, i11, i30, i21, i12, i03};
      for (int h = 0; h < 7; ++h)
        for (int e = 0; e < 7; ++e) gETA[idx[e]] += gHU[h] * dh[h][e];
    }
    const double M00 = f->M[0][moment_index(c, 0, 0, 0)];
    const double cen[3] = {f->M[0][moment_index(c, 1, 0, 0)] / M00, f->M[0][moment_index(c, 0, 1, 0)] / M00,
                           d3 ? f->M[0][moment_index(c, 0, 0, 1)] / M00 : 0.0};
    for (int64_t k = 0; k < N; ++k) {
      const int64_t lin = R->lin[k];
      const double Ik = pixel(c, img, R->b * per + lin);
      const double d = Ik - mean;
      const int64_t xi[3] = {lin % c->nx, (lin / c->nx) % c->ny, lin / (c->nx * c->ny)};
      double dm[7] = {0};
      for (int j = 2; j <= 6; ++j) dm[j] = (double)j / N * (ipow(d, j - 1) - m[j - 1]);
      double acc = gmean / N + gii + gen * 2 * Ik;
      if (N > 1) acc += gvar * dm[2] * N / (N - 1);
      acc += gvarb * dm[2];
      double dstd = (f->std > 0 && N > 1) ? dm[2] * N / (N - 1) / (2 * f->std) : 0.0;
      acc += gstd * dstd + gse * dstd / sqrt((double)N);
      if (m2 > 0) {
        acc += gstdb * dm[2] / (2 * sqrt(m2));
        acc += gskew * (dm[3] * pow(m2, -1.5) - 1.5 * m[3] * pow(m2, -2.5) * dm[2]);
        acc += gkurt * (dm[4] * pow(m2, -2.0) - 2.0 * m[4] * pow(m2, -3.0) * dm[2]);
        acc += ghs * (dm[5] * pow(m2, -2.5) - 2.5 * m[5] * pow(m2, -3.5) * dm[2]);
        acc += ghf * (dm[6] * pow(m2, -3.0) - 3.0 * m[6] * pow(m2, -4.0) * dm[2]);
      }
      if (f->rms > 0) acc += grms * Ik / (N * f->rms);
      acc += gmad * ((d > 0 ? 1.0 : (d < 0 ? -1.0 : 0.0)) - sgn / N) / N;
      if (mean != 0) acc += gcov * (dstd * mean - f->std / N) / (mean * mean);
      double dwc[3] = {0, 0, 0};
      for (int a = 0; a < nax; ++a) {
        dwc[a] = ((double)xi[a] - f->wc[a]) / f->ii;
        acc += gwc[a] * dwc[a];
      }
      if (f->md > 0) {
        double s = 0;
        for (int a = 0; a < nax; ++a) s += (f->wc[a] - f->centroid[a]) * dwc[a];
        acc += gmd * s / f->md;
      }
      /* moments */
      const double u[3] = {(double)(xi[0] - lo[0]) - cen[0], (double)(xi[1] - lo[1]) - cen[1],
                           d3 ? (double)(xi[2] - lo[2]) - cen[2] : 0.0};
      const double xl[3] = {(double)(xi[0] - lo[0]), (double)(xi[1] - lo[1]), (double)(xi[2] - lo[2])};
      const double mu00 = f->MU[0][moment_index(c, 0, 0, 0)];
      double dmu00 = 1.0;
      for (int kk = 0; kk < nm; ++kk) {
        int p, q, rr;
        moment_exp(c, kk, &p, &q, &rr);
        int o = p + q + rr;
        double gam = d3 ? 1.0 + o / 3.0 : 1.0 + o / 2.0;
        double dM = ipow(xl[0], p) * ipow(xl[1], q) * ipow(xl[2], rr);
        double dMU = ipow(u[0], p) * ipow(u[1], q) * ipow(u[2], rr);
        if (p > 0) dMU -= p * f->MU[0][moment_index(c, p - 1, q, rr)] * u[0] / M00;
        if (q > 0) dMU -= q * f->MU[0][moment_index(c, p, q - 1, rr)] * u[1] / M00;
        if (rr > 0) dMU -= rr * f->MU[0][moment_index(c, p, q, rr - 1)] * u[2] / M00;
        acc += gM[kk] * dM + gMU[kk] * dMU;
        if (o >= 2) acc += gETA[kk] * (dMU / pow(mu00, gam) - gam * f->ETA[0][kk] * dmu00 / mu00);
        if (!d3) acc += gNU[kk] * (dM / pow(M00, gam) - gam * f->NU[0][kk] / M00);
      }
      if (ne_e > 0 && is_edge(c, mask, R->b * per, xi, R->label)) {
        acc += geii + gemean / ne_e;
        if (f->edge_std > 0) acc += gestd * (Ik - f->edge_mean) / ((ne_e - 1) * f->edge_std);
      }
      grad[R->b * per + lin] = acc;
    }
    free(f);
  }
  free(names);
  free_rois(r, n);
  return n;
}
