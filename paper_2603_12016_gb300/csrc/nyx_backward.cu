// nyx_backward.cu -- gradient of the smooth intensity features with respect
// to the pixel intensities (vector-Jacobian product).
//
// Not a step of the paper's own pipeline: it makes the per-ROI features
// usable as a differentiable layer for the AI/ML use the paper motivates.
//
// For every smooth feature F of an ROI, dF/dI_k is
//   - a polynomial of degree <= 5 in d_k = I_k - mean plus a multiple of
//     sgn(d_k) (first-order statistics, through N, the mean and the centred
//     moments m_j = sum (I - mean)^j / N), and
//   - a polynomial of total degree <= 3 in the offsets (u, v, w) of the pixel
//     from the ROI's intensity centroid (weighted centroids, mass
//     displacement, raw / central / normalised moments, Hu invariants).
// So the VJP sum_F g_F dF/dI_k collapses, per ROI, to 6 + 1 + 20 numbers.
// k_bwd_coef computes them in FP64 (one thread per ROI, no division inside
// its loops); k_bwd_pixel then streams image and mask once and writes dL/dI
// (HBM-bound).
//
//   d mean / dI_k  = 1/N
//   d m_j / dI_k   = (j/N) (d_k^(j-1) - m_(j-1)),  m_0 = 1, m_1 = 0
//   d MAD / dI_k   = (1/N) (sgn d_k - (1/N) sum_i sgn d_i)
//   d WC_a / dI_k  = u_a / sum I
//   d M_pq / dI_k  = x_k^p y_k^q  (ROI-local coordinates)
//   d mu_pq / dI_k = u^p v^q - p mu_(p-1)q u / M00 - q mu_p(q-1) v / M00
//   d eta / dI_k   = d mu / mu00^g - g eta / mu00
//   d nu  / dI_k   = d M / M00^g  - g nu / M00
#include "nyx_internal.cuh"

namespace nyx {

namespace {

constexpr int CW = 40;  // floats per ROI of coefficients
constexpr int EC0 = 37; // edge-statistics coefficients e0, e1, mean_E (after 17 + 20 moment ones)

__device__ inline double gget(const KParams& p, const double* g, int q) {
  const int c = __ldg(p.col_map + q);
  return c >= 0 ? g[c] : 0.0;
}

template <int NDIM>
__device__ constexpr int bidx(int p, int q, int r) {
  if (NDIM == 2) return (p == 0 ? 0 : p == 1 ? 4 : p == 2 ? 7 : 9) + q;
  int base = p == 0 ? 0 : p == 1 ? 10 : p == 2 ? 16 : 19;
  for (int qq = 0; qq < q; ++qq) base += 4 - p - qq;
  return base + r;
}

__device__ inline double dpow(double x, int k) {
  double r = 1;
  for (int i = 0; i < k; ++i) r *= x;
  return r;
}

// binomial coefficient C(n, k) for n <= 3 (the loops below are unrolled, so
// the lookup folds to a constant; no FP64 division)
__device__ inline double choose(int n, int k) {
  constexpr double t[4][4] = {{1, 0, 0, 0}, {1, 1, 0, 0}, {1, 2, 1, 0}, {1, 3, 3, 1}};
  return t[n][k];
}

// m00^(1 + o/2) (2D) or m00^(1 + o/3) (3D) for o = 0..3, from one square or
// cube root (no pow on the FP64 pipe)
template <int NDIM>
__device__ inline void gnorm_table(double m00, double t[4]) {
  const double r = NDIM == 2 ? sqrt(m00) : cbrt(m00);
  t[0] = m00;
  for (int o = 1; o < 4; ++o) t[o] = t[o - 1] * r;
}

// partial derivatives of Hu's invariants with respect to
// (eta20, eta02, eta11, eta30, eta21, eta12, eta03)
__device__ void hu_partials(const double e[7], double dh[7][7]) {
  const double n20 = e[0], n02 = e[1], n11 = e[2], n30 = e[3], n21 = e[4], n12 = e[5], n03 = e[6];
  const double a = n30 - 3 * n12, b = 3 * n21 - n03, s = n30 + n12, t = n21 + n03;
  // derivatives with respect to the auxiliaries (a, b, s, t) and (n20, n02, n11)
  double da[7] = {0}, db[7] = {0}, ds[7] = {0}, dt[7] = {0}, d20[7] = {0}, d02[7] = {0}, d11[7] = {0};
  d20[0] = 1;
  d02[0] = 1;
  d20[1] = 2 * (n20 - n02);
  d02[1] = -2 * (n20 - n02);
  d11[1] = 8 * n11;
  da[2] = 2 * a;
  db[2] = 2 * b;
  ds[3] = 2 * s;
  dt[3] = 2 * t;
  da[4] = s * (s * s - 3 * t * t);
  db[4] = t * (3 * s * s - t * t);
  ds[4] = a * (3 * s * s - 3 * t * t) + 6 * b * s * t;
  dt[4] = b * (3 * s * s - 3 * t * t) - 6 * a * s * t;
  d20[5] = s * s - t * t;
  d02[5] = -(s * s - t * t);
  d11[5] = 4 * s * t;
  ds[5] = 2 * s * (n20 - n02) + 4 * n11 * t;
  dt[5] = -2 * t * (n20 - n02) + 4 * n11 * s;
  db[6] = s * (s * s - 3 * t * t);
  da[6] = -t * (3 * s * s - t * t);
  ds[6] = b * (3 * s * s - 3 * t * t) - 6 * a * s * t;
  dt[6] = -6 * b * s * t - a * (3 * s * s - 3 * t * t);
  for (int h = 0; h < 7; ++h) {
    dh[h][0] = d20[h];
    dh[h][1] = d02[h];
    dh[h][2] = d11[h];
    dh[h][3] = da[h] + ds[h];          // eta30
    dh[h][4] = 3 * db[h] + dt[h];      // eta21
    dh[h][5] = -3 * da[h] + ds[h];     // eta12
    dh[h][6] = -db[h] + dt[h];         // eta03
  }
}

template <int NDIM>
__global__ void k_bwd_coef(KParams p, const double* gtab, float* coef) {
  constexpr int NM = NDIM == 3 ? 20 : 10;
  const unsigned nroi = *p.n_roi;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < nroi; i += gridDim.x * blockDim.x) {
    float* cf = coef + (size_t)i * CW;
    if ((int64_t)i >= p.cap_roi) {
      for (int k = 0; k < CW; ++k) cf[k] = 0.f;
      continue;
    }
    const double* sv = p.saved + (size_t)i * SV_WORDS;
    const double* g = gtab + (size_t)i * p.n_col;
    const double N = sv[SV_N], mean = sv[SV_MEAN], sumI = sv[SV_SUMI];
    const double m2 = sv[SV_M2], m3 = sv[SV_M3], m4 = sv[SV_M4], m5 = sv[SV_M5], m6 = sv[SV_M6];
    double m[7] = {1, 0, m2, m3, m4, m5, m6};
    // ---- intensity polynomial: a[j] multiplies d^j, asg multiplies sgn(d)
    double a[6] = {0, 0, 0, 0, 0, 0}, asg = 0, c[7] = {0, 0, 0, 0, 0, 0, 0};
    const double iN = 1.0 / N;
    const double var = N > 1 ? m2 * N / (N - 1) : 0.0, sd = sqrt(var);
    const double rms = sqrt(sv[SV_ENERGY] * iN);
    a[0] += gget(p, g, Q_STATS + S_MEAN) * iN + gget(p, g, Q_STATS + S_II);
    {
      const double ge = gget(p, g, Q_STATS + S_ENERGY);  // 2 I = 2 (d + mean)
      a[1] += 2 * ge;
      a[0] += 2 * ge * mean;
      if (rms > 0) {
        const double gr = gget(p, g, Q_STATS + S_RMS) * iN / rms;  // I / (N rms)
        a[1] += gr;
        a[0] += gr * mean;
      }
    }
    if (N > 1) c[2] += gget(p, g, Q_STATS + S_VAR) * N / (N - 1);
    c[2] += gget(p, g, Q_STATS + S_VAR_B);
    if (sd > 0 && N > 1) {
      const double dstd = N / (N - 1) / (2 * sd);
      c[2] += gget(p, g, Q_STATS + S_STD) * dstd + gget(p, g, Q_STATS + S_SE) * dstd / sqrt(N);
      if (mean != 0) {
        const double gc = gget(p, g, Q_STATS + S_COV);
        c[2] += gc * dstd / mean;
        a[0] -= gc * sd * iN / (mean * mean);
      }
    }
    if (m2 > 0) {
      // powers m2^(-k/2) from one reciprocal and one square root
      const double sq = sqrt(m2), ri = 1.0 / m2, rh = ri / sq;  // m2^-1, m2^-1.5
      const double r2 = ri * ri, r25 = r2 / sq, r3 = r2 * ri, r35 = r3 / sq, r4 = r2 * r2;
      c[2] += gget(p, g, Q_STATS + S_STD_B) / (2 * sq);
      const double gs = gget(p, g, Q_STATS + S_SKEW);
      c[3] += gs * rh;
      c[2] -= 1.5 * gs * m3 * r25;
      const double gk = gget(p, g, Q_STATS + S_KURT) + gget(p, g, Q_STATS + S_EXKURT);
      c[4] += gk * r2;
      c[2] -= 2.0 * gk * m4 * r3;
      const double gh = gget(p, g, Q_STATS + S_HSKEW);
      c[5] += gh * r25;
      c[2] -= 2.5 * gh * m5 * r35;
      const double gf = gget(p, g, Q_STATS + S_HFLAT);
      c[6] += gf * r3;
      c[2] -= 3.0 * gf * m6 * r4;
    }
    for (int j = 2; j <= 6; ++j) {  // c_j (j/N) (d^(j-1) - m_(j-1))
      a[j - 1] += c[j] * j * iN;
      a[0] -= c[j] * j * m[j - 1] * iN;
    }
    {
      const double gm = gget(p, g, Q_STATS + S_MAD);
      asg += gm * iN;
      a[0] -= gm * sv[SV_SGN] * iN * iN;
    }
    // ---- spatial polynomial in (u, v, w) = local coords - intensity centroid
    double b[NM];
    for (int k = 0; k < NM; ++k) b[k] = 0;
    const double cxyz[3] = {sv[SV_CX], sv[SV_CY], sv[SV_CZ]};
    const bool wvalid = sumI != 0;
    if (wvalid) {
      const double* MU = sv + SV_MU;
      const double M00 = sumI, iM00 = 1.0 / M00;
      // weighted centroids and mass displacement
      const double wc[3] = {sv[SV_X0] + cxyz[0], sv[SV_Y0] + cxyz[1], sv[SV_Z0] + cxyz[2]};
      const double bc[3] = {sv[SV_BX], sv[SV_BY], sv[SV_BZ]};
      double md2 = 0;
      for (int ax = 0; ax < NDIM; ++ax) md2 += (wc[ax] - bc[ax]) * (wc[ax] - bc[ax]);
      const double md = sqrt(md2);
      const int lin[3] = {bidx<NDIM>(1, 0, 0), bidx<NDIM>(0, 1, 0), NDIM == 3 ? bidx<NDIM>(0, 0, 1) : 0};
      const int swc[3] = {S_WCX, S_WCY, S_WCZ};
      const double gmd = gget(p, g, Q_STATS + S_MD);
      for (int ax = 0; ax < NDIM; ++ax) {
        b[lin[ax]] += gget(p, g, Q_STATS + swc[ax]) / sumI;
        if (md > 0) b[lin[ax]] += gmd * (wc[ax] - bc[ax]) / (sumI * md);
      }
      // normalised central moments and Hu invariants -> gradient on eta
      double geta[NM];
      for (int k = 0; k < NM; ++k) geta[k] = 0;
      const double mu00 = MU[0];
      double nmu[4], nM[4];  // normalisations of the central and raw moments by order
      gnorm_table<NDIM>(mu00, nmu);
      gnorm_table<NDIM>(M00, nM);
      const double imu00 = 1.0 / mu00;
      double inmu[4], inM[4];
      for (int o = 0; o < 4; ++o) {
        inmu[o] = 1.0 / nmu[o];
        inM[o] = 1.0 / nM[o];
      }
#pragma unroll
      for (int pp = 0; pp <= 3; ++pp)
#pragma unroll
        for (int qq = 0; pp + qq <= 3; ++qq)
#pragma unroll
          for (int rr = 0; rr <= (NDIM == 3 ? 3 - pp - qq : 0); ++rr) {
            const int k = bidx<NDIM>(pp, qq, rr);
            if (pp + qq + rr >= 2) geta[k] += gget(p, g, Q_MOM + F_ETA * 20 + k);
          }
      if (NDIM == 2) {
        const int ie[7] = {bidx<2>(2, 0, 0), bidx<2>(0, 2, 0), bidx<2>(1, 1, 0), bidx<2>(3, 0, 0),
                           bidx<2>(2, 1, 0), bidx<2>(1, 2, 0), bidx<2>(0, 3, 0)};
        double e[7], dh[7][7];
        for (int t = 0; t < 7; ++t) e[t] = MU[ie[t]] * inmu[t < 3 ? 2 : 3];
        hu_partials(e, dh);
        for (int h = 0; h < 7; ++h) {
          const double gh = gget(p, g, Q_MOM + F_HU * 20 + h);
          if (gh != 0)
            for (int t = 0; t < 7; ++t) geta[ie[t]] += gh * dh[h][t];
        }
      }
      // d mu_pqr coefficient (without the eta / nu scaling)
      double gmu[NM];
      double cst = 0;  // constant term from the normalisations
      for (int k = 0; k < NM; ++k) gmu[k] = gget(p, g, Q_MOM + F_MU * 20 + k);
#pragma unroll
      for (int pp = 0; pp <= 3; ++pp)
#pragma unroll
        for (int qq = 0; pp + qq <= 3; ++qq)
#pragma unroll
          for (int rr = 0; rr <= (NDIM == 3 ? 3 - pp - qq : 0); ++rr) {
            const int k = bidx<NDIM>(pp, qq, rr), o = pp + qq + rr;
            if (o >= 2 && geta[k] != 0) {
              const double gam = NDIM == 2 ? 1.0 + o / 2.0 : 1.0 + o / 3.0;
              const double iden = inmu[o];
              gmu[k] += geta[k] * iden;
              cst -= geta[k] * gam * (MU[k] * iden) * imu00;
            }
          }
#pragma unroll
      for (int pp = 0; pp <= 3; ++pp)
#pragma unroll
        for (int qq = 0; pp + qq <= 3; ++qq)
#pragma unroll
          for (int rr = 0; rr <= (NDIM == 3 ? 3 - pp - qq : 0); ++rr) {
            const int k = bidx<NDIM>(pp, qq, rr);
            const double gk = gmu[k];
            if (gk == 0) continue;
            b[k] += gk;
            if (pp > 0) b[lin[0]] -= gk * pp * MU[bidx<NDIM>(pp - 1, qq, rr)] * iM00;
            if (qq > 0) b[lin[1]] -= gk * qq * MU[bidx<NDIM>(pp, qq - 1, rr)] * iM00;
            if (NDIM == 3 && rr > 0) b[lin[2]] -= gk * rr * MU[bidx<NDIM>(pp, qq, rr - 1)] * iM00;
          }
      // raw and normalised raw moments: x^p y^q z^r expanded about the centroid
#pragma unroll
      for (int pp = 0; pp <= 3; ++pp)
#pragma unroll
        for (int qq = 0; pp + qq <= 3; ++qq)
#pragma unroll
          for (int rr = 0; rr <= (NDIM == 3 ? 3 - pp - qq : 0); ++rr) {
            const int k = bidx<NDIM>(pp, qq, rr), o = pp + qq + rr;
            double gk = gget(p, g, Q_MOM + F_M * 20 + k);
            if (NDIM == 2) {
              const double gn = gget(p, g, Q_MOM + F_NU * 20 + k);
              if (gn != 0) {
                const double iden = inM[o], gam = 1.0 + o / 2.0;
                double Mk = 0;  // raw moment from the central ones
#pragma unroll
                for (int i2 = 0; i2 <= pp; ++i2)
#pragma unroll
                  for (int j2 = 0; j2 <= qq; ++j2)
                    Mk += choose(pp, i2) * choose(qq, j2) * dpow(cxyz[0], pp - i2) * dpow(cxyz[1], qq - j2) *
                          MU[bidx<2>(i2, j2, 0)];
                gk += gn * iden;
                cst -= gn * gam * (Mk * iden) * iM00;
              }
            }
            if (gk == 0) continue;
#pragma unroll
            for (int i2 = 0; i2 <= pp; ++i2)
#pragma unroll
              for (int j2 = 0; j2 <= qq; ++j2)
#pragma unroll
                for (int l2 = 0; l2 <= rr; ++l2)
                  b[bidx<NDIM>(i2, j2, l2)] += gk * choose(pp, i2) * choose(qq, j2) * choose(rr, l2) *
                                               dpow(cxyz[0], pp - i2) * dpow(cxyz[1], qq - j2) *
                                               dpow(cxyz[2], rr - l2);
          }
      b[0] += cst;
    }
    // ---- scale to O(1) variables and store
    const double s = sd > 0 ? sd : 1.0;
    double L = 1.0;
    if (wvalid && sv[SV_MU] != 0) {
      const double* MU = sv + SV_MU;
      double q2 = (MU[bidx<NDIM>(2, 0, 0)] + MU[bidx<NDIM>(0, 2, 0)] + (NDIM == 3 ? MU[bidx<NDIM>(0, 0, 2)] : 0.0)) /
                  MU[0];
      if (q2 > 1) L = sqrt(q2);
    }
    const float mh = (float)mean;
    cf[0] = mh;
    cf[1] = (float)(mean - (double)mh);
    cf[2] = (float)(1.0 / s);
    for (int j = 0; j < 6; ++j) cf[3 + j] = (float)(a[j] * dpow(s, j));
    cf[9] = (float)asg;
    cf[10] = (float)cxyz[0];
    cf[11] = (float)cxyz[1];
    cf[12] = (float)cxyz[2];
    cf[13] = (float)sv[SV_X0];
    cf[14] = (float)sv[SV_Y0];
    cf[15] = (float)sv[SV_Z0];
    cf[16] = (float)(1.0 / L);
    for (int pp = 0; pp <= 3; ++pp)
      for (int qq = 0; pp + qq <= 3; ++qq)
        for (int rr = 0; rr <= (NDIM == 3 ? 3 - pp - qq : 0); ++rr) {
          const int k = bidx<NDIM>(pp, qq, rr);
          cf[17 + k] = (float)(b[k] * dpow(L, pp + qq + rr));
        }
    for (int k = 17 + NM; k < CW; ++k) cf[k] = 0.f;
    // ---- edge statistics, on edge pixels only: e0 + e1 (I - mean_E)
    const double geii = gget(p, g, Q_EDGE + E_II), gem = gget(p, g, Q_EDGE + E_MEAN),
                 ges = gget(p, g, Q_EDGE + E_STD);
    if (geii != 0 || gem != 0 || ges != 0) {
      const double ne = sv[SV_ECNT], es = sv[SV_ESTD];
      cf[EC0] = (float)(geii + gem / ne);
      cf[EC0 + 1] = (float)(es > 0 && ne > 1 ? ges / ((ne - 1) * es) : 0.0);
      cf[EC0 + 2] = (float)sv[SV_EMEAN];
    }
  }
}

template <class T, int NDIM>
__global__ void k_bwd_pixel(KParams p, const float* coef, float* gimg) {
  const int64_t total = p.rows_total * p.nx;
  const int64_t per = p.nx * p.ny * p.nz;
  const T* img = (const T*)p.img;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int L = __ldg(p.mask + i);
    float out = 0.f;
    if (L > 0) {
      const int64_t b = i / per;
      const unsigned long long key = ((unsigned long long)b << 32) | (unsigned)L;
      const int s = g_find(p.keys, p.hmask, key);
      const int r = s >= 0 ? p.slot_dense[s] : -1;
      if (r >= 0 && (int64_t)r < p.cap_roi) {
        const float* cf = coef + (size_t)r * CW;
        const float I = (float)__ldg(img + i);
        const float t = ((I - cf[0]) - cf[1]) * cf[2];
        float poly = cf[8];
#pragma unroll
        for (int j = 4; j >= 0; --j) poly = poly * t + cf[3 + j];
        poly += t > 0 ? cf[9] : (t < 0 ? -cf[9] : 0.f);
        const int64_t rem = i - b * per;
        const int x = (int)(rem % p.nx), y = (int)((rem / p.nx) % p.ny), z = (int)(rem / (p.nx * p.ny));
        const float e0 = cf[EC0], e1 = cf[EC0 + 1];
        if (e0 != 0.f || e1 != 0.f) {  // edge statistics: face-neighbour test on the mask
          bool edge = x == 0 || x == p.nx - 1 || y == 0 || y == p.ny - 1;
          if (NDIM == 3) edge = edge || z == 0 || z == p.nz - 1;
          if (!edge) {  // all neighbours inside the image: issue the loads together
            const int l0 = __ldg(p.mask + i - 1), l1 = __ldg(p.mask + i + 1);
            const int l2 = __ldg(p.mask + i - p.nx), l3 = __ldg(p.mask + i + p.nx);
            edge = (l0 != L) | (l1 != L) | (l2 != L) | (l3 != L);
            if (NDIM == 3) {
              const int64_t pl = p.nx * p.ny;
              const int l4 = __ldg(p.mask + i - pl), l5 = __ldg(p.mask + i + pl);
              edge |= (l4 != L) | (l5 != L);
            }
          }
          if (edge) poly += e0 + e1 * (I - cf[EC0 + 2]);
        }
        const float il = cf[16];
        const float u = ((float)x - cf[13] - cf[10]) * il, v = ((float)y - cf[14] - cf[11]) * il,
                    w = ((float)z - cf[15] - cf[12]) * il;
        float pu[4] = {1.f, u, u * u, u * u * u}, pv[4] = {1.f, v, v * v, v * v * v}, pw[4] = {1.f, w, w * w, w * w * w};
#pragma unroll
        for (int a = 0; a <= 3; ++a)
#pragma unroll
          for (int bq = 0; a + bq <= 3; ++bq)
#pragma unroll
            for (int c = 0; c <= (NDIM == 3 ? 3 - a - bq : 0); ++c)
              poly += cf[17 + bidx<NDIM>(a, bq, c)] * pu[a] * pv[bq] * pw[c];
        out = poly;
      }
    }
    gimg[i] = out;
  }
}

// k_bwd_coef is bound by the FP64 pipe (a few FP64 operations per clock per
// SM), one thread per ROI: one-warp blocks spread the ROIs over every SM
// instead of filling a few SMs with 128-thread blocks.
static int coef_blocks(const KParams& p, int nsm) {
  int64_t nb = (p.cap_roi + 31) / 32;
  if (nb > 64ll * nsm) nb = 64ll * nsm;
  return nb < 1 ? 1 : (int)nb;
}

template <class T>
cudaError_t launch_bwd_t(const KParams& p, const double* gtab, float* gimg, float* coef, int nsm, cudaStream_t st) {
  if (p.ndim == 3) {
    k_bwd_coef<3><<<coef_blocks(p, nsm), 32, 0, st>>>(p, gtab, coef);
    k_bwd_pixel<T, 3><<<8 * nsm, 256, 0, st>>>(p, coef, gimg);
  } else {
    k_bwd_coef<2><<<coef_blocks(p, nsm), 32, 0, st>>>(p, gtab, coef);
    k_bwd_pixel<T, 2><<<8 * nsm, 256, 0, st>>>(p, coef, gimg);
  }
  return cudaGetLastError();
}

}  // namespace

// coefficient scratch lives after the saved state of the plan
cudaError_t launch_backward(const KParams& p, const double* gtab, float* gimg, int nsm, cudaStream_t st) {
  float* coef = (float*)(p.saved + (size_t)p.max_rois * SV_WORDS);
  switch (p.dtype) {
    case NYX_U16: return launch_bwd_t<uint16_t>(p, gtab, gimg, coef, nsm, st);
    case NYX_I16: return launch_bwd_t<int16_t>(p, gtab, gimg, coef, nsm, st);
    default: return launch_bwd_t<float>(p, gtab, gimg, coef, nsm, st);
  }
}

}  // namespace nyx
