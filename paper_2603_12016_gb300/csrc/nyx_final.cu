// nyx_final.cu -- GLCM features (Table S3 rows 140-174) from the per (ROI,
// offset) accumulators that the accumulation kernels of every size class
// leave in the plan's gacc buffer.
//
// One thread per (ROI, offset) evaluates the 30 features of its offset (the
// exact integer moments and marginal entropies, finalize_glcm) and writes the
// per-offset columns; the block then forms the mean over the directions of
// each distance (offsets without pairs excluded, NaN when none has pairs).
// Doing this outside the accumulation kernels keeps their blocks from idling
// at a barrier while one thread runs the serial feature arithmetic.  Every
// feature is a quotient of exact integer numerators (finalize_glcm); the
// direction means are summed in FP64.
#include "nyx_roi.cuh"

namespace nyx {

constexpr int FIN_STRIDE = NGLCM + 3;  // odd row stride (doubles) of the shared feature matrix

// 1 / c for the number c of directions with pairs (1 .. 13), correctly rounded
__device__ __constant__ const double c_inv_dirs[MAX_DIRS + 1] = {
    0.0, 1.0, 1.0 / 2, 1.0 / 3, 1.0 / 4, 1.0 / 5, 1.0 / 6, 1.0 / 7, 1.0 / 8, 1.0 / 9, 1.0 / 10, 1.0 / 11, 1.0 / 12, 1.0 / 13};

template <class A>
__global__ void __launch_bounds__(256) k_glcm_final(KParams p, int rpb) {
  extern __shared__ __align__(16) unsigned char smem[];
  double* sf = (double*)smem;  // [rpb * n_off][FIN_STRIDE]
  const int n_off = p.n_dist * p.n_dirs;
  const int64_t nroi = min((int64_t)*p.n_roi, p.cap_roi);
  const double nan = anan<double>();
  const int lr = threadIdx.x / n_off, oi = threadIdx.x - lr * n_off;
  for (int64_t base = (int64_t)blockIdx.x * rpb; base < nroi; base += (int64_t)gridDim.x * rpb) {
    const int64_t item = base + lr;
    double* f = sf + threadIdx.x * FIN_STRIDE;
    if (lr < rpb && item < nroi) {
      const long long* g = (const long long*)(p.gacc + ((size_t)item * n_off + oi) * GACC_BYTES);
      double* row = p.table + item * p.n_col;
      const int di = oi / p.n_dirs, dir = oi - di * p.n_dirs;
      long long iv[GN];
#pragma unroll
      for (int k = 0; k < GN; ++k) iv[k] = g[k];
      if (iv[0] == 0) {  // offset without pairs
        if (p.per_offset)
          for (int k = 0; k < NGLCM; ++k) put(p, row, Q_GLCM_O + (di * MAX_DIRS + dir) * NGLCM + k, nan);
        f[NGLCM] = 0;
      } else {
        finalize_glcm<A>(p, row, iv, di, dir, f);
      }
    }
    __syncthreads();
    // direction means (FP64), summed in offset order
    const int per_roi = p.n_dist * NGLCM;
    for (int t = threadIdx.x; t < rpb * per_roi; t += blockDim.x) {
      const int l2 = t / per_roi, rem = t - l2 * per_roi;
      const int di = rem / NGLCM, k = rem - di * NGLCM;
      const int64_t it = base + l2;
      if (it >= nroi) continue;
      double s = 0, c = 0;
      for (int dir = 0; dir < p.n_dirs; ++dir) {
        const double* fo = sf + (l2 * n_off + di * p.n_dirs + dir) * FIN_STRIDE;
        if (fo[NGLCM] == 0) continue;
        s += fo[k];
        c += 1;
      }
      // 1/c from a table (c <= 13 directions): no FP64 division
      put(p, p.table + it * p.n_col, Q_GLCM_D + di * NGLCM + k, c > 0 ? s * c_inv_dirs[(int)c] : nan);
    }
    __syncthreads();
  }
}

template <class A>
static cudaError_t launch_final_t(const KParams& p, int nsm, cudaStream_t st) {
  const int n_off = p.n_dist * p.n_dirs;
  const int rpb = n_off >= 256 ? 1 : 256 / n_off;
  const int nt = rpb * n_off;
  const int smem = nt * FIN_STRIDE * (int)sizeof(double);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  static int configured[64] = {0};
  if (smem > 48 * 1024 && (dev >= 64 || configured[dev] < smem)) {
    e = cudaFuncSetAttribute(k_glcm_final<A>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    if (dev < 64) configured[dev] = smem;
  }
  const int64_t rows = p.cap_roi < p.max_rois ? p.cap_roi : p.max_rois;
  int64_t nb = (rows + rpb - 1) / rpb;
  if (nb > 8ll * nsm) nb = 8ll * nsm;
  if (nb < 1) nb = 1;
  k_glcm_final<A><<<(int)nb, nt, smem, st>>>(p, rpb);
  return cudaGetLastError();
}

cudaError_t launch_glcm_final(const KParams& p, int fp64, int nsm, cudaStream_t st) {
  return fp64 ? launch_final_t<double>(p, nsm, st) : launch_final_t<float>(p, nsm, st);
}

}  // namespace nyx
