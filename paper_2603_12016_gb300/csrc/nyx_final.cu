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
// direction means are compensated sums.
#include "nyx_roi.cuh"

namespace nyx {

constexpr int FIN_STRIDE = NGLCM + 3;  // odd row stride (in A) of the shared feature matrix

template <class A>
__global__ void __launch_bounds__(256) k_glcm_final(KParams p, int rpb) {
  extern __shared__ __align__(16) unsigned char smem[];
  A* sf = (A*)smem;  // [rpb * n_off][FIN_STRIDE]
  const int n_off = p.n_dist * p.n_dirs;
  const int64_t nroi = min((int64_t)*p.n_roi, p.cap_roi);
  const A nan = anan<A>();
  const int lr = threadIdx.x / n_off, oi = threadIdx.x - lr * n_off;
  for (int64_t base = (int64_t)blockIdx.x * rpb; base < nroi; base += (int64_t)gridDim.x * rpb) {
    const int64_t item = base + lr;
    A* f = sf + threadIdx.x * FIN_STRIDE;
    if (lr < rpb && item < nroi) {
      const long long* g = (const long long*)(p.gacc + ((size_t)item * n_off + oi) * GACC_BYTES);
      double* row = p.table + item * p.n_col;
      const int di = oi / p.n_dirs, dir = oi - di * p.n_dirs;
      long long iv[GN];
#pragma unroll
      for (int k = 0; k < GN; ++k) iv[k] = g[k];
      if (iv[0] == 0) {  // offset without pairs
        if (p.per_offset)
          for (int k = 0; k < NGLCM; ++k) putA(p, row, Q_GLCM_O + (di * MAX_DIRS + dir) * NGLCM + k, nan);
        f[NGLCM] = 0;
      } else {
        finalize_glcm<A>(p, row, iv, di, dir, f);
      }
    }
    __syncthreads();
    // direction means, compensated sums in offset order (features that
    // change sign with the direction keep the accuracy of their mean)
    const int per_roi = p.n_dist * NGLCM;
    for (int t = threadIdx.x; t < rpb * per_roi; t += blockDim.x) {
      const int l2 = t / per_roi, rem = t - l2 * per_roi;
      const int di = rem / NGLCM, k = rem - di * NGLCM;
      const int64_t it = base + l2;
      if (it >= nroi) continue;
      A s = 0, e = 0;
      int c = 0;
      for (int dir = 0; dir < p.n_dirs; ++dir) {
        const A* fo = sf + (l2 * n_off + di * p.n_dirs + dir) * FIN_STRIDE;
        if (fo[NGLCM] == 0) continue;
        if constexpr (std::is_same<A, float>::value) {
          float t, er;
          two_sum(s, fo[k], t, er);
          s = t;
          e += er;
        } else {
          s += fo[k];
        }
        ++c;
      }
      putA(p, p.table + it * p.n_col, Q_GLCM_D + di * NGLCM + k, c > 0 ? (s + e) / (A)c : nan);
    }
    __syncthreads();
  }
}

template <class A>
static cudaError_t launch_final_t(const KParams& p, int nsm, cudaStream_t st) {
  const int n_off = p.n_dist * p.n_dirs;
  const int rpb = n_off >= 256 ? 1 : 256 / n_off;
  const int nt = rpb * n_off;
  const int smem = nt * FIN_STRIDE * (int)sizeof(A);
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
