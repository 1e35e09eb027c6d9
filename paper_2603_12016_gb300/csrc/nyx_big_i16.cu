// nyx_big_i16.cu -- multi-block (class 3) ROI kernels for int16_t images (see nyx_roi_big.cuh).
#include "nyx_roi_big.cuh"

namespace nyx {
cudaError_t launch_big_i16(const KParams& p, int fp64, int nsm, cudaStream_t st) {
  return launch_big_t<int16_t>(p, fp64, nsm, st);
}
}  // namespace nyx
