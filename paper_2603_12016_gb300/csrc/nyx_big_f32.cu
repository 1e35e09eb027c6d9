// nyx_big_f32.cu -- multi-block (class 3) ROI kernels for float images (see nyx_roi_big.cuh).
#include "nyx_roi_big.cuh"

namespace nyx {
cudaError_t launch_big_f32(const KParams& p, int fp64, int nsm, cudaStream_t st) {
  return launch_big_t<float>(p, fp64, nsm, st);
}
}  // namespace nyx
