// nyx_roi_f32.cu -- per-ROI feature kernels for float images (see nyx_roi.cuh).
#include "nyx_roi.cuh"

namespace nyx {
cudaError_t launch_roi_f32(const KParams& p, int cls, int fp64, int nsm, cudaStream_t st) {
  return launch_roi_t<float>(p, cls, fp64, nsm, st);
}
}  // namespace nyx
