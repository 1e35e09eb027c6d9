// nyx_roi_i16.cu -- per-ROI feature kernels for int16_t images (see nyx_roi.cuh).
#include "nyx_roi.cuh"

namespace nyx {
cudaError_t launch_roi_i16(const KParams& p, int cls, int fp64, int nsm, cudaStream_t st) {
  return launch_roi_t<int16_t>(p, cls, fp64, nsm, st);
}
}  // namespace nyx
