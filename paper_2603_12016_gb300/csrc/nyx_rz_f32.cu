// nyx_rz_f32.cu -- GLRLM / GLSZM kernels for float images (see nyx_runzone.cuh).
#include "nyx_runzone.cuh"

namespace nyx {
cudaError_t launch_rz_f32(const KParams& p, int big, int nsm, cudaStream_t st) { return launch_rz_t<float>(p, big, nsm, st); }
}  // namespace nyx
