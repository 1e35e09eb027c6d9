// nyx_rz_i16.cu -- GLRLM / GLSZM kernels for int16_t images (see nyx_runzone.cuh).
#include "nyx_runzone.cuh"

namespace nyx {
cudaError_t launch_rz_i16(const KParams& p, int big, int nsm, cudaStream_t st) { return launch_rz_t<int16_t>(p, big, nsm, st); }
}  // namespace nyx
