// FP32 instantiations of the streaming MTTKRP kernels.
#include "mttkrp_kernels.cuh"

namespace ntf {
cudaError_t launch_stream_f32(int kind, int R, dim3 grid, size_t smem, cudaStream_t st, const CUtensorMap& map,
                              const StreamParams& P, bool pdl) {
    return launch_stream_impl<float>(kind, R, grid, smem, st, map, P, pdl);
}
}  // namespace ntf
