// BF16-storage instantiations of the streaming MTTKRP kernels (FP32 accumulate).
#include "mttkrp_kernels.cuh"

namespace ntf {
cudaError_t launch_stream_bf16(int kind, int R, dim3 grid, size_t smem, cudaStream_t st, const CUtensorMap& map,
                               const StreamParams& P, bool pdl) {
    return launch_stream_impl<__nv_bfloat16>(kind, R, grid, smem, st, map, P, pdl);
}
}  // namespace ntf
