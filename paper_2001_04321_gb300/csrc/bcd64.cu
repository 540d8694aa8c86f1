// Step a3 block updates of width 64 (see bcd.cuh).
#include "bcd.cuh"

namespace ntf {

cudaError_t launch_bcd_r64(int method, float* A, int64_t rows, int r, const float* M, const double* V,
                           int inner_max, double tol, double* L, double* parts, int* stopped, float* Y,
                           cudaStream_t st) {
    return bcd_impl<64>(method, A, rows, r, M, V, inner_max, tol, L, parts, stopped, Y, st);
}

}  // namespace ntf
