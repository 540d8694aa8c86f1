// Step a3 launchers (HALS, projected gradient and AO-Nesterov; Sec. 2.1.4, 2.2 and 2.1): widths
// up to 24 here, 32 and 64 in bcd32.cu and bcd64.cu.
#include "bcd.cuh"

namespace ntf {

// [0, 256): L and the stop flag; then 3 G partial sums; then (AO-Nesterov, many CTAs) the
// extrapolated point Y, rows x r floats, 256-byte aligned
static size_t bcd_y_offset(int64_t rows) {
    const int64_t G = (rows + kBcdThreads - 1) / kBcdThreads;
    return (256 + sizeof(double) * (size_t)(3 * G + 8) + 255) & ~size_t(255);
}

size_t bcd_workspace(int64_t rows, int r) { return bcd_y_offset(rows) + sizeof(float) * (size_t)rows * (size_t)r; }

cudaError_t launch_bcd(int method, float* A, int64_t rows, int r, const float* M, const double* V, int inner_max,
                       double tol, void* ws, cudaStream_t st) {
    unsigned char* w = static_cast<unsigned char*>(ws);
    double* L = reinterpret_cast<double*>(w);
    int* stopped = reinterpret_cast<int*>(w + 8);
    double* parts = reinterpret_cast<double*>(w + 256);
    float* Y = reinterpret_cast<float*>(w + bcd_y_offset(rows));
    const int R = r <= 4 ? 4 : r <= 8 ? 8 : r <= 12 ? 12 : r <= 16 ? 16 : r <= 20 ? 20 : r <= 24 ? 24 : r <= 32 ? 32 : 64;
    switch (R) {
        case 4: return bcd_impl<4>(method, A, rows, r, M, V, inner_max, tol, L, parts, stopped, Y, st);
        case 8: return bcd_impl<8>(method, A, rows, r, M, V, inner_max, tol, L, parts, stopped, Y, st);
        case 12: return bcd_impl<12>(method, A, rows, r, M, V, inner_max, tol, L, parts, stopped, Y, st);
        case 16: return bcd_impl<16>(method, A, rows, r, M, V, inner_max, tol, L, parts, stopped, Y, st);
        case 20: return bcd_impl<20>(method, A, rows, r, M, V, inner_max, tol, L, parts, stopped, Y, st);
        case 24: return bcd_impl<24>(method, A, rows, r, M, V, inner_max, tol, L, parts, stopped, Y, st);
        case 32: return launch_bcd_r32(method, A, rows, r, M, V, inner_max, tol, L, parts, stopped, Y, st);
        default: return launch_bcd_r64(method, A, rows, r, M, V, inner_max, tol, L, parts, stopped, Y, st);
    }
}

}  // namespace ntf
