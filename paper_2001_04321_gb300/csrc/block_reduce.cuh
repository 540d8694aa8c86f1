// Warp and block sums in FP64 shared by the non-streaming kernels (small.cu, bcd*.cu).
#pragma once

namespace ntf {

// ---------------------------------------------------------------------------
// block reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// sum over the block (blockDim multiple of 32, <= 1024); result valid in every thread
__device__ inline double block_sum_d(double v, double* sbuf /* >= 33 doubles */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum_d(v);
    __syncthreads();
    if (lane == 0) sbuf[warp] = v;
    __syncthreads();
    if (warp == 0) {
        double t = lane < nw ? sbuf[lane] : 0.0;
        t = warp_sum_d(t);
        if (lane == 0) sbuf[32] = t;
    }
    __syncthreads();
    return sbuf[32];
}

}  // namespace ntf
