// Second pass of the MTTKRP (step a1): the fixed-order sum of the streaming
// kernels' partial results for one output element M(j, p).  Shared by the
// stand-alone reduction kernels and the solver's fused epilogue.
#pragma once

#include "ntf_common.cuh"

namespace ntf {

constexpr int kPartWarps = 8;   // per-warp partial slots of the inner-mode stream

struct ReduceParams {
    int kind;                     // 0 inner, 1 outer, 2 last
    int64_t n_tiles, n_ot, nb, Ii, n_o, C, Cpad;
    int G, Smax, I_T, RP, r;
    int64_t In, stride, hi_count;  // outer mode: o = (hi*In + j)*stride + lo
    const float* part;
    const float* W;
};

#ifdef __CUDACC__
// Inner mode: partials per (CTA, segment, warp, row-in-block).  Only the CTAs
// whose contiguous tile range meets inner block ib contribute.
__device__ __forceinline__ float reduce_inner(const ReduceParams& P, int64_t j, int p) {
    const int64_t ib = j / P.I_T;
    const int b = (int)(j % P.I_T);
    const int64_t t0 = ib * P.n_ot, t1 = t0 + P.n_ot;   // tiles of block ib
    int g = (int)((t0 * P.G) / P.n_tiles);
    while (g > 0 && (P.n_tiles * g) / P.G > t0) --g;
    float s = 0.f;
    for (; g < P.G; ++g) {
        const int64_t tb = (P.n_tiles * g) / P.G, te = (P.n_tiles * (g + 1)) / P.G;
        if (tb >= t1) break;
        if (te <= t0 || te <= tb) continue;
        const int seg = (int)(ib - tb / P.n_ot);
        const float* q = P.part + ((((int64_t)g * P.Smax + seg) * kPartWarps) * P.I_T + b) * P.RP + p;
#pragma unroll
        for (int w = 0; w < kPartWarps; ++w) s += q[(int64_t)w * P.I_T * P.RP];
    }
    return s;
}

// Outer mode: one partial per tile (o, ib), weighted by W(o, p), summed over
// all outer indices o with i_n(o) = j.
__device__ __forceinline__ float reduce_outer(const ReduceParams& P, int64_t j, int p) {
    float s = 0.f;
    for (int64_t hi = 0; hi < P.hi_count; ++hi)
        for (int64_t lo = 0; lo < P.stride; ++lo) {
            const int64_t o = (hi * P.In + j) * P.stride + lo;
            float so = 0.f;
            for (int64_t ib = 0; ib < P.nb; ++ib) so += P.part[(o * P.nb + ib) * P.RP + p];
            s = fmaf(P.W[o * P.RP + p], so, s);
        }
    return s;
}

// Last mode: one partial per streaming CTA along the tile axis.
__device__ __forceinline__ float reduce_last(const ReduceParams& P, int64_t c, int p) {
    float s = 0.f;
    for (int g = 0; g < P.G; ++g) s += P.part[((int64_t)g * P.Cpad + c) * P.RP + p];
    return s;
}

__device__ __forceinline__ float reduce_output(const ReduceParams& P, int64_t j, int p) {
    return P.kind == 0 ? reduce_inner(P, j, p) : P.kind == 1 ? reduce_outer(P, j, p) : reduce_last(P, j, p);
}
#endif

}  // namespace ntf
