// Second pass of the MTTKRP (step a1): the fixed-order sum of the streaming
// kernels' partial results for one output element M(j, p).  Shared by the
// stand-alone reduction kernels and the solver's fused epilogue.
#pragma once

#include "ntf_common.cuh"

namespace ntf {

struct ReduceParams {
    int kind;                     // 0 inner, 1 outer, 2 last
    int64_t n_tiles, n_ot, nb, Ii, n_o, C, Cpad;
    int G, Smax, I_T, RP, r;
    int part_warps;               // inner mode: partial slots per CTA (8 per-warp, or 1)
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
    // CTA g owns tiles [floor(n_tiles g / G), floor(n_tiles (g+1) / G)); the CTA owning tile t is
    // floor(((t + 1) G - 1) / n_tiles)
    const int g0 = (int)(((t0 + 1) * P.G - 1) / P.n_tiles);
    const int g1 = (int)((t1 * P.G - 1) / P.n_tiles);
    // CTA g0 may have started in an earlier block (segment ib - its first block); every later
    // CTA that meets block ib starts inside it (segment 0)
    const int seg0 = (int)(ib - ((P.n_tiles * g0) / P.G) / P.n_ot);
    const int64_t slot = (int64_t)P.part_warps * P.I_T * P.RP;          // one (CTA, segment) slot
    const float* q = P.part + (int64_t)b * P.RP + p;
    float s = 0.f;
    if (P.part_warps == 1) {
        // one partial per CTA: up to 16 independent loads in flight, summed in order
        s = q[((int64_t)g0 * P.Smax + seg0) * slot];
        for (int g = g0 + 1; g <= g1; g += 16) {
            float x[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) x[u] = (g + u <= g1) ? q[((int64_t)(g + u) * P.Smax) * slot] : 0.f;
#pragma unroll
            for (int u = 0; u < 16; ++u) s += x[u];
        }
        return s;
    }
    for (int w = 0; w < P.part_warps; ++w) s += q[((int64_t)g0 * P.Smax + seg0) * slot + (int64_t)w * P.I_T * P.RP];
    for (int g = g0 + 1; g <= g1; ++g) {
        float x[8];
#pragma unroll
        for (int w = 0; w < 8; ++w) x[w] = w < P.part_warps ? q[((int64_t)g * P.Smax) * slot + (int64_t)w * P.I_T * P.RP] : 0.f;
#pragma unroll
        for (int w = 0; w < 8; ++w) s += x[w];
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
#pragma unroll 4
            for (int64_t ib = 0; ib < P.nb; ++ib) so += P.part[(o * P.nb + ib) * P.RP + p];
            s = fmaf(P.W[o * P.RP + p], so, s);
        }
    return s;
}

// Last mode: one partial per streaming CTA along the tile axis.
__device__ __forceinline__ float reduce_last(const ReduceParams& P, int64_t c, int p) {
    float s = 0.f;
    const float* q = P.part + c * P.RP + p;
    const int64_t stride = P.Cpad * P.RP;
    for (int g = 0; g < P.G; g += 16) {
        float x[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) x[u] = (g + u < P.G) ? q[(int64_t)(g + u) * stride] : 0.f;
#pragma unroll
        for (int u = 0; u < 16; ++u) s += x[u];
    }
    return s;
}

__device__ __forceinline__ float reduce_output(const ReduceParams& P, int64_t j, int p) {
    return P.kind == 0 ? reduce_inner(P, j, p) : P.kind == 1 ? reduce_outer(P, j, p) : reduce_last(P, j, p);
}
#endif

}  // namespace ntf
