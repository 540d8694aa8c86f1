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
    int tile_slots;               // inner mode: one slot per tile instead of per (CTA, segment)
    int64_t In, stride, hi_count;  // outer mode: o = (hi*In + j)*stride + lo
    const float* part;
    const float* W;
};

#ifdef __CUDACC__
// Every reduction below is a fixed-order sum over an index range that can be
// split into H contiguous pieces (piece h of H); the caller adds the pieces in
// order h = 0..H-1, so the result does not depend on how the work was spread.
// Loads go out 32 at a time, predicated, so that one piece costs one or two
// round trips to L2.

// Inner mode: partials per (CTA, segment, warp, row-in-block).  Only the CTAs
// whose contiguous tile range meets inner block ib contribute.
__device__ __forceinline__ float reduce_inner(const ReduceParams& P, int64_t j, int p, int h, int H) {
    const int64_t ib = j / P.I_T;
    const int b = (int)(j % P.I_T);
    if (P.tile_slots) {
        // one slot per tile (ib, ot): sum over the n_ot tiles of block ib
        const int64_t oa = (P.n_ot * h) / H, ob = (P.n_ot * (h + 1)) / H;
        const float* q = P.part + ((ib * P.n_ot) * P.I_T + b) * P.RP + p;
        const int64_t tstride = (int64_t)P.I_T * P.RP;
        float s = 0.f;
        for (int64_t o = oa; o < ob; o += 32) {
            float x[32];
#pragma unroll
            for (int u = 0; u < 32; ++u) x[u] = (o + u < ob) ? q[(o + u) * tstride] : 0.f;
#pragma unroll
            for (int u = 0; u < 32; ++u) s += x[u];
        }
        return s;
    }
    const int64_t t0 = ib * P.n_ot, t1 = t0 + P.n_ot;   // tiles of block ib
    // CTA g owns tiles [floor(n_tiles g / G), floor(n_tiles (g+1) / G)); the CTA owning tile t is
    // floor(((t + 1) G - 1) / n_tiles)
    const int g0 = (int)(((t0 + 1) * P.G - 1) / P.n_tiles);
    const int g1 = (int)((t1 * P.G - 1) / P.n_tiles);
    // CTA g0 may have started in an earlier block (segment ib - its first block); every later
    // CTA that meets block ib starts inside it (segment 0)
    const int seg0 = (int)(ib - ((P.n_tiles * g0) / P.G) / P.n_ot);
    const int cnt = g1 - g0 + 1;
    const int ga = g0 + (cnt * h) / H, gb = g0 + (cnt * (h + 1)) / H;   // this piece: CTAs [ga, gb)
    const int64_t slot = (int64_t)P.part_warps * P.I_T * P.RP;          // one (CTA, segment) slot
    const int64_t wstride = (int64_t)P.I_T * P.RP;
    const float* q = P.part + (int64_t)b * P.RP + p;
    float s = 0.f;
    if (P.part_warps == 1) {
        for (int g = ga; g < gb; g += 32) {
            float x[32];
#pragma unroll
            for (int u = 0; u < 32; ++u) {
                const int gg = g + u;
                x[u] = gg < gb ? q[((int64_t)gg * P.Smax + (gg == g0 ? seg0 : 0)) * slot] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 32; ++u) s += x[u];
        }
        return s;
    }
    for (int g = ga; g < gb; g += 4) {
        float x[4][8];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int gg = g + u;
            const float* qg = q + ((int64_t)gg * P.Smax + (gg == g0 ? seg0 : 0)) * slot;
#pragma unroll
            for (int w = 0; w < 8; ++w) x[u][w] = (gg < gb && w < P.part_warps) ? qg[w * wstride] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int w = 0; w < 8; ++w) s += x[u][w];
    }
    return s;
}

// Outer mode: one partial per tile (o, ib), weighted by W(o, p), summed over
// all outer indices o with i_n(o) = j (piece h takes a contiguous range of them).
__device__ __forceinline__ float reduce_outer(const ReduceParams& P, int64_t j, int p, int h, int H) {
    const int64_t n = P.hi_count * P.stride;
    const int64_t ka = (n * h) / H, kb = (n * (h + 1)) / H;
    float s = 0.f;
    for (int64_t k = ka; k < kb; ++k) {
        const int64_t hi = k / P.stride, lo = k - hi * P.stride;
        const int64_t o = (hi * P.In + j) * P.stride + lo;
        float so = 0.f;
#pragma unroll 4
        for (int64_t ib = 0; ib < P.nb; ++ib) so += P.part[(o * P.nb + ib) * P.RP + p];
        s = fmaf(P.W[o * P.RP + p], so, s);
    }
    return s;
}

// Last mode: one partial per streaming CTA along the tile axis.
__device__ __forceinline__ float reduce_last(const ReduceParams& P, int64_t c, int p, int h, int H) {
    const int ga = (P.G * h) / H, gb = (P.G * (h + 1)) / H;
    float s = 0.f;
    const float* q = P.part + c * P.RP + p;
    const int64_t stride = P.Cpad * P.RP;
    for (int g = ga; g < gb; g += 32) {
        float x[32];
#pragma unroll
        for (int u = 0; u < 32; ++u) x[u] = (g + u < gb) ? q[(int64_t)(g + u) * stride] : 0.f;
#pragma unroll
        for (int u = 0; u < 32; ++u) s += x[u];
    }
    return s;
}

// piece h of H of M(j, p)
__device__ __forceinline__ float reduce_piece(const ReduceParams& P, int64_t j, int p, int h, int H) {
    return P.kind == 0 ? reduce_inner(P, j, p, h, H) : P.kind == 1 ? reduce_outer(P, j, p, h, H)
                                                                   : reduce_last(P, j, p, h, H);
}

__device__ __forceinline__ float reduce_output(const ReduceParams& P, int64_t j, int p) {
    return reduce_piece(P, j, p, 0, 1);
}
#endif

}  // namespace ntf
