// Streaming MTTKRP kernels (step a1).  Included by the per-dtype translation
// units mttkrp_f32.cu / mttkrp_bf16.cu, which instantiate them.
//
// View: C = I_{N-1} (contiguous), Ii = I_{N-2}, n_o = prod_{l<N-2} I_l; row
// (o, i) of the (n_o*Ii) x C matrix T_mat has pitch ld.  With
// Y = T_mat * A_{N-1} and W(o,p) = prod_{l<N-2, l != n} A_l(i_l(o), p):
//   inner mode n = N-2 : M(i,p) = sum_o W(o,p) Y((o,i),p)
//   outer mode n < N-2 : S(o,p) = sum_i Y((o,i),p) A_{N-2}(i,p)   (finished by
//                        the reduce kernel: M(j,p) = sum_{i_n(o)=j} W(o,p) S(o,p))
//   last mode  n = N-1 : M(c,p) = sum_{o,i} T((o,i),c) W(o,p) A_{N-2}(i,p)
// This is T_[n] B^n of Sec. 2 (def:B, def:grad) with the Khatri-Rao rows of
// B^n generated on the fly and never stored.
//
// Pipeline: a tile is 128 rows (O_T outer x I_T inner indices) of T_mat; a
// stage holds 64 columns of one tile (2 TMA boxes of 32 f32 or 1 box of 64
// bf16, 128-byte swizzled) plus, for the row kernels, the matching 64 rows of
// the packed last-mode factor (1-D bulk copy).  One producer warp fills a
// 4-stage ring; 8 consumer warps run FP32 FMAs.  All waits are bounded.
#pragma once

#include "ntf_common.cuh"

namespace ntf {

constexpr int kStreamWarps = 8;
constexpr int kStreamThreads = (kStreamWarps + 1) * 32;
constexpr int kStreamStages = 4;
constexpr int kTileRows = 128;
constexpr int kStageCols = 64;

struct StreamParams {
    int64_t C, Ii, n_o;
    int I_T, O_T;
    int64_t nb, n_ot, n_tiles;
    int n_kc;             // 64-column chunks of C
    int RP;               // packed factor width (floats per row)
    int Smax;             // inner mode: segments per CTA
    int64_t Cpad;         // last mode: rows of the partial buffer
    const float* Fc;      // packed A_{N-1}: round_up(C,64) x RP, zero padded
    const float* Fi;      // packed A_{N-2}: Ii x RP
    const float* W;       // n_o x RP
    float* part;          // partial sums (layout per kernel)
    int* err;
};

template <typename TE>
struct TileBytes {
    static constexpr int value = kTileRows * kStageCols * (int)sizeof(TE);  // 32 KB f32, 16 KB bf16
    static constexpr int boxes = (kStageCols * (int)sizeof(TE)) / 128;      // 2 f32, 1 bf16
    static constexpr int box_cols = 128 / (int)sizeof(TE);                  // 32 f32, 64 bf16
};

inline size_t stream_rows_smem(int elem_bytes, int RP) {
    // stages + barriers (128 B) + double-buffered cross-warp sums of the outer mode (2 x 8 x 32 floats)
    return (size_t)kStreamStages * (kTileRows * kStageCols * elem_bytes + kStageCols * RP * 4) + 1024 + 128 + 2048;
}
inline size_t stream_last_smem(int elem_bytes, int R) {
    return (size_t)kStreamStages * (kTileRows * kStageCols * elem_bytes + kTileRows * R * 4) + 1024 + 128;
}

#ifdef __CUDACC__

// shared-memory address of 16-byte chunk `chunk` of row m of a TMA box written
// with CU_TENSOR_MAP_SWIZZLE_128B (box base 1024-byte aligned)
__device__ __forceinline__ uint32_t sw128(uint32_t box_base, int m, int chunk) {
    return box_base + (uint32_t)m * 128u + ((uint32_t)(chunk ^ (m & 7)) << 4);
}

__device__ __forceinline__ float4 lds128f(uint32_t addr) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0,%1,%2,%3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(addr));
    return v;
}
__device__ __forceinline__ uint4 lds128u(uint32_t addr) {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0,%1,%2,%3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(addr));
    return v;
}
__device__ __forceinline__ uint2 lds64u(uint32_t addr) {
    uint2 v;
    asm volatile("ld.shared.v2.u32 {%0,%1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(addr));
    return v;
}

__device__ __forceinline__ void tile_range(int64_t n_tiles, int g, int G, int64_t& b, int64_t& e) {
    b = (n_tiles * g) / G;
    e = (n_tiles * (g + 1)) / G;
}

// Bounded wait taken by a whole warp: every lane polls (so every lane gets the
// barrier's acquire ordering) and the warp agrees on one outcome, so a time-out
// can never split a warp before a shuffle or a named barrier.
__device__ __forceinline__ bool warp_wait_bounded(uint64_t* bar, uint32_t parity) {
    const bool mine = mbar_wait_bounded(bar, parity);
    return __all_sync(0xffffffffu, mine) != 0;
}

// Producer drain: wait (bounded) until every copy this thread issued has
// landed, so that no TMA write is in flight when the CTA retires.
// acc[0..3] += a * (f.x, f.y, f.z, f.w) as two packed FP32x2 FMAs (each lane an
// IEEE fma, round to nearest): half the FMA issue slots of four scalar FMAs
__device__ __forceinline__ void fma4(float* acc, float a, const float4& f) {
    const float2 a2 = make_float2(a, a);
    const float2 lo = __ffma2_rn(a2, make_float2(f.x, f.y), make_float2(acc[0], acc[1]));
    const float2 hi = __ffma2_rn(a2, make_float2(f.z, f.w), make_float2(acc[2], acc[3]));
    acc[0] = lo.x;
    acc[1] = lo.y;
    acc[2] = hi.x;
    acc[3] = hi.y;
}

__device__ __forceinline__ void drain_stages(uint64_t* full, int stage, uint32_t phase, int64_t issued, int* err) {
    const int64_t inflight = issued < kStreamStages ? issued : kStreamStages;
    for (int64_t q = 0; q < inflight; ++q) {
        int s = stage - 1 - (int)q;
        uint32_t ph = phase;
        while (s < 0) { s += kStreamStages; ph ^= 1u; }
        if (!mbar_wait_bounded(&full[s], ph)) { record_device_error(err, kErrWaitDrain); break; }
    }
}

// ---------------------------------------------------------------------------
// rows kernel: inner mode (INNER = true) and outer modes (INNER = false)
// ---------------------------------------------------------------------------
template <typename TE, int R, bool INNER>
__global__ void __launch_bounds__(kStreamThreads, 1)
    k_stream_rows(const __grid_constant__ CUtensorMap tmap, const StreamParams P) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    using TB = TileBytes<TE>;
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char* base_ptr = smem_raw + (base - raw);
    const int fbytes = kStageCols * P.RP * 4;
    unsigned char* fchunk_ptr = base_ptr + kStreamStages * TB::value;
    uint64_t* full = reinterpret_cast<uint64_t*>(fchunk_ptr + kStreamStages * fbytes);
    uint64_t* empty = full + kStreamStages;
    float* zsum = reinterpret_cast<float*>(fchunk_ptr + kStreamStages * fbytes + 128);   // [2][8][32]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = blockIdx.x, G = gridDim.x;
    const int p0 = blockIdx.y * R;
    int64_t t_beg, t_end;
    tile_range(P.n_tiles, g, G, t_beg, t_end);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStreamStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kStreamWarps);
        }
        fence_mbar_init();
    }
    __syncthreads();
    pdl_wait();
    pdl_trigger();

    if (warp == kStreamWarps) {
        // ------------------------------ producer ------------------------------
        if (lane == 0) {
            prefetch_tensormap(&tmap);
            int stage = 0;
            uint32_t phase = 0;
            int64_t issued = 0;
            bool ok = true;
            for (int64_t t = t_beg; t < t_end && ok; ++t) {
                int64_t ib, ot;
                if (INNER) { ib = t / P.n_ot; ot = t % P.n_ot; }
                else { ot = t / P.nb; ib = t % P.nb; }
                for (int kc = 0; kc < P.n_kc; ++kc) {
                    if (!mbar_wait_bounded(&empty[stage], phase ^ 1u)) {
                        record_device_error(P.err, kErrWaitEmpty);
                        ok = false;
                        break;
                    }
                    // boxes that start at or beyond the last column are not issued (their
                    // columns are skipped by the consumers)
                    const int64_t left = P.C - (int64_t)kc * kStageCols;
                    const int nbox = left >= kStageCols ? TB::boxes : (int)((left + TB::box_cols - 1) / TB::box_cols);
                    mbar_arrive_expect_tx(&full[stage], (uint32_t)(nbox * 16384 + fbytes));
                    for (int b = 0; b < nbox; ++b)
                        tma_load_3d(base_ptr + stage * TB::value + b * 16384, &tmap, &full[stage],
                                    kc * kStageCols + b * TB::box_cols, (int)(ib * P.I_T), (int)(ot * P.O_T));
                    bulk_load(fchunk_ptr + stage * fbytes, P.Fc + (int64_t)kc * kStageCols * P.RP, (uint32_t)fbytes,
                              &full[stage]);
                    ++issued;
                    if (++stage == kStreamStages) { stage = 0; phase ^= 1u; }
                }
            }
            drain_stages(full, stage, phase, issued, P.err);
        }
        return;
    }

    // ------------------------------ consumers ------------------------------
    float acc[4][R];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int p = 0; p < R; ++p) acc[j][p] = 0.f;
    float macc[INNER ? R : 4];
#pragma unroll
    for (int p = 0; p < (INNER ? R : 4); ++p) macc[p] = 0.f;

    const uint32_t fchunk_base = smem_u32(fchunk_ptr);
    int stage = 0;
    uint32_t phase = 0;
    int64_t cur_ib = -1;
    int seg = 0;
    int tile_parity = 0;
    bool ok = true;
    const int kw = warp * 8;  // this warp's 8 columns inside a 64-column stage

    // A warp that gives up a bounded wait stops computing and stops arriving on
    // the ring, but keeps walking the tiles so that it still joins every named
    // barrier of the outer-mode epilogue: no barrier can hang.
    for (int64_t t = t_beg; t < t_end; ++t) {
        int64_t ib, ot;
        if (INNER) { ib = t / P.n_ot; ot = t % P.n_ot; }
        else { ot = t / P.nb; ib = t % P.nb; }
        if (INNER && ok && ib != cur_ib) {
            if (cur_ib >= 0) {
                // flush the finished inner block: lanes l, l+I_T, ... share row l % I_T
                for (int off = P.I_T; off < 32; off <<= 1) {
#pragma unroll
                    for (int p = 0; p < R; ++p) macc[p] += __shfl_xor_sync(0xffffffffu, macc[p], off);
                }
                if (lane < P.I_T) {
                    float* dst = P.part +
                                 ((((int64_t)g * P.Smax + seg) * kStreamWarps + warp) * P.I_T + lane) * P.RP + p0;
#pragma unroll
                    for (int p = 0; p < R; p += 4)
                        *reinterpret_cast<float4*>(dst + p) =
                            make_float4(macc[p], macc[p + 1], macc[p + 2], macc[p + 3]);
                }
#pragma unroll
                for (int p = 0; p < R; ++p) macc[p] = 0.f;
                ++seg;
            }
            cur_ib = ib;
        }
        for (int kc = 0; kc < P.n_kc; ++kc) {
            if (ok && !warp_wait_bounded(&full[stage], phase)) {
                if (lane == 0) record_device_error(P.err, kErrWaitFull);
                ok = false;
            }
            if (ok && (int64_t)kc * kStageCols + kw < P.C) {
                const uint32_t tb = base + stage * TB::value;
                const uint32_t fb = fchunk_base + stage * fbytes;
                if constexpr (sizeof(TE) == 4) {
                    const uint32_t box = tb + (kw >> 5) * 16384;
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        const int chunk = ((kw & 31) >> 2) + q;
                        float tv[4][4];
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const float4 v = lds128f(sw128(box, lane + 32 * j, chunk));
                            tv[j][0] = v.x; tv[j][1] = v.y; tv[j][2] = v.z; tv[j][3] = v.w;
                        }
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            const uint32_t frow = fb + (uint32_t)((kw + q * 4 + kk) * P.RP + p0) * 4u;
#pragma unroll
                            for (int p = 0; p < R; p += 4) {
                                const float4 f = lds128f(frow + p * 4);
#pragma unroll
                                for (int j = 0; j < 4; ++j) fma4(acc[j] + p, tv[j][kk], f);
                            }
                        }
                    }
                } else {
                    const int chunk = kw >> 3;  // 8 bf16 columns per 16-byte chunk
                    uint4 tw[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) tw[j] = lds128u(sw128(tb, lane + 32 * j, chunk));
#pragma unroll
                    for (int kk = 0; kk < 8; ++kk) {
                        float tv[4];
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const uint32_t wv = (kk >> 1) == 0 ? tw[j].x : (kk >> 1) == 1 ? tw[j].y
                                              : (kk >> 1) == 2 ? tw[j].z : tw[j].w;
                            tv[j] = (kk & 1) ? bf16_hi(wv) : bf16_lo(wv);
                        }
                        const uint32_t frow = fb + (uint32_t)((kw + kk) * P.RP + p0) * 4u;
#pragma unroll
                        for (int p = 0; p < R; p += 4) {
                            const float4 f = lds128f(frow + p * 4);
#pragma unroll
                            for (int j = 0; j < 4; ++j) fma4(acc[j] + p, tv[j], f);
                        }
                    }
                }
            }
            fence_proxy_async_smem();
            __syncwarp();
            if (ok && lane == 0) mbar_arrive(&empty[stage]);
            if (++stage == kStreamStages) { stage = 0; phase ^= 1u; }
        }
        // ---------------- tile epilogue ----------------
        if (INNER && ok) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int64_t o = ot * P.O_T + (lane + 32 * j) / P.I_T;
                if (o < P.n_o) {
                    const float* wr = P.W + o * P.RP + p0;
#pragma unroll
                    for (int p = 0; p < R; p += 4) {
                        const float4 w4 = __ldg(reinterpret_cast<const float4*>(wr + p));
                        macc[p + 0] = fmaf(w4.x, acc[j][p + 0], macc[p + 0]);
                        macc[p + 1] = fmaf(w4.y, acc[j][p + 1], macc[p + 1]);
                        macc[p + 2] = fmaf(w4.z, acc[j][p + 2], macc[p + 2]);
                        macc[p + 3] = fmaf(w4.w, acc[j][p + 3], macc[p + 3]);
                    }
                }
            }
        } else if (!INNER) {
            // one outer index per tile (I_T = 128, O_T = 1): z = sum_rows Y(row) A_{N-2}(i(row))
            float z[R];
#pragma unroll
            for (int p = 0; p < R; ++p) z[p] = 0.f;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int64_t i = ib * 128 + lane + 32 * j;
                if (i < P.Ii) {
                    const float* fr = P.Fi + i * P.RP + p0;
#pragma unroll
                    for (int p = 0; p < R; p += 4) {
                        const float4 f4 = __ldg(reinterpret_cast<const float4*>(fr + p));
                        z[p + 0] = fmaf(f4.x, acc[j][p + 0], z[p + 0]);
                        z[p + 1] = fmaf(f4.y, acc[j][p + 1], z[p + 1]);
                        z[p + 2] = fmaf(f4.z, acc[j][p + 2], z[p + 2]);
                        z[p + 3] = fmaf(f4.w, acc[j][p + 3], z[p + 3]);
                    }
                }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
                for (int p = 0; p < R; ++p) z[p] += __shfl_xor_sync(0xffffffffu, z[p], off);
            }
            float mine = 0.f;
#pragma unroll
            for (int p = 0; p < R; ++p)
                if (p == lane) mine = z[p];
            // sum the 8 warps' column sums in shared memory (buffer alternates by tile parity,
            // so one barrier per tile suffices) and write one partial per tile
            float* zs = zsum + (tile_parity * kStreamWarps) * 32;
            zs[warp * 32 + lane] = mine;
            named_bar_sync(1, kStreamWarps * 32);
            if (warp == 0 && lane < R && ok) {
                float t = 0.f;
#pragma unroll
                for (int w = 0; w < kStreamWarps; ++w) t += zs[w * 32 + lane];
                P.part[((ot * P.nb) + ib) * P.RP + p0 + lane] = t;
            }
            tile_parity ^= 1;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int p = 0; p < R; ++p) acc[j][p] = 0.f;
    }
    if (INNER && ok && cur_ib >= 0) {
        for (int off = P.I_T; off < 32; off <<= 1) {
#pragma unroll
            for (int p = 0; p < R; ++p) macc[p] += __shfl_xor_sync(0xffffffffu, macc[p], off);
        }
        if (lane < P.I_T) {
            float* dst =
                P.part + ((((int64_t)g * P.Smax + seg) * kStreamWarps + warp) * P.I_T + lane) * P.RP + p0;
#pragma unroll
            for (int p = 0; p < R; p += 4)
                *reinterpret_cast<float4*>(dst + p) = make_float4(macc[p], macc[p + 1], macc[p + 2], macc[p + 3]);
        }
    }
}

// ---------------------------------------------------------------------------
// last-mode kernel: M(c,p) = sum_rows T(row,c) KR(row,p); each CTA owns one
// 64-column block (blockIdx.y) and a contiguous range of tiles (blockIdx.x)
// ---------------------------------------------------------------------------
template <typename TE, int R>
__global__ void __launch_bounds__(kStreamThreads, 1)
    k_stream_last(const __grid_constant__ CUtensorMap tmap, const StreamParams P) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    using TB = TileBytes<TE>;
    constexpr int kKrBytes = kTileRows * R * 4;
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char* base_ptr = smem_raw + (base - raw);
    unsigned char* kr_ptr = base_ptr + kStreamStages * TB::value;
    uint64_t* full = reinterpret_cast<uint64_t*>(kr_ptr + kStreamStages * kKrBytes);
    uint64_t* empty = full + kStreamStages;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = blockIdx.x, G = gridDim.x;
    const int cb = blockIdx.y;
    const int p0 = blockIdx.z * R;
    int64_t t_beg, t_end;
    tile_range(P.n_tiles, g, G, t_beg, t_end);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStreamStages; ++s) {
            mbar_init(&full[s], 2);   // TMA arrival (with bytes) + "KR rows written" arrival
            mbar_init(&empty[s], kStreamWarps);
        }
        fence_mbar_init();
    }
    __syncthreads();
    pdl_wait();
    pdl_trigger();

    if (warp == kStreamWarps) {
        // ------------------------------ producer ------------------------------
        if (lane == 0) prefetch_tensormap(&tmap);
        int stage = 0;
        uint32_t phase = 0;
        int64_t issued = 0;
        for (int64_t t = t_beg; t < t_end; ++t) {
            const int64_t ib = t / P.n_ot, ot = t % P.n_ot;
            int good = 1;
            if (lane == 0) good = mbar_wait_bounded(&empty[stage], phase ^ 1u) ? 1 : 0;
            good = __shfl_sync(0xffffffffu, good, 0);
            if (!good) {
                if (lane == 0) record_device_error(P.err, kErrWaitEmpty);
                break;
            }
            if (lane == 0) {
                const int64_t left = P.C - (int64_t)cb * kStageCols;
                const int nbox = left >= kStageCols ? TB::boxes : (int)((left + TB::box_cols - 1) / TB::box_cols);
                mbar_arrive_expect_tx(&full[stage], (uint32_t)(nbox * 16384));
                for (int b = 0; b < nbox; ++b)
                    tma_load_3d(base_ptr + stage * TB::value + b * 16384, &tmap, &full[stage],
                                cb * kStageCols + b * TB::box_cols, (int)(ib * P.I_T), (int)(ot * P.O_T));
            }
            // Khatri-Rao rows of this tile: KR(m,p) = W(o,p) A_{N-2}(i,p), 0 outside the tensor
            float* kr = reinterpret_cast<float*>(kr_ptr + stage * kKrBytes);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int m = lane + 32 * q;
                const int64_t o = ot * P.O_T + m / P.I_T;
                const int64_t i = ib * P.I_T + m % P.I_T;
                const bool valid = (o < P.n_o) && (i < P.Ii);
#pragma unroll
                for (int p = 0; p < R; p += 4) {
                    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (valid) {
                        const float4 w4 = __ldg(reinterpret_cast<const float4*>(P.W + o * P.RP + p0 + p));
                        const float4 f4 = __ldg(reinterpret_cast<const float4*>(P.Fi + i * P.RP + p0 + p));
                        v = make_float4(w4.x * f4.x, w4.y * f4.y, w4.z * f4.z, w4.w * f4.w);
                    }
                    *reinterpret_cast<float4*>(kr + m * R + p) = v;
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&full[stage]);
            ++issued;
            if (++stage == kStreamStages) { stage = 0; phase ^= 1u; }
        }
        if (lane == 0) drain_stages(full, stage, phase, issued, P.err);
        return;
    }

    // ------------------------------ consumers ------------------------------
    const int c4 = lane & 15, h = lane >> 4;
    const bool col_live = (int64_t)cb * kStageCols + c4 * 4 < P.C;
    float acc[4][R];
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int p = 0; p < R; ++p) acc[c][p] = 0.f;

    const uint32_t kr_base = smem_u32(kr_ptr);
    int stage = 0;
    uint32_t phase = 0;
    for (int64_t t = t_beg; t < t_end; ++t) {
        if (!warp_wait_bounded(&full[stage], phase)) {
            if (lane == 0) record_device_error(P.err, kErrWaitFull);
            break;
        }
        if (col_live) {
            const uint32_t tb = base + stage * TB::value;
            const uint32_t kb = kr_base + stage * kKrBytes;
#pragma unroll 2
            for (int rr = 0; rr < 8; ++rr) {
                const int m = warp * 16 + rr * 2 + h;
                float tv[4];
                if constexpr (sizeof(TE) == 4) {
                    const float4 v = lds128f(sw128(tb + (c4 >> 3) * 16384, m, c4 & 7));
                    tv[0] = v.x; tv[1] = v.y; tv[2] = v.z; tv[3] = v.w;
                } else {
                    const uint2 v = lds64u(sw128(tb, m, c4 >> 1) + (c4 & 1) * 8);
                    tv[0] = bf16_lo(v.x); tv[1] = bf16_hi(v.x); tv[2] = bf16_lo(v.y); tv[3] = bf16_hi(v.y);
                }
                const uint32_t krow = kb + (uint32_t)(m * R) * 4u;
#pragma unroll
                for (int p = 0; p < R; p += 4) {
                    const float4 f = lds128f(krow + p * 4);
#pragma unroll
                    for (int c = 0; c < 4; ++c) fma4(acc[c] + p, tv[c], f);
                }
            }
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[stage]);
        if (++stage == kStreamStages) { stage = 0; phase ^= 1u; }
    }
    // the two half-warps hold the same columns
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int p = 0; p < R; ++p) acc[c][p] += __shfl_xor_sync(0xffffffffu, acc[c][p], 16);

    // Cross-warp sum through shared memory.  Every issued stage was waited
    // for above (or timed out, after which the result is discarded), so the
    // T stage area can be reused: 8 warps x 64 columns x R floats.
    named_bar_sync(1, kStreamWarps * 32);
    float* red = reinterpret_cast<float*>(base_ptr);
    if (h == 0) {
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int p = 0; p < R; p += 4)
                *reinterpret_cast<float4*>(red + ((warp * kStageCols) + c4 * 4 + c) * R + p) =
                    make_float4(acc[c][p], acc[c][p + 1], acc[c][p + 2], acc[c][p + 3]);
    }
    named_bar_sync(1, kStreamWarps * 32);
    for (int idx = threadIdx.x; idx < kStageCols * R; idx += kStreamWarps * 32) {
        const int col = idx / R, p = idx % R;
        const int64_t gcol = (int64_t)cb * kStageCols + col;
        if (gcol < P.C) {
            float s = 0.f;
#pragma unroll
            for (int w = 0; w < kStreamWarps; ++w) s += red[(w * kStageCols + col) * R + p];
            P.part[((int64_t)g * P.Cpad + gcol) * P.RP + p0 + p] = s;
        }
    }
}

#endif  // __CUDACC__

// per-dtype launchers (mttkrp_f32.cu / mttkrp_bf16.cu)
cudaError_t launch_stream_f32(int kind, int R, dim3 grid, size_t smem, cudaStream_t st, const CUtensorMap& map,
                              const StreamParams& P, bool pdl = false);
cudaError_t launch_stream_bf16(int kind, int R, dim3 grid, size_t smem, cudaStream_t st, const CUtensorMap& map,
                               const StreamParams& P, bool pdl = false);

}  // namespace ntf

#ifdef __CUDACC__
namespace ntf {

// kind: 0 = inner, 1 = outer, 2 = last.  R in {4, 8, 12, 16, 20, 24, 32}.
template <typename TE>
cudaError_t launch_stream_impl(int kind, int R, dim3 grid, size_t smem, cudaStream_t st, const CUtensorMap& map,
                               const StreamParams& P, bool pdl) {
    typedef void (*Kern)(const CUtensorMap, const StreamParams);
    Kern k = nullptr;
#define NTF_PICK(RR)                                                \
    case RR:                                                        \
        k = kind == 0 ? (Kern)k_stream_rows<TE, RR, true>           \
          : kind == 1 ? (Kern)k_stream_rows<TE, RR, false>          \
                      : (Kern)k_stream_last<TE, RR>;                \
        break;
    switch (R) {
        NTF_PICK(4) NTF_PICK(8) NTF_PICK(12) NTF_PICK(16) NTF_PICK(20) NTF_PICK(24) NTF_PICK(32)
        default: return cudaErrorInvalidValue;
    }
#undef NTF_PICK
    // opt in to > 48 KB of shared memory once per kernel and size (outside any graph capture:
    // the solver issues a zero-CTA configuration call before capturing)
    static size_t set_bytes[3][8] = {{0}};
    const int ri = R <= 24 ? R / 4 - 1 : 6;
    if (set_bytes[kind][ri] < smem) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        set_bytes[kind][ri] = smem;
    }
    if (grid.x == 0) return cudaSuccess;   // configuration only
    return launch_kernel(k, grid, dim3(kStreamThreads), smem, st, pdl, map, P);
}

}  // namespace ntf
#endif
