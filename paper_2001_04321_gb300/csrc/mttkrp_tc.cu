// Tensor-core (tcgen05, kind::f16) MTTKRP streaming kernels for bfloat16
// tensor storage (step a1; Sec. 2, def:B / def:grad: M_n = T_[n] B^n).
//
// The tensor tile is the A operand exactly as TMA lands it (128 rows x 64
// bf16 columns, 128-byte swizzle).  The other operand carries a factor split
// into bfloat16 high and low parts (x = hi + lo, |x - hi - lo| <= 2^-16 |x|),
// side by side along N, so one MMA gives T*hi and T*lo in FP32 and their sum
// is accurate to FP32 level while T itself is exact in bf16.
//
//   rows kernel (modes < N-1): D[row][p] = sum_k T[row][k] F[k][p], F = A_{N-1};
//       A = T tile (K-major), B = F chunk stored [p][k] (K-major), one TMEM
//       accumulator per 64-column chunk in a ring of four; 4 epilogue warps read
//       one row per thread and apply the inner / outer weighting of the FFMA kernels.
//   last kernel (mode N-1): per tile (one outer index o, 128 inner rows i)
//       D[c][p] = sum_i T[(o,i)][c] A_{N-2}[i][p]; A = T tile (MN-major: its
//       contiguous dimension is c), B = packed bf16 hi|lo rows of A_{N-2}
//       (K-major); the epilogue folds W(o,p) D[c][p] into FP32 registers.
//
// The tensor cores' FP32 accumulation is not round-to-nearest (measured: a
// consistent relative bias of about -8e-7 per accumulated MMA step), so no
// TMEM accumulator takes more than 8 MMA steps: the rows kernel starts a fresh
// accumulator for every 64-column chunk (4 steps), the last-mode kernel for
// every tile (8 steps), and the epilogue sums them in registers with IEEE FP32.
// The Khatri-Rao matrix is never formed: the last mode's weights W(o,:) enter
// in the epilogue, per tile.
//
// Warps: 0-3 epilogue / Khatri-Rao builders (TMEM lanes 0-127), 4 TMA
// producer, 5 MMA issuer (and TMEM owner).  Every wait is bounded.
#include "mttkrp_kernels.cuh"
#include "mttkrp_tc.cuh"

namespace ntf {
namespace {

constexpr int kTcThreads = 192;
constexpr int kTcStages = 4;        // last-mode kernel: stages of two boxes
constexpr int kRowStages = 4;       // rows kernel: stages of one box and one factor chunk
constexpr int kDbuf = 4;             // rows kernel: TMEM accumulators in flight (64 columns each)
constexpr int kRowCtasPerSm = kRowStages * kDbuf <= 16 ? 2 : 1;
// rows kernel: barriers (full, empty per stage; tfull, tempty per accumulator; drain; sfull,
// sempty per tile-ring slot) and the TMEM slot, then the tile ring of 4 records (80 bytes)
constexpr int kRowBarBytes = ((2 * kRowStages + 2 * kDbuf + 1 + 2 * 4) * 8 + 8 + 15) / 16 * 16;
constexpr int kRowMiscBytes = (kRowBarBytes + 128 + 255) / 256 * 256;
constexpr int kBoxBytes = 16384;   // 128 rows x 64 bf16

// ----------------------------------------------------------------------------
// tcgen05 / descriptor helpers
// ----------------------------------------------------------------------------
// Shared-memory matrix descriptor (SM100 UMMA): start address, leading and
// stride byte offsets (16-byte units), version 1, 128-byte swizzle.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr, uint32_t lbo_bytes, uint32_t sbo_bytes) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo_bytes >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo_bytes >> 4) & 0x3FFFu) << 32) | (1ull << 46) | (2ull << 61);
}

// Instruction descriptor, kind::f16: FP32 accumulate, A and B bf16.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, int a_mn_major, int b_mn_major) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn_major << 15) | ((uint32_t)b_mn_major << 16) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D (+)= A x B, both operands in shared memory, issued by one elected lane of a converged
// warp: the whole warp runs the issue loop, so descriptors and addresses stay warp-uniform
// (measured 2.6x faster per MMA than a loop run by one lane alone).
__device__ __forceinline__ void tc_mma_elect(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                             uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p, e;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// commit by the elected lane (the one that issued the MMAs it tracks)
__device__ __forceinline__ void tc_commit_elect(uint64_t* bar) {
    asm volatile(
        "{\n\t.reg .pred e;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}" ::"r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// 32 lanes x 32 bit, 16 consecutive columns per thread
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity) {
    const bool mine = mbar_wait_bounded(bar, parity);
    return __all_sync(0xffffffffu, mine) != 0;
}

// D columns [col0, col0 + 2*RPH) of this thread's TMEM lane -> y[p] = hi + lo
template <int RPH>
__device__ __forceinline__ void read_rows(uint32_t tmem_row, int col0, float (&y)[RPH]) {
    float d[2 * RPH];
#pragma unroll
    for (int c = 0; c < 2 * RPH; c += 16) {
        float v[16];
        tmem_ld16(tmem_row + col0 + c, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) d[c + i] = v[i];
    }
    tmem_wait_ld();
#pragma unroll
    for (int p = 0; p < RPH; ++p) y[p] = d[p] + d[RPH + p];
}

// ----------------------------------------------------------------------------
// rows kernel (inner / outer modes)
//
// Tiles are handed out at run time: the producer takes the next tile index
// from a device counter (reset before every launch), decodes it and passes the
// record to the other warp roles through a small ring guarded by its own pair
// of mbarriers.  Every tile writes its own output slot, so the result does not
// depend on which CTA took which tile, and CTAs that stream faster take more
// tiles (no tail of slow CTAs).
// ----------------------------------------------------------------------------
constexpr int kTileRing = 4;
static_assert(kTileRing == 4, "the rows kernels' barrier blocks hold 4 tile-ring slots");

// the statically assigned first tile of this CTA (-1 if there is none)
__device__ __forceinline__ int g_first_tile(int64_t n_tiles) {
    return (int64_t)blockIdx.x < n_tiles ? (int)blockIdx.x : -1;
}

// wait until the last min(issued, R) loads of a ring of R stages have landed
__device__ __forceinline__ void drain_ring(uint64_t* full, int R, int64_t issued, int* err) {
    const int64_t lo = issued > R ? issued - R : 0;
    for (int64_t i = issued - 1; i >= lo; --i)
        if (!mbar_wait_bounded(&full[i % R], (uint32_t)((i / R) & 1))) {
            record_device_error(err, kErrWaitDrain);
            break;
        }
}

// A scheduled tile as the producer decodes it, once, for every consumer warp: its slot t,
// its chunks [kc0, kc1), and its row block ib and outer block ot.  (Each warp role decoding
// the index itself with 64-bit divisions took thousands of cycles at every tile boundary, on
// the epilogue's critical path.)  Tile counts are below 2^31, so 32-bit arithmetic holds.
// Row tile tb has n_cs output slots, tb n_cs + cs for its column segments cs.  Scheduled units
// below n_whole are whole row tiles (tb = t; they write slot tb n_cs and zeros to the zext
// slots after it); the rest are single segments: unit n_whole + u is segment u % n_cs of row
// tile n_whole + u / n_cs.  Every slot is written once per launch, and the segments' partial
// sums meet only in the fixed-order reduction.  The inner mode numbers row tiles over the outer
// blocks first (tb = ib n_ot + ot), the outer modes over the row blocks first (tb = ot nb + ib).
// t is the output slot (-1: no more tiles).
struct TileRec {
    int t, kc0, kc1, ib, ot, zext;
};

template <bool INNER>
__device__ __forceinline__ TileRec decode_tile(const TcParams& P, int t) {
    TileRec r{t, 0, 0, 0, 0, 0};
    if (t < 0) return r;
    const unsigned int ncs = P.n_cs > 0 ? (unsigned int)P.n_cs : 1u;
    const int per = P.kc_per > 0 ? P.kc_per : P.n_kc;
    unsigned int tb;
    if ((int64_t)t < P.n_whole) {
        tb = (unsigned int)t;
        r.kc1 = P.n_kc;
        r.t = (int)(tb * ncs);
        r.zext = (int)ncs - 1;
    } else {
        const unsigned int u = (unsigned int)t - (unsigned int)P.n_whole;
        const unsigned int q = u / ncs, cs = u - q * ncs;
        tb = (unsigned int)P.n_whole + q;
        r.kc0 = (int)cs * per;
        r.kc1 = r.kc0 + per < P.n_kc ? r.kc0 + per : P.n_kc;
        r.t = (int)(tb * ncs + cs);
    }
    if (INNER) {
        const unsigned int n_ot = (unsigned int)P.n_ot;
        r.ib = (int)(tb / n_ot);
        r.ot = (int)(tb - (unsigned int)r.ib * n_ot);
    } else {
        const unsigned int nb = (unsigned int)P.nb;
        r.ot = (int)(tb / nb);
        r.ib = (int)(tb - (unsigned int)r.ot * nb);
    }
    return r;
}

// v = *p if pred, else 0, without a dependency on the loaded value at the load: the value is
// used only at the end of the tile, so the warp must not wait for it here (a select on the
// loaded value stalled the epilogue for an L2 round trip at every tile boundary)
__device__ __forceinline__ float ldg_or_zero(const float* ptr, bool pred) {
    float v;
    asm volatile(
        "{\n\t.reg .pred q;\n\t"
        "setp.ne.b32 q, %2, 0;\n\t"
        "mov.b32 %0, 0;\n\t"
        "@q ld.global.nc.f32 %0, [%1];\n\t}"
        : "=f"(v)
        : "l"(ptr), "r"((int)pred));
    return v;
}

// v = *ptr (four floats, 16-byte aligned) if pred, else 0, likewise without waiting for the value
__device__ __forceinline__ float4 ldg4_or_zero(const float* ptr, bool pred) {
    float4 v;
    asm volatile(
        "{\n\t.reg .pred q;\n\t"
        "setp.ne.b32 q, %5, 0;\n\t"
        "mov.b32 %0, 0;\n\tmov.b32 %1, 0;\n\tmov.b32 %2, 0;\n\tmov.b32 %3, 0;\n\t"
        "@q ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];\n\t}"
        : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
        : "l"(ptr), "r"((int)pred));
    return v;
}

// The epilogue warps' row weights for one tile (w[p] = 0 for dead rows and p >= r): inner mode
// W(o, :) of the row's outer index, outer modes the row's own weight row.  Each thread loads its
// row; where rows are 16-byte aligned, four columns per load (per-column loads from 128
// different rows kept the load unit busy for hundreds of cycles at every tile boundary).
template <int RPH, bool INNER>
__device__ __forceinline__ void tile_weights(const TcParams& P, const TileRec& tr, int m, int m_o, int m_i,
                                             const float* Wt, const float* Fit, float (&w)[RPH]) {
    bool row_live;
    const float* src;
    if (INNER) {
        const int64_t o = (int64_t)tr.ot * P.O_T + m_o;
        row_live = o < P.n_o && (int64_t)tr.ib * P.I_T + m_i < P.Ii;
        src = Wt + (row_live ? o : 0) * P.ldw;
    } else {
        const int64_t i = (int64_t)tr.ib * 128 + m;
        row_live = i < P.Ii;
        src = Fit + (row_live ? i : 0) * P.ldw;
    }
    if ((P.ldw & 3) == 0 && (P.r & 3) == 0 && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
#pragma unroll
        for (int j = 0; j < RPH / 4; ++j) {
            const float4 v = ldg4_or_zero(src + 4 * j, row_live && 4 * j < P.r);
            w[4 * j] = v.x;
            w[4 * j + 1] = v.y;
            w[4 * j + 2] = v.z;
            w[4 * j + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int p = 0; p < RPH; ++p) w[p] = ldg_or_zero(src + p, row_live && p < P.r);
    }
}

// The reducer warp of the 3xTF32 rows kernel.  For each tile, once the four epilogue warps have
// stored the tile's 128 weighted rows z (thread m = tile row m) in red and arrived on zfull, it
// forms the tile's output slot from them, then frees red (zfree).  Tile row m = a I_T + b
// (I_T = 1 in the outer modes): the slot holds, per entry (b, p), the sum over the tile's rows
// a, in order.  It runs off the tensor-core pipeline's critical path: done by the epilogue warps
// at the end of each tile (tile_flush), the reduction stalled the MMA warps for about 1300 cycles
// at every tile boundary.  (The bf16 kernel keeps tile_flush: with two CTAs per SM the other CTA
// covers its boundaries, and an eighth warp measured slower there.)  Every sum has a fixed order.
template <int RPH, bool INNER>
__device__ void tile_reducer(const TcParams& P, const TileRec* tile_ring, uint64_t* sfull, uint64_t* sempty,
                             uint64_t* zfull, uint64_t* zfree, const int* zok, const float* red, int lane) {
    const int IT = INNER ? P.I_T : 1;
    int q = 0;                                       // tiles reduced
    for (int64_t s = 0;; ++s) {
        const int slot = (int)(s % kTileRing);
        if (!warp_wait(&sfull[slot], (uint32_t)((s / kTileRing) & 1))) {
            if (lane == 0) record_device_error(P.err, kErrWaitFull);
            break;
        }
        const TileRec tr = tile_ring[slot];
        __syncwarp();
        if (lane == 0) mbar_arrive(&sempty[slot]);
        if (tr.t < 0) break;
        if (!warp_wait(zfull, (uint32_t)(q & 1))) {
            if (lane == 0) record_device_error(P.err, kErrWaitFull);
            break;
        }
        const bool write = zok[0] && zok[1] && zok[2] && zok[3];
        if (IT == 1) {
            // all 128 rows in one output row: lane p sums column p, rows in order, 4 running sums
            const int p = lane;
            if (p < P.r) {
                float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll 8
                for (int m = 0; m < 128; m += 4) {
                    s0 += red[(m + 0) * RPH + p];
                    s1 += red[(m + 1) * RPH + p];
                    s2 += red[(m + 2) * RPH + p];
                    s3 += red[(m + 3) * RPH + p];
                }
                if (write) {
                    P.part[(int64_t)tr.t * P.RP + p] = (s0 + s1) + (s2 + s3);
                    for (int k = 1; k <= tr.zext; ++k) P.part[(int64_t)(tr.t + k) * P.RP + p] = 0.f;
                }
            }
        } else {
            // entries (b, p), 32 at a time: rows a I_T + b in order, two running sums
            const int n = IT * P.r, OT = 128 / IT;   // O_T I_T = 128, O_T even
            for (int idx = lane; idx < n; idx += 32) {
                const int b = idx / P.r, p = idx - b * P.r;
                const float* col = red + b * RPH + p;
                const int stride = IT * RPH;
                float s0 = 0.f, s1 = 0.f;
                for (int a = 0; a < OT; a += 2) {
                    s0 += col[a * stride];
                    s1 += col[(a + 1) * stride];
                }
                if (write) {
                    P.part[((int64_t)tr.t * IT + b) * P.RP + p] = s0 + s1;
                    for (int k = 1; k <= tr.zext; ++k) P.part[((int64_t)(tr.t + k) * IT + b) * P.RP + p] = 0.f;
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(zfree);
        ++q;
    }
}

// The epilogue warps' side of the hand-over: wait until the reducer has read the previous tile's
// rows (zfree), store this tile's weighted rows z (thread m = tile row m) and arrive on zfull.
template <int RPH>
__device__ __forceinline__ void tile_handover(const float (&z)[RPH], float* red, int m, int warp, int lane, int q,
                                              bool& ok, uint64_t* zfull, uint64_t* zfree, int* zok, int* err) {
    static_assert(RPH % 4 == 0, "rows of red are float4 groups");
    if (q > 0 && !warp_wait(zfree, (uint32_t)((q - 1) & 1))) {
        if (lane == 0) record_device_error(err, kErrWaitEmpty);
        ok = false;
    }
    float4* dst = reinterpret_cast<float4*>(red + m * RPH);
#pragma unroll
    for (int j = 0; j < RPH / 4; ++j) dst[j] = make_float4(z[4 * j], z[4 * j + 1], z[4 * j + 2], z[4 * j + 3]);
    if (lane == 0) zok[warp] = ok ? 1 : 0;
    __syncwarp();
    if (lane == 0) mbar_arrive(zfull);
}

// A finished tile's output slot from its weighted row sums z (thread m = tile row m), in a
// fixed order.  The four epilogue warps call this together (it holds named barrier 1); red is
// 128 x RPH floats of shared memory.  Every row goes to red first.  Tile row m = a I_T + b:
//   all 128 rows in one output row (outer modes, and the inner mode when I_T = 1): 4 threads
//     per column p each sum 32 rows (rows 4 i + q) and combine by two shuffles;
//   inner mode, I_T > 1: rows with equal b share inner row b of block ib, so the slot holds, per
//     entry (b, p), the sum over the tile's O_T outer indices a: one thread per entry, rows a in
//     order, even and odd a in two running sums.
// (Butterflies across the lanes took 1600 to 2300 cycles at each tile boundary, during which
// the tensor-core pipeline stalled.)
template <int RPH, bool INNER>
__device__ __forceinline__ void tile_flush(const TcParams& P, float (&z)[RPH], int t, int zext, bool write, int warp,
                                           int lane, int m, float* red) {
    static_assert(RPH % 4 == 0 && RPH <= 32, "rows of red are float4 groups; columns fit in 4 x 8 threads");
    named_bar_sync(1, 128);                      // the previous tile's readers are done with red
    float4* dst = reinterpret_cast<float4*>(red + m * RPH);
#pragma unroll
    for (int j = 0; j < RPH / 4; ++j) dst[j] = make_float4(z[4 * j], z[4 * j + 1], z[4 * j + 2], z[4 * j + 3]);
    named_bar_sync(1, 128);
    if (INNER && P.I_T > 1) {
        if (!write) return;
        // entries idx = b r + p for idx = m, m + 128, ...: (b, p) stepped without divisions
        const int IT = P.I_T, OT = 128 / P.I_T;      // O_T I_T = 128, O_T even
        const int n = IT * P.r;
        const int db = 128 / P.r, dp = 128 - db * P.r;
        int b = m / P.r, p = m - b * P.r;
        for (int idx = m; idx < n; idx += 128) {
            float s0 = 0.f, s1 = 0.f;
            const float* col = red + b * RPH + p;
            for (int a = 0; a < OT; a += 2) {
                s0 += col[(a * IT) * RPH];
                s1 += col[((a + 1) * IT) * RPH];
            }
            P.part[((int64_t)t * IT + b) * P.RP + p] = s0 + s1;
            for (int k = 1; k <= zext; ++k) P.part[((int64_t)(t + k) * IT + b) * P.RP + p] = 0.f;
            b += db;
            p += dp;
            if (p >= P.r) {
                p -= P.r;
                ++b;
            }
        }
    } else {
        // column p = 8 warp + lane % 8, quarter q = lane / 8: rows 4 i + q, two running sums;
        // the slot index t I_T + 0 = t also holds for the inner mode with I_T = 1
        const int q = lane >> 3, p = warp * 8 + (lane & 7);
        float s0 = 0.f, s1 = 0.f;
        if (p < P.r) {
#pragma unroll 8
            for (int i = 0; i < 32; i += 2) {
                s0 += red[(4 * i + q) * RPH + p];
                s1 += red[(4 * i + 4 + q) * RPH + p];
            }
        }
        float sum = s0 + s1;
        sum += __shfl_xor_sync(0xffffffffu, sum, 8);
        sum += __shfl_xor_sync(0xffffffffu, sum, 16);
        if (q == 0 && p < P.r && write) {
            P.part[(int64_t)t * P.RP + p] = sum;
            for (int k = 1; k <= zext; ++k) P.part[(int64_t)(t + k) * P.RP + p] = 0.f;
        }
    }
}

template <int RPH, bool INNER>
__global__ void __launch_bounds__(kTcThreads, kRowCtasPerSm) k_tc_rows(const __grid_constant__ CUtensorMap tmap, const TcParams P) {
    constexpr int N = 2 * RPH;
    constexpr int kB = N * 128;                 // factor chunk: N rows x 64 bf16 (swizzled)
    constexpr int kStage = kBoxBytes + kB;      // multiple of 1024 (N multiple of 16)
    constexpr uint32_t kIdesc = idesc_bf16(128, N, 0, 0);
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char* base_ptr = smem_raw + (base - raw);
    uint64_t* full = reinterpret_cast<uint64_t*>(base_ptr + kRowStages * kStage);
    uint64_t* empty = full + kRowStages;
    uint64_t* tfull = empty + kRowStages;        // [kDbuf]: accumulator of one 64-column chunk ready
    uint64_t* tempty = tfull + kDbuf;           // [kDbuf]: accumulator read by the epilogue
    uint64_t* drain = tempty + kDbuf;
    uint64_t* sfull = drain + 1;                // [kTileRing]: tile index published
    uint64_t* sempty = sfull + kTileRing;       // [kTileRing]: tile index read by all consumers
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sempty + kTileRing);
    TileRec* tile_ring = reinterpret_cast<TileRec*>(base_ptr + kRowStages * kStage + kRowBarBytes);   // [kTileRing]
    float* red = reinterpret_cast<float*>(base_ptr + kRowStages * kStage + kRowMiscBytes);   // [128][RPH]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kRowStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < kDbuf; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 4);
        }
        mbar_init(drain, 1);
        for (int k = 0; k < kTileRing; ++k) {
            mbar_init(&sfull[k], 1);
            mbar_init(&sempty[k], 5);           // the MMA thread and the 4 epilogue warps
        }
        fence_mbar_init();
    }
    if (warp == 5) tmem_alloc(tmem_slot, 64 * kDbuf);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    // CTA g's first tile is tile g; the tensor is never written, so its first chunks can
    // be in flight while the kernel before this one finishes (the packed factor chunks,
    // which that kernel writes, follow after the wait)
    const int first_tile = g_first_tile(P.n_tiles);
    const TileRec ft = decode_tile<INNER>(P, first_tile);
    const int npre = first_tile >= 0 ? (ft.kc1 - ft.kc0 < kRowStages ? ft.kc1 - ft.kc0 : kRowStages) : 0;
    if (warp == 4 && lane == 0) {
        prefetch_tensormap(&tmap);
        for (int j = 0; j < npre; ++j) {
            mbar_arrive_expect_tx(&full[j], (uint32_t)kStage);
            tma_load_3d(base_ptr + j * kStage, &tmap, &full[j], (ft.kc0 + j) * 64, ft.ib * P.I_T, ft.ot * P.O_T);
        }
    }
    // With P.early the producer and MMA warps do not wait for the kernel before this one and
    // may trigger the launch of the kernel after it while that one still runs; the host sets
    // early only where the kernel before writes nothing that this stream or the following
    // epilogue reads before its own wait (Solver::early_stream_ok).
    if (!P.early || warp < 4) pdl_wait();
    pdl_trigger();

    if (warp == 4) {
        // ------------------------- scheduler + producer -------------------------
        if (lane == 0) {
            const unsigned char* FcT = P.cur ? P.FcTb[__ldcg(P.cur + P.fct_sel)] : P.FcT;
            int stage = 0;
            uint32_t phase = 0;
            int64_t issued = 0;
            for (int64_t s = 0;; ++s) {
                const int slot = (int)(s % kTileRing);
                if (!mbar_wait_bounded(&sempty[slot], (uint32_t)((s / kTileRing) & 1) ^ 1u)) {
                    record_device_error(P.err, kErrWaitEmpty);
                    break;
                }
                int t = first_tile;
                if (s > 0) {
                    // tiles G, G+1, ... go to whichever CTA asks first
                    const unsigned int grab = atomicAdd(P.sched, 1u) + (unsigned int)gridDim.x;
                    t = grab < (unsigned int)P.n_tiles ? (int)grab : -1;
                }
                const TileRec tr = s == 0 ? ft : decode_tile<INNER>(P, t);
                tile_ring[slot] = tr;
                mbar_arrive(&sfull[slot]);              // releases the slot to the consumers
                if (t < 0) break;
                const int kc0 = tr.kc0, kc1 = tr.kc1;
                bool ok = true;
                for (int kc = kc0; kc < kc1; ++kc) {
                    unsigned char* st = base_ptr + stage * kStage;
                    if (s == 0 && kc - kc0 < npre) {
                        // stage kc already holds (or is receiving) this chunk of the tensor
                        bulk_load(st + kBoxBytes, FcT + (int64_t)kc * kB, (uint32_t)kB, &full[stage]);
                    } else {
                        if (!mbar_wait_bounded(&empty[stage], phase ^ 1u)) {
                            record_device_error(P.err, kErrWaitEmpty);
                            ok = false;
                            break;
                        }
                        mbar_arrive_expect_tx(&full[stage], (uint32_t)kStage);
                        tma_load_3d(st, &tmap, &full[stage], kc * 64, tr.ib * P.I_T, tr.ot * P.O_T);
                        bulk_load(st + kBoxBytes, FcT + (int64_t)kc * kB, (uint32_t)kB, &full[stage]);
                    }
                    ++issued;
                    if (++stage == kRowStages) { stage = 0; phase ^= 1u; }
                }
                if (!ok) break;
            }
            drain_ring(full, kRowStages, issued, P.err);
        }
        return;
    }

    if (warp == 5) {
        // ------------------------------ MMA issuer ------------------------------
        // the whole warp runs the loop; one elected lane issues the MMAs and commits
        int stage = 0;
        uint32_t phase = 0;
        int64_t gq = 0;   // accumulator (chunk) counter of this CTA
        bool ok = true;
        for (int64_t s = 0; ok; ++s) {
            const int slot = (int)(s % kTileRing);
            if (!warp_wait(&sfull[slot], (uint32_t)((s / kTileRing) & 1))) {
                if (lane == 0) record_device_error(P.err, kErrWaitFull);
                break;
            }
            const TileRec tr = tile_ring[slot];
            __syncwarp();
            if (lane == 0) mbar_arrive(&sempty[slot]);
            if (tr.t < 0) break;
            for (int kc = tr.kc0; kc < tr.kc1; ++kc, ++gq) {
                const int d = (int)(gq % kDbuf);
                if (!warp_wait(&tempty[d], (uint32_t)((gq / kDbuf) & 1) ^ 1u) || !warp_wait(&full[stage], phase)) {
                    if (lane == 0) record_device_error(P.err, kErrWaitFull);
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t a0 = base + stage * kStage;
                const uint32_t b0 = a0 + kBoxBytes;
                const uint32_t dt = tmem + (uint32_t)(d * 64);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    tc_mma_elect(dt, smem_desc_sw128(a0 + kk * 32, 16, 1024), smem_desc_sw128(b0 + kk * 32, 16, 1024),
                                 kIdesc, kk > 0 ? 1u : 0u);
                tc_commit_elect(&empty[stage]);          // frees the stage once these MMAs have read it
                tc_commit_elect(&tfull[d]);              // this chunk's accumulator is complete
                if (++stage == kRowStages) { stage = 0; phase ^= 1u; }
            }
        }
        // make sure nothing is still running on the tensor cores before TMEM is freed
        tc_commit_elect(drain);
        if (!warp_wait(drain, 0) && lane == 0) record_device_error(P.err, kErrWaitDrain);
        __syncwarp();
        named_bar_sync(2, 160);
        tc_fence_after();
        tmem_dealloc(tmem, 64 * kDbuf);
        return;
    }

    // ------------------------------ epilogue (warps 0-3) ------------------------------
    // before the first accumulator is ready: this CTA's share of the Grams and V for the
    // epilogue that follows the stream
    gram_job_run(P.job, (int)blockIdx.x * 4 + warp, (int)gridDim.x * 4);
    const float* Wt = P.cur ? P.Wb[__ldcg(P.cur + P.w_sel) ^ P.w_flip] : P.W;
    const float* Fit = P.cur ? P.Fib[__ldcg(P.cur + P.fi_sel) ^ P.fi_flip] : P.Fi;
    const int m = threadIdx.x;                       // tile row = TMEM lane
    const int m_o = m / P.I_T, m_i = m - m_o * P.I_T;   // inner mode: row m = (outer m_o, inner m_i)
    const uint32_t tmem_row = tmem + ((uint32_t)(warp * 32) << 16);
    bool ok = true;
    int64_t gq = 0;
    for (int64_t s = 0; ok; ++s) {
        const int slot = (int)(s % kTileRing);
        if (!warp_wait(&sfull[slot], (uint32_t)((s / kTileRing) & 1))) {
            if (lane == 0) record_device_error(P.err, kErrWaitFull);
            break;
        }
        const TileRec tr = tile_ring[slot];
        __syncwarp();
        if (lane == 0) mbar_arrive(&sempty[slot]);
        if (tr.t < 0) break;
        const int kc0 = tr.kc0, kc1 = tr.kc1;
        // this row's weights, fetched while the tile is being contracted
        float w[RPH];
        tile_weights<RPH, INNER>(P, tr, m, m_o, m_i, Wt, Fit, w);
        // Y(row) = sum over the tile's 64-column chunks of the chunk accumulators (IEEE FP32 adds)
        float y[RPH];
#pragma unroll
        for (int p = 0; p < RPH; ++p) y[p] = 0.f;
        for (int kc = kc0; kc < kc1; ++kc, ++gq) {
            const int d = (int)(gq % kDbuf);
            if (ok && !warp_wait(&tfull[d], (uint32_t)((gq / kDbuf) & 1))) {
                if (lane == 0) record_device_error(P.err, kErrWaitFull);
                ok = false;
            }
            if (ok) {
                tc_fence_after();
                float yc[RPH];
                read_rows<RPH>(tmem_row, d * 64, yc);
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&tempty[d]);
#pragma unroll
                for (int p = 0; p < RPH; ++p) y[p] += yc[p];
            }
        }
        float z[RPH];
#pragma unroll
        for (int p = 0; p < RPH; ++p) z[p] = w[p] * y[p];
        tile_flush<RPH, INNER>(P, z, tr.t, tr.zext, ok, warp, lane, m, red);
    }
    tc_fence_before();
    named_bar_sync(2, 160);
}

// ----------------------------------------------------------------------------
// last-mode kernel
//   M(c,p) = sum_o W(o,p) * sum_i T((o,i),c) A_{N-2}(i,p)
// A tile is one outer index o and 128 inner rows i of one 128-column block;
// the inner sum is one MMA chain (A = T tile, MN-major; B = the packed bf16
// hi|lo block of A_{N-2} for those rows, K-major), and the epilogue folds
// W(o,:) times each tile's accumulator into FP32 registers.
// ----------------------------------------------------------------------------
template <int RPH>
__global__ void __launch_bounds__(kTcThreads, 1) k_tc_last(const __grid_constant__ CUtensorMap tmap, const TcParams P) {
    constexpr int N = 2 * RPH;
    constexpr int kT = 2 * kBoxBytes;          // 128 rows x 128 columns (two 64-column boxes)
    constexpr int kB = 2 * N * 128;            // A_{N-2} block: 2 K-atoms x N rows x 128 B
    constexpr int kStage = kT + kB;
    constexpr int kLastDbuf = 4;
    constexpr uint32_t kIdesc = idesc_bf16(128, N, 1, 0);
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char* base_ptr = smem_raw + (base - raw);
    uint64_t* full = reinterpret_cast<uint64_t*>(base_ptr + kTcStages * kStage);
    uint64_t* empty = full + kTcStages;
    uint64_t* tfull = empty + kTcStages;        // [kLastDbuf]
    uint64_t* tempty = tfull + kLastDbuf;       // [kLastDbuf]
    uint64_t* drain = tempty + kLastDbuf;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = blockIdx.x, G = gridDim.x;
    const int cb = blockIdx.y;
    int64_t t_beg, t_end;
    tile_range(P.n_tiles, g, G, t_beg, t_end);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kTcStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < kLastDbuf; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 4);
        }
        mbar_init(drain, 1);
        fence_mbar_init();
    }
    if (warp == 5) tmem_alloc(tmem_slot, 64 * kLastDbuf);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    // the first tiles of this CTA's range: the tensor is never written, so their boxes
    // can be in flight while the kernel before this one finishes (the packed A_{N-2}
    // blocks, which that kernel writes, follow after the wait)
    const int64_t left = P.C - (int64_t)cb * 128;
    const int nbox = left > 64 ? 2 : 1;
    const int npre = (int)(t_end - t_beg < kTcStages ? t_end - t_beg : kTcStages);
    if (warp == 4 && lane == 0) {
        prefetch_tensormap(&tmap);
        for (int q = 0; q < npre; ++q) {
            const int64_t t = t_beg + q;
            const int64_t ib = t / P.n_ot, o = t % P.n_ot;   // I_T = 128, O_T = 1
            mbar_arrive_expect_tx(&full[q], (uint32_t)(nbox * kBoxBytes + kB));
            for (int b = 0; b < nbox; ++b)
                tma_load_3d(base_ptr + q * kStage + b * kBoxBytes, &tmap, &full[q], cb * 128 + b * 64, (int)(ib * 128),
                            (int)o);
        }
    }
    pdl_wait();
    pdl_trigger();

    if (warp == 4) {
        if (lane == 0) {
            const unsigned char* FcT = P.cur ? P.FcTb[__ldcg(P.cur + P.fct_sel)] : P.FcT;
            int stage = 0;
            uint32_t phase = 0;
            int64_t issued = 0;
            for (int64_t t = t_beg; t < t_end; ++t) {
                const int64_t ib = t / P.n_ot, o = t % P.n_ot;   // I_T = 128, O_T = 1
                unsigned char* st = base_ptr + stage * kStage;
                if (issued < npre) {
                    // stage `issued` already receives this tile's boxes
                    bulk_load(st + kT, FcT + ib * kB, (uint32_t)kB, &full[stage]);
                } else {
                    if (!mbar_wait_bounded(&empty[stage], phase ^ 1u)) {
                        record_device_error(P.err, kErrWaitEmpty);
                        break;
                    }
                    mbar_arrive_expect_tx(&full[stage], (uint32_t)(nbox * kBoxBytes + kB));
                    for (int b = 0; b < nbox; ++b)
                        tma_load_3d(st + b * kBoxBytes, &tmap, &full[stage], cb * 128 + b * 64, (int)(ib * 128),
                                    (int)o);
                    bulk_load(st + kT, FcT + ib * kB, (uint32_t)kB, &full[stage]);
                }
                ++issued;
                if (++stage == kTcStages) { stage = 0; phase ^= 1u; }
            }
            drain_stages(full, stage, phase, issued, P.err);
        }
        return;
    }

    if (warp == 5) {
        // the whole warp runs the loop; one elected lane issues the MMAs and commits
        int stage = 0;
        uint32_t phase = 0;
        int64_t tl = 0;
        for (int64_t t = t_beg; t < t_end; ++t, ++tl) {
            const int d = (int)(tl % kLastDbuf);
            if (!warp_wait(&tempty[d], (uint32_t)((tl / kLastDbuf) & 1) ^ 1u) || !warp_wait(&full[stage], phase)) {
                if (lane == 0) record_device_error(P.err, kErrWaitFull);
                break;
            }
            tc_fence_after();
            const uint32_t a0 = base + stage * kStage;
            const uint32_t b0 = a0 + kT;
            const uint32_t dt = tmem + (uint32_t)(d * 64);
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
                // A: 16 tile rows (two 8-row groups 1024 B apart), 128 columns in two
                // 64-column blocks 16 KB apart; B: K-atom kk/4, 32-byte step kk%4
                const uint64_t ad = smem_desc_sw128(a0 + kk * 2048, kBoxBytes, 1024);
                const uint64_t bd = smem_desc_sw128(b0 + (kk >> 2) * (N * 128) + (kk & 3) * 32, 16, 1024);
                tc_mma_elect(dt, ad, bd, kIdesc, kk > 0 ? 1u : 0u);
            }
            tc_commit_elect(&empty[stage]);
            tc_commit_elect(&tfull[d]);
            if (++stage == kTcStages) { stage = 0; phase ^= 1u; }
        }
        tc_commit_elect(drain);
        if (!warp_wait(drain, 0) && lane == 0) record_device_error(P.err, kErrWaitDrain);
        __syncwarp();
        named_bar_sync(2, 160);
        tc_fence_after();
        tmem_dealloc(tmem, 64 * kLastDbuf);
        return;
    }

    // ---------------- warps 0-3: fold W(o,:) x tile accumulator into registers ----------------
    // first, this CTA's share of the Grams and V for the epilogue that follows the stream
    gram_job_run(P.job, ((int)blockIdx.y * (int)gridDim.x + (int)blockIdx.x) * 4 + warp,
                 (int)(gridDim.x * gridDim.y) * 4);
    const float* Wt = P.cur ? P.Wb[__ldcg(P.cur + P.w_sel) ^ P.w_flip] : P.W;
    const int m = threadIdx.x;
    const uint32_t tmem_row = tmem + ((uint32_t)(warp * 32) << 16);
    bool ok = true;
    float acc[RPH];
#pragma unroll
    for (int p = 0; p < RPH; ++p) acc[p] = 0.f;
    int64_t tl = 0;
    for (int64_t t = t_beg; t < t_end; ++t, ++tl) {
        const int64_t o = t % P.n_ot;
        float w[RPH];
        const float* wr = Wt + o * P.ldw;
#pragma unroll
        for (int p = 0; p < RPH; ++p) w[p] = p < P.r ? __ldg(wr + p) : 0.f;
        const int d = (int)(tl % kLastDbuf);
        if (ok && !warp_wait(&tfull[d], (uint32_t)((tl / kLastDbuf) & 1))) {
            if (lane == 0) record_device_error(P.err, kErrWaitFull);
            ok = false;
        }
        if (ok) {
            tc_fence_after();
            float y[RPH];
            read_rows<RPH>(tmem_row, d * 64, y);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[d]);
#pragma unroll
            for (int p = 0; p < RPH; ++p) acc[p] = fmaf(w[p], y[p], acc[p]);
        }
    }
    // row m of the result = column cb*128 + m of M_{N-1}
    const int64_t c = (int64_t)cb * 128 + m;
    if (ok && c < P.C) {
        float* dst = P.part + ((int64_t)g * P.Cpad + c) * P.RP;
#pragma unroll
        for (int p = 0; p < RPH; ++p)
            if (p < P.r) dst[p] = acc[p];
    }
    tc_fence_before();
    named_bar_sync(2, 160);
}

// ----------------------------------------------------------------------------
// TF32 rows kernel: FP32 tensor storage, modes < N-1 (step a1 for the FP32 form)
//
// The tensor core reads TF32 (10 explicit mantissa bits), so both operands are
// split: T ~ T_hi + T_lo with T_hi = tf32(T) and T_lo = tf32(T - T_hi), both rounded to
// nearest (the tensor core would otherwise truncate the remainder), F likewise.  Per
// 32-column chunk the MMAs take T_hi [F_hi | F_lo] and T_lo [F_hi | F_lo] (8 steps,
// N = 2 RPH: at M = 128 the shape wants N a multiple of 16) into one accumulator (see
// kTfAccCols); the rounded remainders leave an error of about 2^-22 relative per product.
//
// The split tensor never goes back to shared memory.  Four converter warps read each
// landed box (one row per thread), release the box at once, and write T_hi | T_lo into
// one of four tensor-memory A slots; the MMAs take A from tensor memory and B (the packed
// factor chunk) from a ring of its own.  Shared memory carries each tensor byte twice
// (the TMA write and the converter's read), and eight boxes are in flight.
//
// Warps of the rows kernel: 0-3 epilogue (as in k_tc_rows, but they hand each tile's
// weighted rows to the reducer), 4 scheduler + TMA producer, 5 MMA issuer and TMEM owner,
// 6-13 converters (two groups of four), 14 second MMA issuer, 15 factor-chunk producer, 16
// tile reducer.  One CTA per SM; 512 TMEM columns (four 64-column accumulators, then four A
// slots).  The last-mode kernel has the first sixteen.
// ----------------------------------------------------------------------------
constexpr int kTfThreads = 512;       // last-mode kernel
constexpr int kTfConvGroups = 2;       // converter groups of 4 warps (6-9, 10-13), taking chunks in turn
constexpr int kTfMmaWarp2 = 14;        // second MMA warp (the first is warp 5); the two take chunks in turn
constexpr int kTfBWarp = 15;           // factor-chunk producer
constexpr int kTfRaw = 8;              // tensor boxes in flight
constexpr int kTfB = 8;                // factor chunks in flight (a producer warp of their own, so
                                       // that the boxes run ahead of the MMAs by the whole box ring)
constexpr int kTfA = 4;                // tensor-memory A slots of 64 columns (T_hi | T_lo)
// Accumulators: the tensor core's FP32 accumulation drops about half a unit in the last place
// (toward zero) whenever it adds into a large running sum, measured as a bias of -3e-8 per
// such add.  Taking T_hi's steps first and T_lo's after gave -2.3e-7 in every result; T_lo's
// four K steps first (their sum stays small), then T_hi's on top, gives -6e-8.
constexpr int kTfDbuf = 4;             // chunks whose accumulators are in flight
constexpr int kTfAccCols = 64;         // one 64-column accumulator per chunk
constexpr int kTfBox = 16384;          // 128 rows x 32 fp32
constexpr int kTfBars = 640;           // barrier block (52 barriers, TMEM slot, status words, tile ring of 4 records)
constexpr uint32_t kTfAcol = kTfAccCols * kTfDbuf;
constexpr uint32_t kTfCols = 512;

// Instruction descriptor, kind::tf32: FP32 accumulate, A and B TF32, both K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D (+)= A x B with A (M x 8, one TF32 per 32-bit column, row m in lane m) in tensor memory,
// issued by one elected lane of a converged warp.  The whole warp runs the issue
// loop, so its descriptors and addresses stay warp-uniform; a loop run by one lane alone
// was measured at about 1.6x the time per MMA.
__device__ __forceinline__ void tc_mma_tf32_ts_elect(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc,
                                                     uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p, e;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}


// 32 lanes x 32 bit, 32 consecutive columns per thread
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
        "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]),
        "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]),
        "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
        : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// The rows kernel tells the three consumers of a chunk's operands and result with one commit
// per chunk (done[g % 8]): the epilogue (accumulator ready), the converter group of chunk g + 4
// (A slot free) and the factor-chunk producer of chunk g + 8 (factor slot free).  Each waits
// on the phase of its own chunk before that barrier can complete the next one: chunk g + 8
// needs the accumulator of chunk g + 4 released (the epilogue reads in order), its A slot
// written by the converters after chunk g + 4, and its factor chunk loaded, so no waiter sees
// a phase twice removed.
constexpr int kTrThreads = 544;
constexpr int kTrReducerWarp = 16;     // tile reducer
constexpr int kTrMmaWarps = 2;
constexpr int kTrDone = 8;             // done barriers: lcm of the accumulator / A (4) and factor (8) rings
constexpr int kTrBWarp = 15;           // factor-chunk producer

// D (+)= A x B (A in tensor memory) by the lane whose predicate `leader` is set (elected once
// per warp, so every MMA and the commit that tracks it come from the same thread)
__device__ __forceinline__ void tc_mma_tf32_ts_lead(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc,
                                                    uint32_t idesc, uint32_t accumulate, uint32_t leader) {
    asm volatile(
        "{\n\t.reg .pred p, e;\n\t"
        "setp.ne.b32 e, %5, 0;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate), "r"(leader)
        : "memory");
}

__device__ __forceinline__ void tc_commit_lead(uint64_t* bar, uint32_t leader) {
    asm volatile(
        "{\n\t.reg .pred e;\n\t"
        "setp.ne.b32 e, %1, 0;\n\t"
        "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}" ::"r"(smem_u32(bar)),
        "r"(leader)
        : "memory");
}

__device__ __forceinline__ uint32_t elect_leader() {
    uint32_t e;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "elect.sync _|p, 0xffffffff;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(e));
    return e;
}

// 32 lanes x 32 bit, 8 consecutive columns per thread
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// y[p] += D[col0 + p] + D[col0 + RPH + p]: the hi and lo halves of one accumulator, read 16 (or
// 8) columns of each at a time so that no more than 32 loaded values are live
template <int RPH>
__device__ __forceinline__ void add_rows(uint32_t tmem_row, int col0, float (&y)[RPH]) {
    // (at 32 columns 8 at a time: with the row weights and the sums live, 16 at a time would not
    // fit the 96 registers that the kernel's 17 warps leave each thread)
    constexpr int kStep = RPH >= 32 ? 8 : 16;
#pragma unroll
    for (int c = 0; c < RPH; c += kStep) {
        if (kStep == 16 && RPH - c >= 16) {
            float h[16], l[16];
            tmem_ld16(tmem_row + col0 + c, h);
            tmem_ld16(tmem_row + col0 + RPH + c, l);
            tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < 16; ++i) y[c + i] += h[i] + l[i];
        } else {
            float h[8], l[8];
            tmem_ld8(tmem_row + col0 + c, h);
            tmem_ld8(tmem_row + col0 + RPH + c, l);
            tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < 8; ++i) y[c + i] += h[i] + l[i];
        }
    }
}

template <int RPH, bool INNER>
__global__ void __launch_bounds__(kTrThreads, 1) k_tf32_rows(const __grid_constant__ CUtensorMap tmap, const TcParams P) {
    constexpr int N = 2 * RPH;
    constexpr int kB = N * 128;                       // factor chunk: N rows x 32 fp32 (swizzled)
    constexpr uint32_t kIdesc = idesc_tf32(128, N);
    static_assert(kTfDbuf == 4 && kTfA == 4 && kTrMmaWarps == 2 && kTrDone % kTfB == 0 && kTrDone % kTfA == 0,
                  "chunk g owns accumulator and A slot g % 4; chunk pairs alternate between two MMA warps");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char* base_ptr = smem_raw + (base - raw);
    unsigned char* boxes = base_ptr;                               // [kTfRaw][kTfBox]
    unsigned char* bring = base_ptr + kTfRaw * kTfBox;             // [kTfB][kB]
    unsigned char* misc = bring + kTfB * kB;
    uint64_t* rfull = reinterpret_cast<uint64_t*>(misc);           // box landed
    uint64_t* rempty = rfull + kTfRaw;                             // box read by the 4 converter warps
    uint64_t* bfull = rempty + kTfRaw;                             // factor chunk landed
    uint64_t* afull = bfull + kTfB;                                // A slot written by the 4 converter warps
    uint64_t* done = afull + kTfA;                                 // [kTrDone] chunk's MMAs complete
    uint64_t* tempty = done + kTrDone;                             // [kTfDbuf] accumulator read
    uint64_t* drain = tempty + kTfDbuf;                            // [kTrMmaWarps]
    uint64_t* sfull = drain + kTrMmaWarps;                         // [kTileRing]
    uint64_t* sempty = sfull + kTileRing;                          // [kTileRing]
    uint64_t* zfull = sempty + kTileRing;                          // a tile's rows handed to the reducer
    uint64_t* zfree = zfull + 1;                                   // ... and read by it
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(zfree + 1);
    int* zok = reinterpret_cast<int*>(tmem_slot + 1);              // [4]: epilogue warps' status per tile
    TileRec* tile_ring = reinterpret_cast<TileRec*>(zok + 4);      // [kTileRing]
    float* red = reinterpret_cast<float*>(misc + kTfBars);         // [128][RPH]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kTfRaw; ++s) {
            mbar_init(&rfull[s], 1);
            mbar_init(&rempty[s], 4);
        }
        for (int s = 0; s < kTfB; ++s) mbar_init(&bfull[s], 1);
        for (int s = 0; s < kTfA; ++s) mbar_init(&afull[s], 4);
        for (int s = 0; s < kTrDone; ++s) mbar_init(&done[s], 1);
        for (int b = 0; b < kTfDbuf; ++b) mbar_init(&tempty[b], 4);
        for (int w = 0; w < kTrMmaWarps; ++w) mbar_init(&drain[w], 1);
        for (int k = 0; k < kTileRing; ++k) {
            mbar_init(&sfull[k], 1);
            // the MMA warps, the 4 epilogue warps, the factor producer, the converters, the reducer
            mbar_init(&sempty[k], kTrMmaWarps + 5 + 4 * kTfConvGroups + 1);
        }
        mbar_init(zfull, 4);
        mbar_init(zfree, 1);
        fence_mbar_init();
    }
    if (warp == 5) tmem_alloc(tmem_slot, kTfCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    // CTA g's first tile is tile g; its first tensor boxes go out before the wait
    const int first_tile = g_first_tile(P.n_tiles);
    const TileRec ft = decode_tile<INNER>(P, first_tile);
    const int npre = first_tile >= 0 ? (ft.kc1 - ft.kc0 < kTfRaw ? ft.kc1 - ft.kc0 : kTfRaw) : 0;
    if (warp == 4 && lane == 0) {
        prefetch_tensormap(&tmap);
        for (int j = 0; j < npre; ++j) {
            mbar_arrive_expect_tx(&rfull[j], (uint32_t)kTfBox);
            tma_load_3d(boxes + j * kTfBox, &tmap, &rfull[j], (ft.kc0 + j) * 32, ft.ib * P.I_T, ft.ot * P.O_T);
        }
    }
    // With P.early only the epilogue warps (Grams, V and the row weights that the kernel before
    // writes) wait for that kernel; the producers, converters and MMA warps read the tensor, the
    // packed operand and the tile counter, all written two or more kernels back (see k_tc_rows)
    if (!P.early || warp < 4 || warp == kTrReducerWarp) pdl_wait();
    pdl_trigger();

    if (warp == kTrReducerWarp) {
        // ------------------------------ tile reducer ------------------------------
        tile_reducer<RPH, INNER>(P, tile_ring, sfull, sempty, zfull, zfree, zok, red, lane);
        return;
    }

    if (warp == kTrBWarp) {
        // --------------------- factor-chunk producer (all tiles alike) ---------------------
        if (lane == 0) {
            const unsigned char* FcT = P.cur ? P.FcTb[__ldcg(P.cur + P.fct_sel)] : P.FcT;
            int64_t g = 0, b_issued = 0;
            bool ok = true;
            for (int64_t s = 0; ok; ++s) {
                const int slot = (int)(s % kTileRing);
                if (!mbar_wait_bounded(&sfull[slot], (uint32_t)((s / kTileRing) & 1))) {
                    record_device_error(P.err, kErrWaitFull);
                    break;
                }
                const TileRec tr = tile_ring[slot];
                mbar_arrive(&sempty[slot]);
                if (tr.t < 0) break;
                for (int kc = tr.kc0; kc < tr.kc1; ++kc, ++g) {
                    const int bs = (int)(g % kTfB);
                    // slot bs last held chunk g - kTfB: wait for that chunk's MMAs
                    if (g >= kTfB && !mbar_wait_bounded(&done[(g - kTfB) % kTrDone],
                                                        (uint32_t)(((g - kTfB) / kTrDone) & 1))) {
                        record_device_error(P.err, kErrWaitEmpty);
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&bfull[bs], (uint32_t)kB);
                    bulk_load(bring + bs * kB, FcT + (int64_t)kc * kB, (uint32_t)kB, &bfull[bs]);
                    b_issued = g + 1;
                }
            }
            drain_ring(bfull, kTfB, b_issued, P.err);
        }
        return;
    }

    if (warp == 4) {
        // ------------------------- scheduler + box producer -------------------------
        if (lane == 0) {
            int64_t g = 0;                      // chunks of this CTA
            int64_t raw_issued = npre;
            bool ok = true;
            for (int64_t s = 0; ok; ++s) {
                const int slot = (int)(s % kTileRing);
                if (!mbar_wait_bounded(&sempty[slot], (uint32_t)((s / kTileRing) & 1) ^ 1u)) {
                    record_device_error(P.err, kErrWaitEmpty);
                    break;
                }
                int t = first_tile;
                if (s > 0) {
                    const unsigned int grab = atomicAdd(P.sched, 1u) + (unsigned int)gridDim.x;
                    t = grab < (unsigned int)P.n_tiles ? (int)grab : -1;
                }
                const TileRec tr = s == 0 ? ft : decode_tile<INNER>(P, t);
                tile_ring[slot] = tr;
                mbar_arrive(&sfull[slot]);
                if (t < 0) break;
                const int kc0 = tr.kc0, kc1 = tr.kc1;
                for (int kc = kc0; kc < kc1; ++kc, ++g) {
                    if (!(s == 0 && kc - kc0 < npre)) {
                        const int rs = (int)(g % kTfRaw);
                        if (!mbar_wait_bounded(&rempty[rs], (uint32_t)((g / kTfRaw) & 1) ^ 1u)) {
                            record_device_error(P.err, kErrWaitEmpty);
                            ok = false;
                            break;
                        }
                        mbar_arrive_expect_tx(&rfull[rs], (uint32_t)kTfBox);
                        tma_load_3d(boxes + rs * kTfBox, &tmap, &rfull[rs], kc * 32, tr.ib * P.I_T, tr.ot * P.O_T);
                        raw_issued = g + 1;
                    }
                }
            }
            drain_ring(rfull, kTfRaw, raw_issued, P.err);
        }
        return;
    }

    if (warp >= 6 && warp < 6 + 4 * kTfConvGroups) {
        // ------------------------------ converters ------------------------------
        // warp w may reach TMEM lanes 32 (w % 4) .. 32 (w % 4) + 31: tile row m = TMEM lane m.
        // Group cg converts the chunks g with g % kTfConvGroups == cg, so that the latency of
        // one chunk's loads, conversion and tensor-memory stores overlaps the next chunk's.
        const int cg = (warp - 6) >> 2;
        const int q = warp & 3;
        const int m = q * 32 + lane;
        const uint32_t tmem_lane = tmem + ((uint32_t)(q * 32) << 16);
        int64_t g = 0;
        bool ok = true;
        for (int64_t s = 0; ok; ++s) {
            const int slot = (int)(s % kTileRing);
            if (!warp_wait(&sfull[slot], (uint32_t)((s / kTileRing) & 1))) {
                if (lane == 0) record_device_error(P.err, kErrWaitFull);
                break;
            }
            const TileRec tr = tile_ring[slot];
            __syncwarp();
            if (lane == 0) mbar_arrive(&sempty[slot]);
            if (tr.t < 0) break;
            for (int kc = tr.kc0; kc < tr.kc1; ++kc, ++g) {
                if ((int)(g % kTfConvGroups) != cg) continue;
                const int rs = (int)(g % kTfRaw);
                if (!warp_wait(&rfull[rs], (uint32_t)((g / kTfRaw) & 1))) {
                    if (lane == 0) record_device_error(P.err, kErrWaitFull);
                    ok = false;
                    break;
                }
                // logical 16-byte group j of row m sits at group j ^ (m & 7) (128-byte swizzle);
                // the eight lanes of a quarter-warp thus touch eight different bank groups
                const float4* row = reinterpret_cast<const float4*>(boxes + rs * kTfBox + m * 128);
                float v[32];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float4 x = row[j ^ (m & 7)];
                    v[4 * j] = x.x;
                    v[4 * j + 1] = x.y;
                    v[4 * j + 2] = x.z;
                    v[4 * j + 3] = x.w;
                }
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(&rempty[rs]);
                uint32_t hi[32], lo[32];
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const float h = tf32_rna(v[i]);
                    hi[i] = __float_as_uint(h);
                    lo[i] = __float_as_uint(tf32_rna(v[i] - h));
                }
                // A slot g % 4 last held chunk g - 4: wait for that chunk's MMAs
                const int a = (int)(g % kTfA);
                if (g >= kTfA && !warp_wait(&done[(g - kTfA) % kTrDone], (uint32_t)(((g - kTfA) / kTrDone) & 1))) {
                    if (lane == 0) record_device_error(P.err, kErrWaitEmpty);
                    ok = false;
                    break;
                }
                tc_fence_after();
                tmem_st32(tmem_lane + kTfAcol + (uint32_t)(a * 64), hi);
                tmem_st32(tmem_lane + kTfAcol + (uint32_t)(a * 64 + 32), lo);
                tmem_wait_st();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&afull[a]);
            }
        }
        return;
    }

    if (warp == 5 || warp == kTfMmaWarp2) {
        // ------------------------------ MMA issuers ------------------------------
        // The 8 MMAs of one chunk accumulate into one tensor-memory accumulator, so each waits
        // for the one before it (about 90 cycles), and the tensor pipe runs them in issue
        // order.  A warp therefore takes two chunks at a time (g, g + 1) and interleaves their
        // MMAs, so that two independent chains share the pipe.  Warp 5 takes the pairs with
        // g % 4 == 0, warp 14 those with g % 4 == 2; chunk g keeps accumulator and A slot g % 4.
        // A first chunk waits for its partner, which may come with the next tile; the CTA's
        // last chunk may have none and goes alone.  The issuing lane is elected once, and it
        // also commits.
        const int mg = warp == 5 ? 0 : 1;
        const uint32_t leader = elect_leader();
        int64_t g = 0;
        bool ok = true, pending = false;
        auto issue = [&](int64_t c0, int n) -> bool {
            for (int j = 0; j < n; ++j) {
                const int64_t c = c0 + j;
                if (!warp_wait(&tempty[c % kTfDbuf], (uint32_t)((c / kTfDbuf) & 1) ^ 1u) ||
                    !warp_wait(&afull[c % kTfA], (uint32_t)((c / kTfA) & 1)) ||
                    !warp_wait(&bfull[c % kTfB], (uint32_t)((c / kTfB) & 1))) {
                    if (lane == 0) record_device_error(P.err, kErrWaitFull);
                    return false;
                }
            }
            tc_fence_after();
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {       // T_lo x [F_hi | F_lo] first (kk < 4), then T_hi on top
                for (int j = 0; j < n; ++j) {
                    const int64_t c = c0 + j;
                    const uint32_t b0 = base + (uint32_t)(kTfRaw * kTfBox + (int)(c % kTfB) * kB);
                    const uint32_t dt = tmem + (uint32_t)((int)(c % kTfDbuf) * kTfAccCols);
                    const uint32_t at = tmem + kTfAcol + (uint32_t)((int)(c % kTfA) * 64) + (kk < 4 ? 32u : 0u);
                    tc_mma_tf32_ts_lead(dt, at + (kk & 3) * 8, smem_desc_sw128(b0 + (kk & 3) * 32, 16, 1024), kIdesc,
                                        kk > 0 ? 1u : 0u, leader);
                }
            }
            for (int j = 0; j < n; ++j) tc_commit_lead(&done[(c0 + j) % kTrDone], leader);
            return true;
        };
        for (int64_t s = 0; ok; ++s) {
            const int slot = (int)(s % kTileRing);
            if (!warp_wait(&sfull[slot], (uint32_t)((s / kTileRing) & 1))) {
                if (lane == 0) record_device_error(P.err, kErrWaitFull);
                break;
            }
            const TileRec tr = tile_ring[slot];
            __syncwarp();
            if (lane == 0) mbar_arrive(&sempty[slot]);
            if (tr.t < 0) break;
            for (int kc = tr.kc0; kc < tr.kc1 && ok; ++kc, ++g) {
                if ((int)((g >> 1) & 1) != mg) continue;
                if ((g & 1) == 0) {
                    pending = true;
                } else {
                    ok = issue(g - 1, 2);
                    pending = false;
                }
            }
        }
        if (ok && pending) ok = issue(g - 1, 1);
        tc_commit_lead(&drain[mg], leader);
        if (!warp_wait(&drain[mg], 0) && lane == 0) record_device_error(P.err, kErrWaitDrain);
        __syncwarp();
        named_bar_sync(2, 128 + 32 * kTrMmaWarps);
        if (warp == 5) {
            tc_fence_after();
            tmem_dealloc(tmem, kTfCols);
        }
        return;
    }

    // ------------------------------ epilogue (warps 0-3) ------------------------------
    gram_job_run(P.job, (int)blockIdx.x * 4 + warp, (int)gridDim.x * 4);
    const float* Wt = P.cur ? P.Wb[__ldcg(P.cur + P.w_sel) ^ P.w_flip] : P.W;
    const float* Fit = P.cur ? P.Fib[__ldcg(P.cur + P.fi_sel) ^ P.fi_flip] : P.Fi;
    const int m = threadIdx.x;                       // tile row = TMEM lane
    const int m_o = m / P.I_T, m_i = m - m_o * P.I_T;   // inner mode: row m = (outer m_o, inner m_i)
    const uint32_t tmem_row = tmem + ((uint32_t)(warp * 32) << 16);
    bool ok = true;
    int64_t gq = 0;
    int q = 0;                                       // tiles handed to the reducer
    for (int64_t s = 0; ok; ++s) {
        const int slot = (int)(s % kTileRing);
        if (!warp_wait(&sfull[slot], (uint32_t)((s / kTileRing) & 1))) {
            if (lane == 0) record_device_error(P.err, kErrWaitFull);
            break;
        }
        const TileRec tr = tile_ring[slot];
        __syncwarp();
        if (lane == 0) mbar_arrive(&sempty[slot]);
        if (tr.t < 0) break;
        float w[RPH];
        tile_weights<RPH, INNER>(P, tr, m, m_o, m_i, Wt, Fit, w);
        float y[RPH];
#pragma unroll
        for (int p = 0; p < RPH; ++p) y[p] = 0.f;
        for (int kc = tr.kc0; kc < tr.kc1; ++kc, ++gq) {
            const int d = (int)(gq % kTfDbuf);
            if (ok && !warp_wait(&done[gq % kTrDone], (uint32_t)((gq / kTrDone) & 1))) {
                if (lane == 0) record_device_error(P.err, kErrWaitFull);
                ok = false;
            }
            if (ok) {
                tc_fence_after();
                add_rows<RPH>(tmem_row, d * kTfAccCols, y);
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&tempty[d]);
            }
        }
#pragma unroll
        for (int p = 0; p < RPH; ++p) y[p] *= w[p];
        tile_handover<RPH>(y, red, m, warp, lane, q, ok, zfull, zfree, zok, P.err);
        ++q;
    }
    tc_fence_before();
    named_bar_sync(2, 128 + 32 * kTrMmaWarps);
}

// TF32 last-mode kernel: FP32 tensor storage, mode N-1 (step a1 for the FP32 form)
//
// M_{N-1}(c, :) = sum_o W(o, :) (*) sum_i T(o, i, c) A_{N-2}(i, :).  A tile is one outer
// index o, 32 rows i and a block of 128 columns c (four 32 x 32 boxes, 16 KB).  The MMAs
// take A = the split tile transposed (lane = column c, K = row i) from tensor memory and
// B = the packed A_{N-2} rows of the tile (32-row chunks, as the rows kernel's factor
// operand), and the epilogue folds W(o, :) x accumulator into registers, one column per
// thread, over the CTA's contiguous tile range.  The converter warp of lane quarter q reads
// box q one row (32 columns) per instruction, free of bank conflicts, and writes its column's
// 32 split values into its tensor-memory lane.  Warps, rings, MMA issue and the split are
// those of k_tf32_rows; tiles are static ranges (grid = CTAs x column blocks).
// ----------------------------------------------------------------------------
template <int RPH>
__global__ void __launch_bounds__(kTfThreads, 1) k_tf32_last(const __grid_constant__ CUtensorMap tmap, const TcParams P) {
    constexpr int N = 2 * RPH;
    constexpr int kB = N * 128;                       // A_{N-2} chunk: N rows x 32 fp32 (swizzled)
    constexpr int kSub = 4096;                        // one 32 x 32 box
    constexpr uint32_t kIdesc = idesc_tf32(128, N);
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char* base_ptr = smem_raw + (base - raw);
    unsigned char* boxes = base_ptr;                               // [kTfRaw][4 x kSub]
    unsigned char* bring = base_ptr + kTfRaw * kTfBox;             // [kTfB][kB]
    unsigned char* misc = bring + kTfB * kB;
    uint64_t* rfull = reinterpret_cast<uint64_t*>(misc);
    uint64_t* rempty = rfull + kTfRaw;
    uint64_t* bfull = rempty + kTfRaw;
    uint64_t* bempty = bfull + kTfB;
    uint64_t* afull = bempty + kTfB;
    uint64_t* aempty = afull + kTfA;
    uint64_t* tfull = aempty + kTfA;
    uint64_t* tempty = tfull + kTfDbuf;
    uint64_t* drain = tempty + kTfDbuf;                            // [2]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 2);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = blockIdx.x, G = gridDim.x;
    const int cb = blockIdx.y;
    int64_t t_beg, t_end;
    tile_range(P.n_tiles, g, G, t_beg, t_end);
    const int64_t nt = t_end - t_beg;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kTfRaw; ++s) {
            mbar_init(&rfull[s], 1);
            mbar_init(&rempty[s], 4);
        }
        for (int s = 0; s < kTfB; ++s) {
            mbar_init(&bfull[s], 1);
            mbar_init(&bempty[s], 1);
        }
        for (int s = 0; s < kTfA; ++s) {
            mbar_init(&afull[s], 4);
            mbar_init(&aempty[s], 1);
        }
        for (int b = 0; b < kTfDbuf; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 4);
        }
        mbar_init(&drain[0], 1);
        mbar_init(&drain[1], 1);
        fence_mbar_init();
    }
    if (warp == 5) tmem_alloc(tmem_slot, kTfCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    // the first tiles' boxes go out before the wait (the tensor is never written)
    const int npre = (int)(nt < kTfRaw ? nt : kTfRaw);
    if (warp == 4 && lane == 0) {
        prefetch_tensormap(&tmap);
        for (int q = 0; q < npre; ++q) {
            const int64_t t = t_beg + q;
            const int64_t ib = t / P.n_ot, o = t % P.n_ot;     // I_T = 32, O_T = 1
            mbar_arrive_expect_tx(&rfull[q], (uint32_t)kTfBox);
            for (int j = 0; j < 4; ++j)
                tma_load_3d(boxes + q * kTfBox + j * kSub, &tmap, &rfull[q], cb * 128 + 32 * j, (int)(ib * 32), (int)o);
        }
    }
    pdl_wait();
    pdl_trigger();

    if (warp == kTfBWarp) {
        // --------------------------- A_{N-2} chunk producer ---------------------------
        if (lane == 0) {
            const unsigned char* FcT = P.cur ? P.FcTb[__ldcg(P.cur + P.fct_sel)] : P.FcT;
            int64_t b_issued = 0;
            for (int64_t q = 0; q < nt; ++q) {
                const int64_t ib = (t_beg + q) / P.n_ot;
                const int bs = (int)(q % kTfB);
                if (!mbar_wait_bounded(&bempty[bs], (uint32_t)((q / kTfB) & 1) ^ 1u)) {
                    record_device_error(P.err, kErrWaitEmpty);
                    break;
                }
                mbar_arrive_expect_tx(&bfull[bs], (uint32_t)kB);
                bulk_load(bring + bs * kB, FcT + ib * kB, (uint32_t)kB, &bfull[bs]);
                b_issued = q + 1;
            }
            drain_ring(bfull, kTfB, b_issued, P.err);
        }
        return;
    }

    if (warp == 4) {
        // ------------------------------- box producer -------------------------------
        if (lane == 0) {
            int64_t raw_issued = npre;
            for (int64_t q = 0; q < nt; ++q) {
                const int64_t t = t_beg + q;
                const int64_t ib = t / P.n_ot, o = t % P.n_ot;
                if (q >= npre) {
                    const int rs = (int)(q % kTfRaw);
                    if (!mbar_wait_bounded(&rempty[rs], (uint32_t)((q / kTfRaw) & 1) ^ 1u)) {
                        record_device_error(P.err, kErrWaitEmpty);
                        break;
                    }
                    mbar_arrive_expect_tx(&rfull[rs], (uint32_t)kTfBox);
                    for (int j = 0; j < 4; ++j)
                        tma_load_3d(boxes + rs * kTfBox + j * kSub, &tmap, &rfull[rs], cb * 128 + 32 * j, (int)(ib * 32),
                                    (int)o);
                    raw_issued = q + 1;
                }
            }
            drain_ring(rfull, kTfRaw, raw_issued, P.err);
        }
        return;
    }

    if (warp >= 6 && warp < kTfMmaWarp2) {
        // ------------------------------ converters ------------------------------
        // lane quarter q = column group q of the block: thread = column 32 q + lane = TMEM lane
        const int cg = (warp - 6) >> 2;
        const int q = warp & 3;
        const uint32_t tmem_lane = tmem + ((uint32_t)(q * 32) << 16);
        for (int64_t k = cg; k < nt; k += kTfConvGroups) {
            const int rs = (int)(k % kTfRaw);
            if (!warp_wait(&rfull[rs], (uint32_t)((k / kTfRaw) & 1))) {
                if (lane == 0) record_device_error(P.err, kErrWaitFull);
                break;
            }
            // row i of box q: 128 bytes, 16-byte group j at j ^ (i & 7); this lane's column is
            // in group lane / 4
            const unsigned char* box = boxes + rs * kTfBox + q * kSub + (lane & 3) * 4;
            float v[32];
#pragma unroll
            for (int i = 0; i < 32; ++i)
                v[i] = *reinterpret_cast<const float*>(box + i * 128 + (((lane >> 2) ^ (i & 7)) << 4));
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(&rempty[rs]);
            uint32_t hi[32], lo[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const float h = tf32_rna(v[i]);
                hi[i] = __float_as_uint(h);
                lo[i] = __float_as_uint(tf32_rna(v[i] - h));
            }
            const int a = (int)(k % kTfA);
            if (!warp_wait(&aempty[a], (uint32_t)((k / kTfA) & 1) ^ 1u)) {
                if (lane == 0) record_device_error(P.err, kErrWaitEmpty);
                break;
            }
            tc_fence_after();
            tmem_st32(tmem_lane + kTfAcol + (uint32_t)(a * 64), hi);
            tmem_st32(tmem_lane + kTfAcol + (uint32_t)(a * 64 + 32), lo);
            tmem_wait_st();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&afull[a]);
        }
        return;
    }

    if (warp == 5 || warp == kTfMmaWarp2) {
        // ------------------------------ MMA issuers (tiles in turn) ------------------------------
        const int mg = warp == 5 ? 0 : 1;
        for (int64_t k = mg; k < nt; k += 2) {
            const int d = (int)(k % kTfDbuf), a = (int)(k % kTfA), bs = (int)(k % kTfB);
            if (!warp_wait(&tempty[d], (uint32_t)((k / kTfDbuf) & 1) ^ 1u) ||
                !warp_wait(&afull[a], (uint32_t)((k / kTfA) & 1)) || !warp_wait(&bfull[bs], (uint32_t)((k / kTfB) & 1))) {
                if (lane == 0) record_device_error(P.err, kErrWaitFull);
                break;
            }
            tc_fence_after();
            const uint32_t b0 = base + (uint32_t)(kTfRaw * kTfBox + bs * kB);
            const uint32_t dt = tmem + (uint32_t)(d * kTfAccCols);
            const uint32_t at = tmem + kTfAcol + (uint32_t)(a * 64);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)     // T_lo^T x [F_hi | F_lo], first accumulator
                tc_mma_tf32_ts_elect(dt, at + 32 + kk * 8, smem_desc_sw128(b0 + kk * 32, 16, 1024), kIdesc,
                                     kk > 0 ? 1u : 0u);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)     // T_hi^T x [F_hi | F_lo] on top
                tc_mma_tf32_ts_elect(dt, at + kk * 8, smem_desc_sw128(b0 + kk * 32, 16, 1024), kIdesc, 1u);
            tc_commit_elect(&aempty[a]);
            tc_commit_elect(&bempty[bs]);
            tc_commit_elect(&tfull[d]);
        }
        tc_commit_elect(&drain[mg]);
        if (!warp_wait(&drain[mg], 0) && lane == 0) record_device_error(P.err, kErrWaitDrain);
        __syncwarp();
        named_bar_sync(2, 192);
        if (warp == 5) {
            tc_fence_after();
            tmem_dealloc(tmem, kTfCols);
        }
        return;
    }

    // ---------------- warps 0-3: fold W(o,:) x tile accumulator into registers ----------------
    gram_job_run(P.job, ((int)blockIdx.y * (int)gridDim.x + (int)blockIdx.x) * 4 + warp,
                 (int)(gridDim.x * gridDim.y) * 4);
    const float* Wt = P.cur ? P.Wb[__ldcg(P.cur + P.w_sel) ^ P.w_flip] : P.W;
    const int m = threadIdx.x;
    const uint32_t tmem_row = tmem + ((uint32_t)(warp * 32) << 16);
    bool ok = true;
    float acc[RPH];
#pragma unroll
    for (int p = 0; p < RPH; ++p) acc[p] = 0.f;
    for (int64_t k = 0; k < nt && ok; ++k) {
        const int64_t o = (t_beg + k) % P.n_ot;
        float w[RPH];
        const float* wr = Wt + o * P.ldw;
#pragma unroll
        for (int p = 0; p < RPH; ++p) w[p] = p < P.r ? __ldg(wr + p) : 0.f;
        const int d = (int)(k % kTfDbuf);
        if (!warp_wait(&tfull[d], (uint32_t)((k / kTfDbuf) & 1))) {
            if (lane == 0) record_device_error(P.err, kErrWaitFull);
            ok = false;
            break;
        }
        tc_fence_after();
        float y[RPH];
        read_rows<RPH>(tmem_row, d * kTfAccCols, y);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[d]);
#pragma unroll
        for (int p = 0; p < RPH; ++p) acc[p] = fmaf(w[p], y[p], acc[p]);
    }
    // row m of the result = column cb*128 + m of M_{N-1}
    const int64_t c = (int64_t)cb * 128 + m;
    if (ok && c < P.C) {
        float* dst = P.part + ((int64_t)g * P.Cpad + c) * P.RP;
#pragma unroll
        for (int p = 0; p < RPH; ++p)
            if (p < P.r) dst[p] = acc[p];
    }
    tc_fence_before();
    named_bar_sync(2, 192);
}

template <int RPH>
cudaError_t launch_tf32_impl(int kind, dim3 grid, size_t smem, cudaStream_t st, const CUtensorMap& map,
                             const TcParams& P, bool pdl) {
    typedef void (*Kern)(const CUtensorMap, const TcParams);
    Kern k = kind == 0 ? (Kern)k_tf32_rows<RPH, true> : kind == 1 ? (Kern)k_tf32_rows<RPH, false> : (Kern)k_tf32_last<RPH>;
    static size_t set_bytes[3] = {0, 0, 0};
    if (set_bytes[kind] < smem) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        set_bytes[kind] = smem;
    }
    if (grid.x == 0) return cudaSuccess;
    return launch_kernel(k, grid, dim3(kind == 2 ? kTfThreads : kTrThreads), smem, st, pdl, map, P);
}

template <int RPH>
cudaError_t launch_tc_impl(int kind, dim3 grid, size_t smem, cudaStream_t st, const CUtensorMap& map,
                           const TcParams& P, bool pdl) {
    typedef void (*Kern)(const CUtensorMap, const TcParams);
    Kern k = kind == 0 ? (Kern)k_tc_rows<RPH, true> : kind == 1 ? (Kern)k_tc_rows<RPH, false> : (Kern)k_tc_last<RPH>;
    static size_t set_bytes[3] = {0, 0, 0};
    if (set_bytes[kind] < smem) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        set_bytes[kind] = smem;
    }
    if (grid.x == 0) return cudaSuccess;
    return launch_kernel(k, grid, dim3(kTcThreads), smem, st, pdl, map, P);
}

}  // namespace

int tc_rows_ctas_per_sm() { return kRowCtasPerSm; }
size_t tc_rows_smem(int rph) {
    const int N = 2 * rph;
    return (size_t)kRowStages * (kBoxBytes + N * 128) + 1024 + kRowMiscBytes + 128 * rph * 4;
}
size_t tc_last_smem(int rph) {
    const int N = 2 * rph;
    return (size_t)kTcStages * (2 * kBoxBytes + 2 * N * 128) + 1024 + 256;
}
// bytes of the packed A_{N-2} operand of the last-mode kernel per 128-row block
size_t tc_last_b_bytes(int rph) { return (size_t)2 * (2 * rph) * 128; }
size_t tf32_rows_smem(int rph) {
    const int N = 2 * rph;
    return (size_t)kTfRaw * kTfBox + (size_t)kTfB * N * 128 + 1024 + kTfBars + 128 * rph * 4;
}

cudaError_t launch_stream_tf32(int kind, int rph, dim3 grid, size_t smem, cudaStream_t st, const CUtensorMap& map,
                               const TcParams& P, bool pdl) {
    if (kind > 2) return cudaErrorInvalidValue;
    switch (rph) {
        case 8: return launch_tf32_impl<8>(kind, grid, smem, st, map, P, pdl);
        case 16: return launch_tf32_impl<16>(kind, grid, smem, st, map, P, pdl);
        case 24: return launch_tf32_impl<24>(kind, grid, smem, st, map, P, pdl);
        case 32: return launch_tf32_impl<32>(kind, grid, smem, st, map, P, pdl);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_stream_tc(int kind, int rph, dim3 grid, size_t smem, cudaStream_t st, const CUtensorMap& map,
                             const TcParams& P, bool pdl) {
    switch (rph) {
        case 8: return launch_tc_impl<8>(kind, grid, smem, st, map, P, pdl);
        case 16: return launch_tc_impl<16>(kind, grid, smem, st, map, P, pdl);
        case 24: return launch_tc_impl<24>(kind, grid, smem, st, map, P, pdl);
        case 32: return launch_tc_impl<32>(kind, grid, smem, st, map, P, pdl);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ntf
