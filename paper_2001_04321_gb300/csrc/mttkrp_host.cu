// Host side of the MTTKRP (step a1): planning, workspace layout, the small
// pack / weight-table / reduction kernels, and the launch sequence
//   pack factors -> weight table W -> streaming kernel -> reduction.
#include "mttkrp.cuh"
#include "mttkrp_kernels.cuh"
#include "mttkrp_reduce.cuh"
#include "epilogue.cuh"
#include "mttkrp_tc.cuh"

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>

namespace ntf {

// ---------------------------------------------------------------------------
// tensor view
// ---------------------------------------------------------------------------
ntf_status make_view(const ntf_tensor* T, TensorView* v) {
    if (!T) return fail(NTF_EINVAL, "tensor is NULL");
    if (T->order < 2 || T->order > NTF_MAX_ORDER)
        return fail(NTF_EINVAL, "tensor order must be in [2, 8], got " + std::to_string(T->order));
    if (T->dtype != NTF_F32 && T->dtype != NTF_BF16) return fail(NTF_EINVAL, "unknown tensor dtype");
    if (!T->data) return fail(NTF_EINVAL, "tensor data is NULL");
    if (reinterpret_cast<uintptr_t>(T->data) % 16) return fail(NTF_EINVAL, "tensor data must be 16-byte aligned");
    v->order = T->order;
    for (int l = 0; l < T->order; ++l) {
        if (T->dims[l] < 1) return fail(NTF_EINVAL, "tensor dims must be >= 1");
        if (T->dims[l] > (int64_t(1) << 31)) return fail(NTF_EINVAL, "tensor dim exceeds 2^31");
        v->dims[l] = T->dims[l];
    }
    v->dtype = T->dtype;
    v->es = T->dtype == NTF_F32 ? 4 : 2;
    v->C = T->dims[T->order - 1];
    v->ld = T->ld ? T->ld : v->C;
    if (v->ld < v->C) return fail(NTF_EINVAL, "tensor ld must be >= dims[order-1]");
    if ((v->ld * v->es) % 16)
        return fail(NTF_EINVAL, "tensor row pitch ld*sizeof(element) must be a multiple of 16 bytes (ld=" +
                                    std::to_string(v->ld) + "); pad the last mode or use ntf_tensor_to_bf16/ntf_solve");
    v->Ii = T->dims[T->order - 2];
    v->n_o = 1;
    for (int l = 0; l < T->order - 2; ++l) v->n_o *= T->dims[l];
    v->data = T->data;
    return NTF_OK;
}

int num_sms() {
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!cached[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
        cached[dev] = n;
    }
    return cached[dev];
}

// ---------------------------------------------------------------------------
// tensor map
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

ntf_status encode_tensor_map_3d(CUtensorMap* map, ntf_dtype dtype, const void* base, uint64_t d0, uint64_t d1,
                                uint64_t d2, uint64_t stride1_bytes, uint64_t stride2_bytes, uint32_t box0,
                                uint32_t box1, uint32_t box2) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return fail(NTF_ECUDA, "cuTensorMapEncodeTiled entry point unavailable");
    const cuuint64_t dims[3] = {d0, d1, d2};
    const cuuint64_t strides[2] = {stride1_bytes, stride2_bytes};
    const cuuint32_t box[3] = {box0, box1, box2};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(map, dtype == NTF_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
                    const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(NTF_ECUDA, "cuTensorMapEncodeTiled failed with code " + std::to_string((int)r));
    return NTF_OK;
}

// ---------------------------------------------------------------------------
// planning
// ---------------------------------------------------------------------------
static double util(int64_t n, int64_t t) { return (double)n / (double)(t * ceil_div(n, t)); }

// tile shape (I_T inner x O_T outer, I_T * O_T = 128) with the fewest padded rows;
// on ties the inner mode prefers the smallest I_T (fewer streaming CTAs share an
// inner block, so its reduction sums fewer partials), the last mode the largest
static void choose_tile(int64_t Ii, int64_t n_o, int max_IT, bool prefer_small, int* I_T, int* O_T) {
    double best = -1;
    for (int k = 0; (1 << k) <= max_IT; ++k) {
        const int it = prefer_small ? (1 << k) : (max_IT >> k);
        const int ot = 128 / it;
        const double u = util(Ii, it) * util(n_o, ot);
        if (u > best + 1e-9) { best = u; *I_T = it; *O_T = ot; }
    }
}

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// NTF_TF32: unset or 1 = 3xTF32 tensor-core kernels for every mode of an FP32 tensor,
// 2 = for the modes before the last only, 0 = the FFMA kernels
static int tf32_mode() {
    static const int m = [] {
        const char* e = std::getenv("NTF_TF32");
        return (e && (e[0] == '0' || e[0] == '2')) ? e[0] - '0' : 1;
    }();
    return m;
}

// Row tiles at the end of the 3xTF32 row streams' schedule that are handed out as two column
// segments, in quarters of the CTA count (NTF_TAIL_SPLIT, read once per process; 2 by default,
// 0 = none).  Tiles go to CTAs at run time, so the last ones decide when the stream ends: halving
// them halves the tail.
static int tail_split_quarters() {
    static int v = -1;
    if (v < 0) {
        const char* e = std::getenv("NTF_TAIL_SPLIT");
        const int x = e ? std::atoi(e) : 2;
        v = x >= 0 && x <= 16 ? x : 2;
    }
    return v;
}

// Target of scheduled tiles per CTA below which the tensor-core row streams split row tiles into
// column segments (NTF_SEG_TILES, read once per process; 2 by default).
static int seg_tiles_per_cta() {
    static int v = 0;
    if (!v) {
        const char* e = std::getenv("NTF_SEG_TILES");
        const int x = e ? std::atoi(e) : 0;
        v = x >= 1 && x <= 64 ? x : 2;
    }
    return v;
}

ntf_status plan_mttkrp(const TensorView& v, int rank, int mode, MttkrpPlan* p) {
    if (rank < 1 || rank > NTF_MAX_RANK) return fail(NTF_EINVAL, "rank must be in [1, 64]");
    if (mode < 0 || mode >= v.order) return fail(NTF_EINVAL, "mode out of range");
    MttkrpPlan P{};
    P.mode = mode;
    P.rank = rank;
    if (rank <= 32) {
        P.RP = (int)round_up(rank, 4);
        if (P.RP == 28) P.RP = 32;    // FFMA kernels are instantiated for 4..24 and 32 columns
        P.R = P.RP;
    } else {
        P.RP = 64;
        P.R = 32;
    }
    P.n_pb = P.RP / P.R;
    P.kind = mode == v.order - 1 ? ModeKind::Last : mode == v.order - 2 ? ModeKind::Inner : ModeKind::Outer;
    // bf16: tensor cores for every mode; fp32: the FFMA kernels, or the 3xTF32 tensor-core
    // kernels as NTF_TF32 selects
    P.tf32 = v.dtype == NTF_F32 && rank <= 32 && (tf32_mode() == 1 || (tf32_mode() == 2 && P.kind != ModeKind::Last));
    P.tc = (v.dtype == NTF_BF16 && rank <= 32) || P.tf32;
    P.RPH = (int)round_up(rank, 8);
    // inner mode: the tensor-core kernel keeps one slot per tile, so the smallest inner
    // extent (fewest tiles per output row) is preferred; the FFMA kernel the largest
    if (P.kind == ModeKind::Inner) choose_tile(v.Ii, v.n_o, 32, P.tc, &P.I_T, &P.O_T);
    else if (P.kind == ModeKind::Last && P.tf32) { P.I_T = 32; P.O_T = 1; }     // tf32 last mode: 32-row tiles
    else if (P.kind == ModeKind::Outer || P.tc) { P.I_T = 128; P.O_T = 1; }   // tc last mode: W(o,:) per tile
    else choose_tile(v.Ii, v.n_o, 128, false, &P.I_T, &P.O_T);
    P.nb = ceil_div(v.Ii, P.I_T);
    P.n_ot = ceil_div(v.n_o, P.O_T);
    P.n_tiles = P.nb * P.n_ot;
    P.n_kc = (int)ceil_div(v.C, P.tf32 ? 32 : kStageCols);   // tf32: 32 fp32 columns per chunk
    const int sms = num_sms();
    const int cb_cols = P.tc ? 128 : kStageCols;
    P.n_cb = (int)ceil_div(v.C, cb_cols);
    P.Cpad = (int64_t)P.n_cb * cb_cols;
    // tensor-core row kernels take tiles at run time and keep one slot per tile; the
    // others own contiguous tile ranges and keep one slot per (CTA, segment)
    P.tile_slots = P.tc && P.kind != ModeKind::Last;
    P.n_cs = 1;
    P.kc_per = P.n_kc;
    if (P.kind == ModeKind::Last) {
        int gs = sms / P.n_cb;
        if (gs < 1) gs = 1;
        if (gs > P.n_tiles) gs = (int)P.n_tiles;
        P.G = gs;
    } else {
        const int per_sm =
            (P.tc && !P.tf32 && tc_rows_ctas_per_sm() >= 2 && 2 * tc_rows_smem(P.RPH) <= 227 * 1024) ? 2 : 1;
        const int64_t cap = (int64_t)sms * per_sm;
        const int per_cta = seg_tiles_per_cta();
        if (P.tile_slots && P.n_tiles < per_cta * cap && P.n_kc >= 8) {
            // Few row tiles with long rows (e.g. merged modes): split each row tile into column
            // segments of at least 4 chunks so that every CTA gets about per_cta tiles to stream
            const int64_t want = ceil_div(per_cta * cap, P.n_tiles);
            const int64_t most = P.n_kc / 4;
            const int64_t ncs = std::max<int64_t>(1, std::min(want, most));
            P.kc_per = (int)ceil_div(P.n_kc, ncs);
            P.n_cs = (int)ceil_div(P.n_kc, P.kc_per);     // no empty segment
        } else if (P.tile_slots && P.tf32 && P.n_kc >= 8 && tail_split_quarters() > 0) {
            // many row tiles: only the last ones go out as two column segments of >= 4 chunks.
            // (3xTF32 only: a 500^3 rank-20 FP32 stream took 94.4 -> 93.0 us; the bf16 streams'
            // tiles are half as long, and the two slots per row tile that the epilogue then reads
            // cost the iteration more than the shorter tail saves.)
            const int64_t split = std::min<int64_t>(P.n_tiles - cap, cap * tail_split_quarters() / 4);
            if (split > 0) {
                P.kc_per = (int)ceil_div(P.n_kc, 2);
                P.n_cs = 2;
                P.n_whole = P.n_tiles - split;
            }
        }
        P.n_units = P.n_whole + (P.n_tiles - P.n_whole) * P.n_cs;
        P.G = (int)std::min<int64_t>(P.n_units, cap);
    }
    P.Smax = 1;
    if (P.kind == ModeKind::Inner && !P.tile_slots) {
        for (int g = 0; g < P.G; ++g) {
            const int64_t b = (P.n_tiles * g) / P.G, e = (P.n_tiles * (g + 1)) / P.G;
            if (e > b) {
                const int s = (int)((e - 1) / P.n_ot - b / P.n_ot + 1);
                if (s > P.Smax) P.Smax = s;
            }
        }
    }
    size_t off = 0;
    P.off_Fc = off;
    if (P.tc && P.kind == ModeKind::Last)                               // packed A_{N-2} blocks
        off = align256(off + (size_t)P.nb * (P.tf32 ? (size_t)(2 * P.RPH) * 128 : tc_last_b_bytes(P.RPH)));
    else if (P.tc)
        off = align256(off + (size_t)P.n_kc * (2 * P.RPH) * 128);       // packed A_{N-1} chunks
    else
        off = align256(off + sizeof(float) * (size_t)round_up(v.C, kStageCols) * P.RP);
    P.off_Fi = off;
    off = align256(off + sizeof(float) * (size_t)v.Ii * P.RP);
    P.off_W = off;
    off = align256(off + sizeof(float) * (size_t)v.n_o * P.RP);
    P.off_part = off;
    size_t part = 0;
    if (P.kind == ModeKind::Inner)
        part = P.tile_slots ? (size_t)P.n_tiles * P.n_cs * P.I_T * P.RP
                            : (size_t)P.G * P.Smax * kStreamWarps * P.I_T * P.RP;
    else if (P.kind == ModeKind::Outer)
        part = (size_t)v.n_o * P.nb * P.n_cs * P.RP;
    else
        part = (size_t)P.G * P.Cpad * P.RP;
    off = align256(off + sizeof(float) * part);
    // the run-time tile counter of the tensor-core row kernels
    P.off_sched = off;
    if (P.tile_slots) off = align256(off + sizeof(unsigned int));
    P.total = off;
    *p = P;
    return NTF_OK;
}

// ---------------------------------------------------------------------------
// small kernels
// ---------------------------------------------------------------------------
struct FactorPtrs {
    const float* a[NTF_MAX_ORDER];
};
struct Dims {
    int64_t d[NTF_MAX_ORDER];
};

// out (rows_out x RP) <- A (rows x r) with zero padding
__global__ void k_pack(const float* __restrict__ A, int64_t rows, int r, int RP, int64_t rows_out,
                       float* __restrict__ out) {
    const int64_t n = rows_out * RP;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / RP;
        const int p = (int)(idx % RP);
        out[idx] = (i < rows && p < r) ? A[i * r + p] : 0.f;
    }
}

// Tensor-core B operand of the rows kernel: for every 64-row chunk kc of A_{N-1},
// N = 2*RPH rows of 128 bytes holding [k = 0..63] of column n as bfloat16, high
// parts (n < RPH) then low parts (x - hi), 16-byte chunks XOR-swizzled by (n & 7)
// exactly as a 128-byte-swizzled TMA box would hold them in shared memory.
__global__ void k_pack_fct(const float* __restrict__ A, int64_t rows, int r, int RPH, int n_kc,
                           __nv_bfloat16* __restrict__ out) {
    const int N = 2 * RPH;
    const int64_t total = (int64_t)n_kc * N * 64;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int kl = (int)(idx % 64);
        const int n = (int)((idx / 64) % N);
        const int64_t kc = idx / (64 * (int64_t)N);
        const int64_t k = kc * 64 + kl;
        const int p = n < RPH ? n : n - RPH;
        const float x = (k < rows && p < r) ? A[k * r + p] : 0.f;
        const __nv_bfloat16 hi = __float2bfloat16_rn(x);
        const __nv_bfloat16 v = n < RPH ? hi : __float2bfloat16_rn(x - __bfloat162float(hi));
        const int64_t byte = (kc * N + n) * 128 + (((kl >> 3) ^ (n & 7)) << 4) + (kl & 7) * 2;
        out[byte / 2] = v;
    }
}

// The 3xTF32 operand: F_hi = tf32(F) | F_lo = tf32(F - F_hi) as FP32 words, 32-row chunks of
// 2 RPH rows x 128 B, 16-byte groups swizzled as a 128-byte-swizzled TMA box.
__global__ void k_pack_fct_tf32(const float* __restrict__ A, int64_t rows, int r, int RPH, int n_kc,
                                float* __restrict__ out) {
    const int N = 2 * RPH;
    const int64_t total = (int64_t)n_kc * N * 32;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int kl = (int)(idx % 32);
        const int n = (int)((idx / 32) % N);
        const int64_t kc = idx / (32 * (int64_t)N);
        const int64_t k = kc * 32 + kl;
        const int p = n < RPH ? n : n - RPH;
        const float x = (k < rows && p < r) ? A[k * r + p] : 0.f;
        const float hi = tf32_rna(x);
        const int64_t byte = (kc * N + n) * 128 + (((kl >> 2) ^ (n & 7)) << 4) + (kl & 3) * 4;
        out[byte / 4] = n < RPH ? hi : tf32_rna(x - hi);
    }
}

// The tensor-core operand of a merged pair of modes (a, b): the Khatri-Rao rows
// K(ka Ib + kb, p) = A_a(ka, p) A_b(kb, p), packed exactly as k_pack_fct (bf16 hi | lo, 64-row
// chunks) or k_pack_fct_tf32 (TF32 hi | lo, 32-row chunks) pack a factor.  The two factors are
// read from the solver's buffers, chosen on the device: buffer cur[sel] ^ flip.
__global__ void k_pack_kr(KrPack K) {
    const float* Aa = K.cur ? K.a[__ldcg(K.cur + K.sel_a) ^ K.flip_a] : K.a[0];
    const float* Ab = K.cur ? K.b[__ldcg(K.cur + K.sel_b) ^ K.flip_b] : K.b[0];
    const int N = 2 * K.RPH;
    const int kw = K.tf32 ? 32 : 64;                   // rows per chunk
    const int64_t rows = K.Ia * K.Ib;
    const int64_t total = (int64_t)K.n_kc * N * kw;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int kl = (int)(idx % kw);
        const int n = (int)((idx / kw) % N);
        const int64_t kc = idx / (kw * (int64_t)N);
        const int64_t k = kc * kw + kl;
        const int p = n < K.RPH ? n : n - K.RPH;
        float x = 0.f;
        if (k < rows && p < K.r) {
            const int64_t ka = k / K.Ib, kb = k - ka * K.Ib;
            x = Aa[ka * K.r + p] * Ab[kb * K.r + p];
        }
        if (K.tf32) {
            const float hi = tf32_rna(x);
            const int64_t byte = (kc * N + n) * 128 + (((kl >> 2) ^ (n & 7)) << 4) + (kl & 3) * 4;
            static_cast<float*>(K.out)[byte / 4] = n < K.RPH ? hi : tf32_rna(x - hi);
        } else {
            const __nv_bfloat16 hi = __float2bfloat16_rn(x);
            const __nv_bfloat16 v = n < K.RPH ? hi : __float2bfloat16_rn(x - __bfloat162float(hi));
            const int64_t byte = (kc * N + n) * 128 + (((kl >> 3) ^ (n & 7)) << 4) + (kl & 7) * 2;
            static_cast<__nv_bfloat16*>(K.out)[byte / 2] = v;
        }
    }
}

cudaError_t launch_pack_kr(const KrPack& K, cudaStream_t st) {
    const int64_t total = (int64_t)K.n_kc * 2 * K.RPH * (K.tf32 ? 32 : 64);
    const int64_t blocks = std::min<int64_t>((total + 255) / 256, 4096);
    k_pack_kr<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, st>>>(K);
    count_launch();
    return cudaGetLastError();
}

// W(o,p) = prod_{l < N-2, l != skip} A_l(i_l(o), p)   (o in C order over modes 0..N-3)
__global__ void k_weights(FactorPtrs F, Dims D, int order, int skip, int r, int RP, int64_t n_o,
                          float* __restrict__ W) {
    const int64_t n = n_o * RP;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = idx / RP;
        const int p = (int)(idx % RP);
        float w = 0.f;
        if (p < r) {
            w = 1.f;
            int64_t rem = o;
            for (int l = order - 3; l >= 0; --l) {
                const int64_t il = rem % D.d[l];
                rem /= D.d[l];
                if (l != skip) w *= F.a[l][il * r + p];
            }
        }
        W[idx] = w;
    }
}

__global__ void k_reduce(const ReduceParams P, int64_t n_out, float* __restrict__ out) {
    const int64_t n = n_out * P.r;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x)
        out[idx] = reduce_output(P, idx / P.r, (int)(idx % P.r));
}

static int grid_for(int64_t n, int threads) {
    int64_t b = ceil_div(n, threads);
    if (b > 4096) b = 4096;
    if (b < 1) b = 1;
    return (int)b;
}

ReduceParams make_reduce_params(const TensorView& v, const MttkrpPlan& P, const float* part, const float* W) {
    ReduceParams R{};
    R.kind = P.kind == ModeKind::Inner ? 0 : P.kind == ModeKind::Outer ? 1 : 2;
    R.n_tiles = P.n_tiles;
    R.n_ot = P.n_ot;
    R.nb = P.nb;
    R.Ii = v.Ii;
    R.n_o = v.n_o;
    R.C = v.C;
    R.Cpad = P.Cpad;
    R.G = P.G;
    R.Smax = P.Smax;
    R.I_T = P.I_T;
    R.RP = P.RP;
    R.r = P.rank;
    R.part_warps = P.tc ? 1 : kStreamWarps;
    R.tile_slots = P.tile_slots ? 1 : 0;
    R.part = part;
    R.W = W;
    if (P.tile_slots) {
        // one slot per scheduled tile: a row tile's column segments are consecutive slots
        if (P.kind == ModeKind::Inner) R.n_ot = P.n_ot * P.n_cs;
        if (P.kind == ModeKind::Outer) R.nb = P.nb * P.n_cs;
    }
    if (P.kind == ModeKind::Outer) {
        R.In = v.dims[P.mode];
        int64_t stride = 1;
        for (int l = P.mode + 1; l < v.order - 2; ++l) stride *= v.dims[l];
        R.stride = stride;
        R.hi_count = v.n_o / (R.In * stride);
    }
    return R;
}

// ---------------------------------------------------------------------------
// launch sequence
// ---------------------------------------------------------------------------
// Inside a stream capture an event record has to be an external node to
// record anything when the graph runs; outside a capture a plain record.
static cudaError_t record_timer_event(cudaEvent_t ev, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return e;
    return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal)
                                               : cudaEventRecord(ev, st);
}

static ntf_status get_tensor_map(const TensorView& v, const MttkrpPlan& P, TmapCache* cache, CUtensorMap* local,
                                 const CUtensorMap** map) {
    if (cache && cache->valid && cache->data == v.data && cache->I_T == P.I_T && cache->O_T == P.O_T) {
        *map = &cache->map;
        return NTF_OK;
    }
    const uint32_t box0 = 128 / v.es;
    ntf_status s = encode_tensor_map_3d(local, v.dtype, v.data, (uint64_t)v.C, (uint64_t)v.Ii, (uint64_t)v.n_o,
                                        (uint64_t)(v.ld * v.es), (uint64_t)(v.Ii * v.ld * v.es), box0,
                                        (uint32_t)P.I_T, (uint32_t)P.O_T);
    if (s != NTF_OK) return s;
    *map = local;
    if (cache) {
        cache->valid = true;
        cache->data = v.data;
        cache->I_T = P.I_T;
        cache->O_T = P.O_T;
        cache->map = *local;
        *map = &cache->map;
    }
    return NTF_OK;
}

ntf_status run_mttkrp_stream(const TensorView& v, const MttkrpPlan& P, void* workspace, cudaStream_t st,
                             TmapCache* cache, StreamTimer* timer, bool pdl, const TcParams* fused) {
    unsigned char* ws = static_cast<unsigned char*>(workspace);
    CUtensorMap local_map;
    const CUtensorMap* map = nullptr;
    ntf_status s = get_tensor_map(v, P, cache, &local_map, &map);
    if (s != NTF_OK) return s;
    StreamParams S{};
    S.C = v.C;
    S.Ii = v.Ii;
    S.n_o = v.n_o;
    S.I_T = P.I_T;
    S.O_T = P.O_T;
    S.nb = P.nb;
    S.n_ot = P.n_ot;
    S.n_tiles = P.n_tiles;
    S.n_kc = P.n_kc;
    S.RP = P.RP;
    S.Smax = P.Smax;
    S.Cpad = P.Cpad;
    S.Fc = reinterpret_cast<const float*>(ws + P.off_Fc);
    S.Fi = reinterpret_cast<const float*>(ws + P.off_Fi);
    S.W = reinterpret_cast<const float*>(ws + P.off_W);
    S.part = reinterpret_cast<float*>(ws + P.off_part);
    S.err = device_error_word();
    const int kind = P.kind == ModeKind::Inner ? 0 : P.kind == ModeKind::Outer ? 1 : 2;
    dim3 grid;
    size_t smem;
    cudaError_t e;
    if (P.tc) {
        TcParams T{};
        T.C = v.C;
        T.Ii = v.Ii;
        T.n_o = v.n_o;
        T.I_T = P.I_T;
        T.O_T = P.O_T;
        T.nb = P.nb;
        T.n_ot = P.n_ot;
        T.n_tiles = P.tile_slots ? P.n_units : P.n_tiles;
        T.n_kc = P.n_kc;
        T.n_cs = P.n_cs;
        T.kc_per = P.kc_per;
        T.n_whole = P.n_whole;
        T.sched = P.tile_slots ? reinterpret_cast<unsigned int*>(ws + P.off_sched) : nullptr;
        T.RP = P.RP;
        T.r = P.rank;
        T.Smax = P.Smax;
        T.Cpad = P.Cpad;
        T.FcT = ws + P.off_Fc;
        T.Fi = S.Fi;
        T.W = S.W;
        T.ldw = P.RP;
        T.part = S.part;
        T.err = S.err;
        if (fused) {
            // operands chosen on the device, and the Gram job for the following epilogue
            T.ldw = fused->ldw;
            T.cur = fused->cur;
            for (int k = 0; k < 2; ++k) {
                T.FcTb[k] = fused->FcTb[k];
                T.Fib[k] = fused->Fib[k];
                T.Wb[k] = fused->Wb[k];
            }
            T.fct_sel = fused->fct_sel;
            T.fi_sel = fused->fi_sel;
            T.fi_flip = fused->fi_flip;
            T.w_sel = fused->w_sel;
            T.w_flip = fused->w_flip;
            T.job = fused->job;
            T.early = fused->early;
        }
        grid = P.kind == ModeKind::Last ? dim3(P.G, P.n_cb, 1) : dim3(P.G, 1, 1);
        smem = P.tf32 ? tf32_rows_smem(P.RPH) : P.kind == ModeKind::Last ? tc_last_smem(P.RPH) : tc_rows_smem(P.RPH);
        if (timer && timer->start) NTF_CUDA_TRY(record_timer_event(timer->start, st));
        e = P.tf32 ? launch_stream_tf32(kind, P.RPH, grid, smem, st, *map, T, pdl && !timer)
                   : launch_stream_tc(kind, P.RPH, grid, smem, st, *map, T, pdl && !timer);
    } else {
        if (P.kind == ModeKind::Last) {
            grid = dim3(P.G, P.n_cb, P.n_pb);
            smem = stream_last_smem(v.es, P.R);
        } else {
            grid = dim3(P.G, P.n_pb, 1);
            smem = stream_rows_smem(v.es, P.RP);
        }
        if (timer && timer->start) NTF_CUDA_TRY(record_timer_event(timer->start, st));
        e = v.dtype == NTF_F32 ? launch_stream_f32(kind, P.R, grid, smem, st, *map, S, pdl && !timer)
                               : launch_stream_bf16(kind, P.R, grid, smem, st, *map, S, pdl && !timer);
    }
    count_launch();
    if (e != cudaSuccess) return cuda_fail(e, "MTTKRP streaming kernel launch");
    if (timer && timer->stop) NTF_CUDA_TRY(record_timer_event(timer->stop, st));
    return NTF_OK;
}

ntf_status run_mttkrp(const TensorView& v, const MttkrpPlan& P, const float* const* factors, float* out,
                      void* workspace, cudaStream_t st, TmapCache* cache, StreamTimer* timer) {
    const int N = v.order, r = P.rank, n = P.mode;
    unsigned char* ws = static_cast<unsigned char*>(workspace);
    float* Fc = reinterpret_cast<float*>(ws + P.off_Fc);
    float* Fi = reinterpret_cast<float*>(ws + P.off_Fi);
    float* W = reinterpret_cast<float*>(ws + P.off_W);
    float* part = reinterpret_cast<float*>(ws + P.off_part);

    // 1. packed factors and weight table
    if (P.kind != ModeKind::Last) {
        if (P.tf32) {
            k_pack_fct_tf32<<<grid_for((int64_t)P.n_kc * 2 * P.RPH * 32, 256), 256, 0, st>>>(
                factors[N - 1], v.C, r, P.RPH, P.n_kc, Fc);
            NTF_LAUNCH_CHECK("k_pack_fct_tf32");
        } else if (P.tc) {
            k_pack_fct<<<grid_for((int64_t)P.n_kc * 2 * P.RPH * 64, 256), 256, 0, st>>>(
                factors[N - 1], v.C, r, P.RPH, P.n_kc, reinterpret_cast<__nv_bfloat16*>(Fc));
            NTF_LAUNCH_CHECK("k_pack_fct");
        } else {
            const int64_t rows_out = round_up(v.C, kStageCols);
            k_pack<<<grid_for(rows_out * P.RP, 256), 256, 0, st>>>(factors[N - 1], v.C, r, P.RP, rows_out, Fc);
            NTF_LAUNCH_CHECK("k_pack(A_last)");
        }
    }
    if (P.tf32 && P.kind == ModeKind::Last) {
        // TF32 operand of the last mode: A_{N-2} in 32-row chunks, one per tile row block
        k_pack_fct_tf32<<<grid_for((int64_t)P.nb * 2 * P.RPH * 32, 256), 256, 0, st>>>(factors[N - 2], v.Ii, r,
                                                                                          P.RPH, (int)P.nb, Fc);
        NTF_LAUNCH_CHECK("k_pack_fct_tf32(A_second_to_last)");
    } else if (P.tc && P.kind == ModeKind::Last) {
        // tensor-core operand of the last mode: A_{N-2} in 64-row chunks, two per 128-row block
        const int chunks = (int)(2 * P.nb);
        k_pack_fct<<<grid_for((int64_t)chunks * 2 * P.RPH * 64, 256), 256, 0, st>>>(
            factors[N - 2], v.Ii, r, P.RPH, chunks, reinterpret_cast<__nv_bfloat16*>(Fc));
        NTF_LAUNCH_CHECK("k_pack_fct(A_second_to_last)");
    } else if (P.kind != ModeKind::Inner) {
        k_pack<<<grid_for(v.Ii * P.RP, 256), 256, 0, st>>>(factors[N - 2], v.Ii, r, P.RP, v.Ii, Fi);
        NTF_LAUNCH_CHECK("k_pack(A_second_to_last)");
    }
    {
        FactorPtrs F{};
        Dims D{};
        for (int l = 0; l < N; ++l) {
            F.a[l] = factors[l];
            D.d[l] = v.dims[l];
        }
        const int skip = P.kind == ModeKind::Outer ? n : -1;
        k_weights<<<grid_for(v.n_o * P.RP, 256), 256, 0, st>>>(F, D, N, skip, r, P.RP, v.n_o, W);
        NTF_LAUNCH_CHECK("k_weights");
    }

    // 2. streaming kernel
    if (P.tile_slots) NTF_CUDA_TRY(cudaMemsetAsync(ws + P.off_sched, 0, sizeof(unsigned int), st));
    ntf_status s = run_mttkrp_stream(v, P, workspace, st, cache, timer);
    if (s != NTF_OK) return s;

    // 3. deterministic reduction into the user's I_n x r output
    ReduceParams R = make_reduce_params(v, P, part, W);
    const int64_t n_out = v.dims[n];
    k_reduce<<<grid_for(n_out * r, 128), 128, 0, st>>>(R, n_out, out);
    NTF_LAUNCH_CHECK("k_reduce");
    return NTF_OK;
}

}  // namespace ntf

namespace ntf {
cudaError_t launch_weights_all(const TensorView& v, const float* const* factors, int r, int RP, float* W,
                               cudaStream_t st) {
    FactorPtrs F{};
    Dims D{};
    for (int l = 0; l < v.order; ++l) {
        F.a[l] = factors[l];
        D.d[l] = v.dims[l];
    }
    k_weights<<<grid_for(v.n_o * RP, 256), 256, 0, st>>>(F, D, v.order, -1, r, RP, v.n_o, W);
    count_launch();
    return cudaGetLastError();
}
}  // namespace ntf

namespace ntf {
// Opt the streaming kernel of a plan in to its shared-memory size without
// launching it (so that no attribute call happens inside a graph capture).
ntf_status configure_mttkrp(const TensorView& v, const MttkrpPlan& P) {
    const int kind = P.kind == ModeKind::Inner ? 0 : P.kind == ModeKind::Outer ? 1 : 2;
    CUtensorMap dummy;
    std::memset(&dummy, 0, sizeof(dummy));
    if (P.tf32) {
        TcParams T{};
        cudaError_t e = launch_stream_tf32(kind, P.RPH, dim3(0, 1, 1), tf32_rows_smem(P.RPH), nullptr, dummy, T);
        if (e != cudaSuccess) return cuda_fail(e, "configure MTTKRP kernel");
        return NTF_OK;
    }
    if (P.tc) {
        TcParams T{};
        const size_t smem = P.kind == ModeKind::Last ? tc_last_smem(P.RPH) : tc_rows_smem(P.RPH);
        cudaError_t e = launch_stream_tc(kind, P.RPH, dim3(0, 1, 1), smem, nullptr, dummy, T);
        if (e != cudaSuccess) return cuda_fail(e, "configure MTTKRP kernel");
        return NTF_OK;
    }
    const size_t smem = P.kind == ModeKind::Last ? stream_last_smem(v.es, P.R) : stream_rows_smem(v.es, P.RP);
    StreamParams S{};
    cudaError_t e = v.dtype == NTF_F32 ? launch_stream_f32(kind, P.R, dim3(0, 1, 1), smem, nullptr, dummy, S)
                                       : launch_stream_bf16(kind, P.R, dim3(0, 1, 1), smem, nullptr, dummy, S);
    if (e != cudaSuccess) return cuda_fail(e, "configure MTTKRP kernel");
    return NTF_OK;
}
}  // namespace ntf
