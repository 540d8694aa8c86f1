// Internal interface of the MTTKRP launcher (step a1).
#pragma once

#include "ntf_common.cuh"
#include "mttkrp_reduce.cuh"

namespace ntf {

// Tensor view shared by the MTTKRP, residual and norm kernels.
struct TensorView {
    int order = 0;
    int64_t dims[NTF_MAX_ORDER] = {0};
    ntf_dtype dtype = NTF_F32;
    int64_t ld = 0;      // row pitch of the last mode, elements
    int es = 4;          // element size, bytes
    const void* data = nullptr;
    int64_t C = 0, Ii = 0, n_o = 0;   // last dim, second-to-last dim, product of the others
    int64_t rows() const { return Ii * n_o; }
    int64_t numel() const { return rows() * C; }
};

// Validates an ntf_tensor and fills the view (NTF_EINVAL with a message on error).
ntf_status make_view(const ntf_tensor* T, TensorView* v);

enum class ModeKind { Inner, Outer, Last };

struct MttkrpPlan {
    ModeKind kind;
    bool tc;             // tcgen05 kernels (bf16 storage, or fp32 rows modes via TF32; rank <= 32)
    bool tf32;           // ... the 3xTF32 rows kernel for fp32 storage
    int RPH;             // tc: rank rounded up to 8 (B operand holds hi | lo, N = 2 RPH)
    int mode, rank, RP, R, n_pb;
    int I_T, O_T;
    int64_t nb, n_ot, n_tiles;   // row tiles
    int n_kc;
    int n_cs = 1, kc_per = 0;    // tensor-core row kernels: column segments per row tile, chunks per segment
    // tensor-core row kernels: scheduled units.  Units below n_whole are whole row tiles (their
    // other segment slots are written as zeros); the rest are single segments of the row tiles
    // from n_whole on.  n_units = n_whole + (n_tiles - n_whole) n_cs.
    int64_t n_whole = 0, n_units = 0;
    int G;               // streaming CTAs along the tile axis
    int n_cb;            // last mode: 64-column blocks
    int Smax;
    bool tile_slots;     // one partial-sum slot per tile (tensor-core row kernels, scheduled at run time)
    int64_t Cpad;
    // workspace layout (byte offsets)
    size_t off_Fc, off_Fi, off_W, off_part, off_sched, total;   // off_Fc holds FcT (bf16) on the tc path
};

ntf_status plan_mttkrp(const TensorView& v, int rank, int mode, MttkrpPlan* plan);

// Cached 3-D tensor map of T for a plan's tile shape.
struct TmapCache {
    bool valid = false;
    const void* data = nullptr;
    int I_T = 0, O_T = 0;
    CUtensorMap map;
};

// Optional CUDA-event timing of the streaming kernel.
struct StreamTimer {
    cudaEvent_t start = nullptr, stop = nullptr;
};

ntf_status run_mttkrp(const TensorView& v, const MttkrpPlan& plan, const float* const* factors, float* out,
                      void* workspace, cudaStream_t st, TmapCache* cache, StreamTimer* timer);

int num_sms();

// Packed tensor-core operand of the Khatri-Rao product of two factors (a merged pair of modes):
// rows ka * Ib + kb, factors read from buffer cur[sel] ^ flip of each pair (cur NULL: a[0], b[0]).
struct KrPack {
    const float* a[2];
    const float* b[2];
    const int* cur;
    int sel_a, flip_a, sel_b, flip_b;
    int64_t Ia, Ib;
    int r, RPH, n_kc, tf32;
    void* out;
};
cudaError_t launch_pack_kr(const KrPack& K, cudaStream_t st);
ReduceParams make_reduce_params(const TensorView& v, const MttkrpPlan& P, const float* part, const float* W);
ntf_status configure_mttkrp(const TensorView& v, const MttkrpPlan& P);

}  // namespace ntf
