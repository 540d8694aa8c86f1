// Tucker-format data (Appendix A): the tensor (U_0 (x) ... (x) U_{N-1}) G given by a small
// core G and bases U_p, never expanded.  Internal interface shared by tucker.cu and the solver.
#pragma once

#include "mttkrp.cuh"

namespace ntf {

constexpr int kTuckerMaxRank = 64;   // Tucker ranks r_p (the core's dims) are at most this

struct TuckerView {
    int order = 0;
    int64_t dims[NTF_MAX_ORDER] = {0};   // n_p: rows of U_p (the expanded tensor's dims)
    TensorView core;                     // G, dims r_p, FP32
    const float* U[NTF_MAX_ORDER] = {nullptr};
};

// Validates an ntf_tucker (pointers are checked by the caller) and fills the view.
ntf_status make_tucker_view(const ntf_tucker* X, TuckerView* v);

// Workspace layout of one MTTKRP of the Tucker-format tensor (byte offsets).
struct TuckerPlan {
    int mode = 0, rank = 0;
    MttkrpPlan core;                 // the core's MTTKRP
    size_t off_W[NTF_MAX_ORDER];     // W_p = U_p^T A_p, r_p x rank floats
    size_t off_part;                 // projection partial sums
    size_t off_Y;                    // core MTTKRP, r_mode x rank floats
    size_t off_core;                 // the core MTTKRP's own workspace
    size_t total;
};

ntf_status plan_tucker_mttkrp(const TuckerView& v, int rank, int mode, TuckerPlan* P);

// out (dims[mode] x rank) <- U_mode MTTKRP(G, {U_p^T A_p}, mode)
ntf_status run_tucker_mttkrp(const TuckerView& v, const TuckerPlan& P, const float* const* factors, float* out,
                             void* workspace, cudaStream_t st, TmapCache* cache);

size_t tucker_norm_workspace(const TuckerView& v);
// *out <- ||(U_0 (x) ... (x) U_{N-1}) G||_F^2 = <G, G x_0 Q_0 ... x_{N-1} Q_{N-1}>, Q_p = U_p^T U_p
ntf_status run_tucker_norm_sq(const TuckerView& v, double* out, void* workspace, cudaStream_t st);

}  // namespace ntf
