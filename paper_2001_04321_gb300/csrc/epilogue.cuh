// Fused prep / epilogue / finish kernels of the solver's main path (see epilogue.cu).
#pragma once

#include "fused.cuh"
#include "mttkrp.cuh"
#include "mttkrp_tc.cuh"
#include "small.cuh"

namespace ntf {

// Two buffers per mode for the factor and its Gram.  At the start of every
// iteration A_l and A_hat_l are equal (Alg. 2 sets one to the other) and live
// in X[l][cur[l]]; during the iteration mode l's update writes A_l there and
// A_hat_l to X[l][1 - cur[l]] (with HER).  Accepting the extrapolation flips
// cur[l]; restarting keeps it.  No factor is ever copied.
struct FusedBufs {
    float* X[NTF_MAX_ORDER][2];
    double* GB[NTF_MAX_ORDER][2];   // Gram of the factor in X[l][k]
    int* cur;                       // device: current buffer of each mode
    const int* iters;               // device: outer iterations completed (decisions taken)
    int her;
};

struct PrepParams {
    FusedBufs B;
    int order, mode, skip, r, RP;
    int64_t C, Ii, n_o, Fc_rows_out;
    int64_t dims[NTF_MAX_ORDER];
    double* V;                          // r x r
    float* Vf;                          // r x r, V rounded to FP32 (read by the epilogue's HALS sweep)
    float* Fc;                          // packed last-mode factor (FFMA stream), or nullptr
    __nv_bfloat16* FcT;                 // tensor-core operand (64-row chunks, bf16 hi|lo), or nullptr
    int fct_mode;                       // mode packed into FcT
    int64_t fct_rows;                   // its rows
    int RPH, n_kc;                      // n_kc: chunks of FcT (64 rows; 32 rows for tf32)
    int fct_tf32;                       // FcT in the 3xTF32 layout (FP32 words) instead of bf16
    float* Fi;                          // packed second-to-last factor (FFMA stream), or nullptr
    float* W;                           // weight table
    unsigned int* sched;                // tile counter of the next stream (set to 0 here), or nullptr
    // Grams of the mode updated just before (fin_mode) are finished here from the
    // epilogue partials; for mode 0 that is the last mode of the previous iteration
    int fin_mode, fin_blocks;
    const float* gpart;                 // [blocks][2][r*r]
    const ntf_her_state* her;           // decision of the previous iteration (mode-0 prep), or nullptr
};

struct EpiParams {
    FusedBufs B;
    ReduceParams red;
    int mode, order;
    int64_t rows;
    int r;
    int last;              // 1 for mode N-1: also partial sum(V (*) G(A)), then the end of the iteration
    const double* beta;    // device beta_{k-1}
    const double* V;       // r x r
    const float* Vf;       // r x r, FP32
    float* gpart;          // [blocks][2][r*r]: partial Grams of A and A_hat
    double* ipart;         // [blocks]: partial <M, A>
    double* qpart;         // [blocks]: partial sum(V (*) G(A)) (last mode)
    // end of the iteration (last mode only), taken by the CTA that finishes last:
    // F_hat, the restart decision of Alg. 2 and the buffer flip
    int* ticket;           // device counter, 0 between launches
    const double* tnorm;   // ||T||^2
    double* fhat_out;
    int* iters_out;        // outer-iteration counter
    ntf_her_state* her;    // nullptr without HER
    // fused 3-way tensor-core path: the operands of the next stream written here
    __nv_bfloat16* packA[2];   // A_k's rows go to packA[cur] (if set), in the tensor-core layout
    __nv_bfloat16* packH[2];   // A_hat_k's rows go to packH[1 - cur] (if set)
    int pack_rph;
    int pack_tf32;             // the 3xTF32 layout (FP32 words, 32-row chunks) instead of bf16 hi | lo
    unsigned int* sched_next;  // run-time tile counter of the next stream, set to 0 here (or nullptr)
    int v_from_stream;         // V is formed by the preceding stream (read after the wait)
};

cudaError_t launch_prep(const PrepParams& P, cudaStream_t st, bool pdl);
cudaError_t launch_epilogue(const EpiParams& P, cudaStream_t st, bool pdl);
int epilogue_blocks(int64_t rows);

// streaming kernel of a plan alone (the packed factors / W already in place)
// `fused` (tensor-core plans only): device-chosen operands and the Gram job (see TcParams)
ntf_status run_mttkrp_stream(const TensorView& v, const MttkrpPlan& P, void* workspace, cudaStream_t st,
                             TmapCache* cache, StreamTimer* timer, bool pdl = false,
                             const TcParams* fused = nullptr);

}  // namespace ntf
