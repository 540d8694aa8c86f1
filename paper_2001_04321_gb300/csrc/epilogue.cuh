// Fused prep / epilogue kernels of the solver's main path (see epilogue.cu).
#pragma once

#include "mttkrp.cuh"

namespace ntf {

struct PrepParams {
    int order, mode, skip, r, RP;
    int64_t C, Ii, n_o, Fc_rows_out;
    int64_t dims[NTF_MAX_ORDER];
    const float* A[NTF_MAX_ORDER];     // factors entering the MTTKRP (the pairing A_hat)
    const double* Gh[NTF_MAX_ORDER];   // their Grams
    double* V;                          // r x r, or nullptr
    float* Fc;                          // packed last-mode factor, or nullptr
    float* Fi;                          // packed second-to-last factor, or nullptr
    float* W;                           // weight table, or nullptr
};

struct EpiParams {
    ReduceParams red;
    int64_t rows;
    int r;
    float* A;              // in: A_{k-1}^n, out: A_k^n
    float* Ah;             // out: A_hat_k^n (nullptr without HER)
    const double* beta;    // device beta_{k-1}
    const double* V;       // r x r
    float* gpart;          // [blocks][2][r*r]
    double* ipart;         // [blocks]
    unsigned* ticket;      // zero between launches
    double* G_out;         // Gram of A_k^n
    double* Gh_out;        // Gram of A_hat_k^n (nullptr without HER)
    int last;              // 1 for mode N-1: objective and restart decision
    const double* tnorm;
    double* fhat_out;
    ntf_her_state* her;    // nullptr without HER
};

cudaError_t launch_prep(const PrepParams& P, cudaStream_t st);
cudaError_t launch_epilogue(const EpiParams& P, cudaStream_t st);
int epilogue_blocks(int64_t rows);

// streaming kernel of a plan alone (the packed factors / W already in place)
ntf_status run_mttkrp_stream(const TensorView& v, const MttkrpPlan& P, void* workspace, cudaStream_t st,
                             TmapCache* cache, StreamTimer* timer);

}  // namespace ntf
