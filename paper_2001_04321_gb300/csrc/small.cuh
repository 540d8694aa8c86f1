// Internal launchers of the non-streaming kernels (steps a2-a8).
#pragma once

#include "mttkrp.cuh"

namespace ntf {

struct GramPtrs {
    const double* g[NTF_MAX_ORDER];
};

// factor pairs (A, A_hat) and Gram pairs (G(A), G(A_hat)) touched by a HER decision
struct CopyPairs {
    int count = 0;
    float* a[NTF_MAX_ORDER];
    float* ah[NTF_MAX_ORDER];
    int64_t n[NTF_MAX_ORDER];
    int gcount = 0;
    double* g[NTF_MAX_ORDER];
    double* gh[NTF_MAX_ORDER];
    int gn = 0;
};

size_t gram_smem(int r);
cudaError_t launch_gram(const float* A, int64_t rows, int r, double* G, cudaStream_t st);
// the same Gram over several CTAs for many rows (parts: gram_parts_bytes; NULL = one CTA)
size_t gram_parts_bytes(int64_t rows, int r);
cudaError_t launch_gram_parts(const float* A, int64_t rows, int r, double* G, double* parts, cudaStream_t st);
cudaError_t launch_hadamard(const GramPtrs& P, int order, int skip, int r, double* V, cudaStream_t st);

size_t bcd_workspace(int64_t rows, int r);
cudaError_t launch_bcd(int method, float* A, int64_t rows, int r, const float* M, const double* V, int inner_max,
                       double tol, void* ws, cudaStream_t st);

cudaError_t launch_wait_check(int64_t limit_ns, int* err, cudaStream_t st);
cudaError_t launch_block_gradient(const float* A, int64_t rows, int r, const float* M, const double* V,
                                  const double* scale_dev, double scale, float* out, cudaStream_t st);
cudaError_t launch_extrapolate(const float* A, const float* Ap, const double* beta, int64_t n, float* Ah,
                               cudaStream_t st);

// out = *tn - 2<M,A> + sum(V (*) A^T A); optionally stores A^T A in G_out
cudaError_t launch_objective(const double* tn, const float* M, const float* A, int64_t rows, int r, const double* V,
                             double* out, double* G_out, cudaStream_t st, const double* G_in = nullptr);

int stream_red_blocks();
cudaError_t launch_sum_parts(const double* parts, int n, double* out, cudaStream_t st);   // fixed order
cudaError_t launch_add(float* y, const float* x, int64_t n, cudaStream_t st);              // y += x
// copy of v with the trailing modes [split, N) first: (I_split..I_{N-1}, I_0..I_{split-1}), the
// last mode of the copy (I_{split-1}) with row pitch ld_dst
bool permute_split_fits(const TensorView& v, int split);
cudaError_t launch_permute_split(const TensorView& v, int split, void* dst, int64_t ld_dst, cudaStream_t st);
// 3-way tensor with its modes reversed, (I_2, I_1, I_0), rows pitched by ld_dst
bool permute_rev3_fits(const TensorView& v);
cudaError_t launch_permute_rev3(const TensorView& v, void* dst, int64_t ld_dst, cudaStream_t st);
cudaError_t launch_norm_sq(const TensorView& v, double* parts, double* out, cudaStream_t st);
cudaError_t launch_residual_sq(const TensorView& v, int r, const float* W, int RP, const float* Ai, const float* Ac,
                               double* parts, double* out, cudaStream_t st);
cudaError_t launch_to_bf16(const float* src, int64_t rows, int64_t C, int64_t ld_src, void* dst, int64_t ld_dst,
                           cudaStream_t st);

cudaError_t launch_her_init(ntf_her_state* s, double beta0, double gamma, double gamma_bar, double eta,
                            const double* f0, cudaStream_t st);
cudaError_t launch_her_step(ntf_her_state* s, const double* fhat, const CopyPairs& P, cudaStream_t st);
cudaError_t launch_her_copy(const ntf_her_state* s, const CopyPairs& P, cudaStream_t st);

// W(o,p) for the residual: product over all modes < N-2 (packed width RP)
cudaError_t launch_weights_all(const TensorView& v, const float* const* factors, int r, int RP, float* W,
                               cudaStream_t st);

}  // namespace ntf
