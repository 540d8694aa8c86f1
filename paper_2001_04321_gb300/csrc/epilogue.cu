// Fused per-mode kernels of the solver's main path (HALS with one sweep per
// block update, rank <= 32):
//
//   k_prep      V_n = Hadamard product of the Grams of A_hat_l, l != n (Appendix A),
//               packed factors and the weight table W for the MTTKRP stream;
//   k_epilogue  per row j of mode n: M(j,:) from the stream's partial sums (a1),
//               one HALS sweep (Sec. 2.1.4, Gauss-Seidel over columns), the HER
//               extrapolation (Alg. 2, eq. extproj_her), per-CTA partial Grams of
//               A and A_hat (a2); the last CTA to finish (atomic ticket, no
//               waiting) sums the Grams in FP64 and, for the last mode, forms
//               F_hat = ||T||^2 - 2<M,A> + sum(V (*) A^T A) (Sec. 3.1, a5) and
//               takes the restart decision of Alg. 2 (a6).
//
// One warp owns rows: lane p holds column p of the row, so the HALS column
// update is a warp-wide dot product.  Every sum has a fixed order.
#include "epilogue.cuh"

namespace ntf {

constexpr int kEpiWarps = 8;
constexpr int kEpiRowsPerWarp = 4;
constexpr int kEpiRows = kEpiWarps * kEpiRowsPerWarp;   // rows per CTA

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

__device__ __forceinline__ double warp_sum_dd(double v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// ---------------------------------------------------------------------------
// prep
// ---------------------------------------------------------------------------
__global__ void k_prep(const PrepParams P) {
    const int64_t nV = P.V ? (int64_t)P.r * P.r : 0;
    const int64_t nFc = P.Fc ? P.Fc_rows_out * P.RP : 0;
    const int64_t nFi = P.Fi ? P.Ii * P.RP : 0;
    const int64_t nW = P.W ? P.n_o * P.RP : 0;
    const int64_t total = nV + nFc + nFi + nW;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t k = idx;
        if (k < nV) {
            double v = 1.0;
            for (int l = 0; l < P.order; ++l)
                if (l != P.mode) v *= P.Gh[l][k];
            P.V[k] = v;
            continue;
        }
        k -= nV;
        if (k < nFc) {
            const int64_t i = k / P.RP;
            const int p = (int)(k % P.RP);
            P.Fc[k] = (i < P.C && p < P.r) ? P.A[P.order - 1][i * P.r + p] : 0.f;
            continue;
        }
        k -= nFc;
        if (k < nFi) {
            const int64_t i = k / P.RP;
            const int p = (int)(k % P.RP);
            P.Fi[k] = p < P.r ? P.A[P.order - 2][i * P.r + p] : 0.f;
            continue;
        }
        k -= nFi;
        {
            const int64_t o = k / P.RP;
            const int p = (int)(k % P.RP);
            float w = 0.f;
            if (p < P.r) {
                w = 1.f;
                int64_t rem = o;
                for (int l = P.order - 3; l >= 0; --l) {
                    const int64_t il = rem % P.dims[l];
                    rem /= P.dims[l];
                    if (l != P.skip) w *= P.A[l][il * P.r + p];
                }
            }
            P.W[k] = w;
        }
    }
}

cudaError_t launch_prep(const PrepParams& P, cudaStream_t st) {
    const int64_t total = (P.V ? (int64_t)P.r * P.r : 0) + (P.Fc ? P.Fc_rows_out * P.RP : 0) +
                          (P.Fi ? P.Ii * P.RP : 0) + (P.W ? P.n_o * P.RP : 0);
    int64_t g = (total + 255) / 256;
    if (g > 2 * num_sms()) g = 2 * num_sms();
    if (g < 1) g = 1;
    k_prep<<<(int)g, 256, 0, st>>>(P);
    count_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// epilogue
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kEpiWarps * 32) k_epilogue(const EpiParams P) {
    __shared__ float Vs[32 * 32];
    __shared__ float rowsA[kEpiRows][32];
    __shared__ float rowsH[kEpiRows][32];
    __shared__ float winner[kEpiWarps];
    __shared__ double sred[kEpiWarps];
    __shared__ int is_last;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = P.r;
    const bool her = P.Ah != nullptr;
    for (int q = threadIdx.x; q < 32 * 32; q += blockDim.x) {
        const int l = q >> 5, c = q & 31;
        Vs[q] = (l < r && c < r) ? (float)P.V[l * r + c] : 0.f;
    }
    const float beta = her ? (float)*P.beta : 0.f;

    // M rows from the stream's partial sums (independent loads, issued up front)
    int64_t row[kEpiRowsPerWarp];
    float m[kEpiRowsPerWarp], a[kEpiRowsPerWarp], a_old[kEpiRowsPerWarp];
#pragma unroll
    for (int k = 0; k < kEpiRowsPerWarp; ++k) {
        row[k] = (int64_t)blockIdx.x * kEpiRows + warp * kEpiRowsPerWarp + k;
        const bool live = row[k] < P.rows && lane < r;
        m[k] = live ? reduce_output(P.red, row[k], lane) : 0.f;
        a_old[k] = live ? P.A[row[k] * r + lane] : 0.f;
        a[k] = a_old[k];
    }
    __syncthreads();

    // one HALS sweep per row: a_j <- max(0, M_j - sum_{l != j} a_l V_lj) / V_jj, j = 0..r-1
    for (int jj = 0; jj < r; ++jj) {
        const float vlj = Vs[lane * 32 + jj];
        const float vjj = Vs[jj * 32 + jj];
        float t[kEpiRowsPerWarp];
#pragma unroll
        for (int k = 0; k < kEpiRowsPerWarp; ++k) t[k] = lane != jj ? a[k] * vlj : 0.f;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
#pragma unroll
            for (int k = 0; k < kEpiRowsPerWarp; ++k) t[k] += __shfl_xor_sync(0xffffffffu, t[k], off);
        if (lane == jj && vjj > 0.f) {
#pragma unroll
            for (int k = 0; k < kEpiRowsPerWarp; ++k) a[k] = fmaxf(m[k] - t[k], 0.f) / vjj;
        }
    }

    float inner = 0.f;
#pragma unroll
    for (int k = 0; k < kEpiRowsPerWarp; ++k) {
        const bool live = row[k] < P.rows && lane < r;
        float ah = a[k];
        if (live) {
            P.A[row[k] * r + lane] = a[k];
            if (her) {
                ah = fmaxf(fmaf(beta, a[k] - a_old[k], a[k]), 0.f);
                P.Ah[row[k] * r + lane] = ah;
            }
            inner = fmaf(m[k], a[k], inner);
        }
        rowsA[warp * kEpiRowsPerWarp + k][lane] = live ? a[k] : 0.f;
        rowsH[warp * kEpiRowsPerWarp + k][lane] = live ? ah : 0.f;
    }
    inner = warp_sum_f(inner);
    if (lane == 0) winner[warp] = inner;
    __syncthreads();

    // per-CTA partial Grams (FP32 over this CTA's rows)
    const int rr = r * r;
    for (int q = threadIdx.x; q < rr; q += blockDim.x) {
        const int p = q / r, c = q % r;
        float sa = 0.f, sh = 0.f;
#pragma unroll 8
        for (int i = 0; i < kEpiRows; ++i) {
            sa = fmaf(rowsA[i][p], rowsA[i][c], sa);
            sh = fmaf(rowsH[i][p], rowsH[i][c], sh);
        }
        P.gpart[((int64_t)blockIdx.x * 2 + 0) * rr + q] = sa;
        if (her) P.gpart[((int64_t)blockIdx.x * 2 + 1) * rr + q] = sh;
    }
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kEpiWarps; ++w) s += (double)winner[w];
        P.ipart[blockIdx.x] = s;
    }
    // the last CTA to arrive finishes the mode (classic fence + ticket; nobody waits)
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = (atomicAdd(P.ticket, 1u) == gridDim.x - 1) ? 1 : 0;
    __syncthreads();
    if (!is_last) return;
    __threadfence();

    const int nblk = gridDim.x;
    double quad = 0.0;
    for (int q = threadIdx.x; q < rr; q += blockDim.x) {
        double ga = 0.0, gh = 0.0;
        for (int b = 0; b < nblk; ++b) {
            ga += (double)P.gpart[((int64_t)b * 2 + 0) * rr + q];
            if (her) gh += (double)P.gpart[((int64_t)b * 2 + 1) * rr + q];
        }
        P.G_out[q] = ga;
        if (her) P.Gh_out[q] = gh;
        quad += P.V[q] * ga;
    }
    if (P.last) {
        quad = warp_sum_dd(quad);
        if (lane == 0) sred[warp] = quad;
        __syncthreads();
        if (threadIdx.x == 0) {
            double qsum = 0.0, isum = 0.0;
            for (int w = 0; w < kEpiWarps; ++w) qsum += sred[w];
            for (int b = 0; b < nblk; ++b) isum += P.ipart[b];
            const double fhat = *P.tnorm - 2.0 * isum + qsum;
            *P.fhat_out = fhat;
            if (her) {
                // Alg. 2: restart if F_hat_k > F_hat_{k-1}; a non-finite F_hat restarts and is flagged
                ntf_her_state* s = P.her;
                const double b0 = s->beta, bb = s->beta_bar;
                const bool finite = isfinite(fhat);
                const bool restart = !finite || fhat > s->f_hat_prev;
                if (restart) {
                    s->beta_bar = b0;
                    s->beta = b0 / s->eta;
                } else {
                    s->beta_bar = fmin(1.0, s->gamma_bar * bb);
                    s->beta = fmin(bb, s->gamma * b0);
                }
                s->f_hat_prev = fhat;
                s->iters += 1;
                s->restarts += restart ? 1 : 0;
                s->last_restart = restart ? 1 : 0;
                if (!finite) s->numeric_error = 1;
            }
        }
    }
    if (threadIdx.x == 0) *P.ticket = 0u;
}

int epilogue_blocks(int64_t rows) { return (int)((rows + kEpiRows - 1) / kEpiRows); }

cudaError_t launch_epilogue(const EpiParams& P, cudaStream_t st) {
    k_epilogue<<<epilogue_blocks(P.rows), kEpiWarps * 32, 0, st>>>(P);
    count_launch();
    return cudaGetLastError();
}

}  // namespace ntf
