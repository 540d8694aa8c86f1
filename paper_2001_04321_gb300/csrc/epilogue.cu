// Fused per-mode kernels of the solver's main path (HALS with one sweep per
// block update, rank <= 32).  Per mode n:
//
//   k_prep      finishes the Grams of the mode updated just before (FP64 sums
//               of the epilogue's per-CTA partials; at mode 0 the last mode of
//               the previous iteration, kept or discarded by its restart
//               decision), forms V_n = Hadamard product of the Grams of the
//               pairing factors A_hat_l, l != n (Appendix A), and packs the
//               factors and the weight table W for the MTTKRP stream;
//   k_epilogue  per row j of mode n: M(j,:) from the stream's partial sums (a1),
//               one HALS sweep (Sec. 2.1.4, Gauss-Seidel over columns), the HER
//               extrapolation (Alg. 2, eq. extproj_her), and per-CTA partials of
//               the Grams of A and A_hat, of <M, A> and (last mode) of
//               sum(V (*) A^T A);
//
// and, in the CTA of the last mode's epilogue that finishes last, the end of
// the iteration: F_hat = ||T||^2 - 2<M,A> + sum(V (*) A^T A) from those
// partials (Sec. 3.1, a5), the restart decision of Alg. 2 (a6), and the
// accept/restart step as a flip of the current-buffer indices.
//
// GB300 runs FP64 at a small fraction of its FP32 rate (a dependent FP64 add
// costs about 70 cycles), so the per-entry sums here are FP32 butterflies in a
// fixed order, and FP64 is kept for the few scalars where cancellation matters.
//
// The HALS sweep keeps the residual g = M - A V of the row in the lanes (lane
// p holds column p): updating column j is one scalar step on lane j followed
// by one broadcast and one FMA per lane.  Every sum has a fixed order.
#include "epilogue.cuh"

namespace ntf {

constexpr int kEpiWarps = 8;
constexpr int kEpiRowsPerWarp = 2;
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

// butterfly sum over the lanes: every lane ends with the same value
__device__ __forceinline__ float warp_allsum_f(float v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Gram entry q (k = 0: A, 1: A_hat) from the epilogue CTAs' partials: lane u adds
// the partials of CTAs u, u + 32, ... in order, then a butterfly over the lanes.
// Every entry of a Gram of nonnegative factors is a sum of nonnegative terms,
// so FP32 summation keeps a relative error of a few units in the last place.
__device__ __forceinline__ float gram_entry(const float* gpart, int nblk, int rr, int k, int q, int lane) {
    const float* base = gpart + (int64_t)k * rr + q;
    const int64_t stride = 2 * (int64_t)rr;
    float s = 0.f;
    for (int b = lane; b < nblk; b += 32) s += base[(int64_t)b * stride];
    return warp_allsum_f(s);
}

// pairing factor A_hat_l as seen by the update of mode n (eq. NNLS_her_exact):
// modes already updated in this iteration use their extrapolated buffer
__device__ __forceinline__ const float* pairing_factor(const FusedBufs& B, int l, int n) {
    const int c = B.cur[l];
    return (B.her && l < n) ? B.X[l][1 - c] : B.X[l][c];
}
__device__ __forceinline__ const double* pairing_gram(const FusedBufs& B, int l, int n) {
    const int c = B.cur[l];
    return (B.her && l < n) ? B.GB[l][1 - c] : B.GB[l][c];
}

// ---------------------------------------------------------------------------
// prep
// ---------------------------------------------------------------------------
__global__ void k_prep(const PrepParams P) {
    const int rr = P.r * P.r;
    const int n = P.mode;
    const FusedBufs& B = P.B;
    // Gram finishing for fin_mode; at mode 0 only once an iteration has completed
    const bool end_of_iter = n == 0;
    const bool fin = P.fin_mode >= 0 && (!end_of_iter || *B.iters > 0);
    const bool two = fin && !end_of_iter && B.her;     // mid-iteration with HER: Grams of A and A_hat
    const int nVG = rr * (two ? 2 : 1);
    // (1) the finished Grams of fin_mode and V_n: one warp per entry q, the
    // warps of different blocks first
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    const int keep = (end_of_iter && B.her && P.her && P.her->last_restart == 0) ? 1 : 0;
    for (int q = blockIdx.x + gridDim.x * warp; q < rr; q += nwarps) {
        float sA = 0.f, sH = 0.f;
        if (fin) {
            sA = gram_entry(P.gpart, P.fin_blocks, rr, end_of_iter ? keep : 0, q, lane);
            if (two) sH = gram_entry(P.gpart, P.fin_blocks, rr, 1, q, lane);
        }
        if (lane == 0) {
            double v = 1.0;
            for (int l = 0; l < P.order; ++l) {
                if (l == n) continue;
                double gl;
                if (fin && l == P.fin_mode) {
                    const int c = B.cur[l];
                    // end of iteration: the kept factor (A on restart, A_hat on accept), already current;
                    // mid-iteration with HER: A_{n-1} is stored, A_hat_{n-1} pairs with mode n
                    B.GB[l][c][q] = (double)sA;
                    gl = (double)sA;
                    if (two) {
                        gl = (double)sH;
                        B.GB[l][1 - c][q] = gl;
                    }
                } else {
                    gl = pairing_gram(B, l, n)[q];
                }
                v *= gl;
            }
            P.V[q] = v;
            P.Vf[q] = (float)v;
        }
    }
    // (2) packed factors and weights
    const int64_t nFc = P.Fc ? P.Fc_rows_out * P.RP : P.FcT ? (int64_t)P.n_kc * 2 * P.RPH * 64 : 0;
    const int64_t nFi = P.Fi ? P.Ii * P.RP : 0;
    const int64_t nW = P.W ? P.n_o * P.RP : 0;
    const int64_t total = nFc + nFi + nW;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t k = idx;
        if (k < nFc) {
            if (P.Fc) {
                const float* src = pairing_factor(B, P.order - 1, n);
                const int64_t i = k / P.RP;
                const int p = (int)(k % P.RP);
                P.Fc[k] = (i < P.C && p < P.r) ? src[i * P.r + p] : 0.f;
            } else {
                // tensor-core B operand: bf16 hi | lo columns, 128-byte rows, swizzled like a TMA box
                const float* src = pairing_factor(B, P.fct_mode, n);
                const int N = 2 * P.RPH;
                const int kl = (int)(k % 64);
                const int nn = (int)((k / 64) % N);
                const int64_t kc = k / (64 * (int64_t)N);
                const int64_t i = kc * 64 + kl;
                const int p = nn < P.RPH ? nn : nn - P.RPH;
                const float x = (i < P.fct_rows && p < P.r) ? src[i * P.r + p] : 0.f;
                const __nv_bfloat16 hi = __float2bfloat16_rn(x);
                const __nv_bfloat16 v = nn < P.RPH ? hi : __float2bfloat16_rn(x - __bfloat162float(hi));
                P.FcT[((kc * N + nn) * 128 + (((kl >> 3) ^ (nn & 7)) << 4) + (kl & 7) * 2) / 2] = v;
            }
            continue;
        }
        k -= nFc;
        if (k < nFi) {
            const float* src = pairing_factor(B, P.order - 2, n);
            const int64_t i = k / P.RP;
            const int p = (int)(k % P.RP);
            P.Fi[k] = p < P.r ? src[i * P.r + p] : 0.f;
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
                    if (l != P.skip) w *= pairing_factor(B, l, n)[il * P.r + p];
                }
            }
            P.W[k] = w;
        }
    }
}

cudaError_t launch_prep(const PrepParams& P, cudaStream_t st) {
    const int64_t total = (int64_t)32 * P.r * P.r +
                          (P.Fc ? P.Fc_rows_out * P.RP : P.FcT ? (int64_t)P.n_kc * 2 * P.RPH * 64 : 0) +
                          (P.Fi ? P.Ii * P.RP : 0) + (P.W ? P.n_o * P.RP : 0);
    int64_t g = (total + 255) / 256;
    if (g > 2 * num_sms()) g = 2 * num_sms();
    if (g < 8) g = 8;
    k_prep<<<(int)g, 256, 0, st>>>(P);
    count_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// epilogue
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kEpiWarps * 32) k_epilogue(const EpiParams P) {
    __shared__ float Vs[32 * 33];
    __shared__ float rinv[32];
    __shared__ float rowsA[kEpiRows][32];
    __shared__ float rowsH[kEpiRows][32];
    __shared__ float winner[kEpiWarps];
    __shared__ double dred[kEpiWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = P.r, n = P.mode;
    const bool her = P.B.her != 0;
    const int cn = P.B.cur[n];
    float* A = P.B.X[n][cn];                      // in: A_{k-1}, out: A_k
    float* Ah = her ? P.B.X[n][1 - cn] : nullptr; // out: A_hat_k
    for (int q = threadIdx.x; q < 32 * 32; q += blockDim.x) {
        const int l = q >> 5, c = q & 31;
        Vs[l * 33 + c] = (l < r && c < r) ? P.Vf[l * r + c] : 0.f;
    }
    const float beta = her ? (float)*P.beta : 0.f;

    // M rows from the stream's partial sums, and the previous rows
    int64_t row[kEpiRowsPerWarp];
    float m[kEpiRowsPerWarp], a[kEpiRowsPerWarp], a_old[kEpiRowsPerWarp];
#pragma unroll
    for (int k = 0; k < kEpiRowsPerWarp; ++k) {
        row[k] = (int64_t)blockIdx.x * kEpiRows + warp * kEpiRowsPerWarp + k;
        const bool live = row[k] < P.rows && lane < r;
        a_old[k] = live ? A[row[k] * r + lane] : 0.f;
        m[k] = live ? reduce_output(P.red, row[k], lane) : 0.f;
        a[k] = a_old[k];
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const float d = Vs[threadIdx.x * 33 + threadIdx.x];
        rinv[threadIdx.x] = (threadIdx.x < r && d > 0.f) ? 1.f / d : 0.f;
    }
    __syncthreads();

    // residual g_p = M_p - sum_l a_l V(l,p), lane p
    float g[kEpiRowsPerWarp];
#pragma unroll
    for (int k = 0; k < kEpiRowsPerWarp; ++k) g[k] = m[k];
    for (int l = 0; l < r; ++l) {
        const float vlp = Vs[l * 33 + lane];
#pragma unroll
        for (int k = 0; k < kEpiRowsPerWarp; ++k) g[k] = fmaf(-__shfl_sync(0xffffffffu, a[k], l), vlp, g[k]);
    }
    // one HALS sweep: a_j <- max(0, M_j - sum_{l != j} a_l V_lj) / V_jj = max(0, g_j + a_j V_jj) / V_jj
    for (int jj = 0; jj < r; ++jj) {
        const float vjj = Vs[jj * 33 + jj];
        const float rj = rinv[jj];
        const float vjp = Vs[jj * 33 + lane];
#pragma unroll
        for (int k = 0; k < kEpiRowsPerWarp; ++k) {
            float delta = 0.f;
            if (lane == jj && rj > 0.f) {
                const float nv = fmaxf(fmaf(a[k], vjj, g[k]), 0.f) * rj;
                delta = nv - a[k];
                a[k] = nv;
            }
            delta = __shfl_sync(0xffffffffu, delta, jj);
            g[k] = fmaf(-delta, vjp, g[k]);
        }
    }

    float inner = 0.f;
#pragma unroll
    for (int k = 0; k < kEpiRowsPerWarp; ++k) {
        const bool live = row[k] < P.rows && lane < r;
        float ah = a[k];
        if (live) {
            A[row[k] * r + lane] = a[k];
            if (her) {
                ah = fmaxf(fmaf(beta, a[k] - a_old[k], a[k]), 0.f);
                Ah[row[k] * r + lane] = ah;
            }
            inner = fmaf(m[k], a[k], inner);
        }
        rowsA[warp * kEpiRowsPerWarp + k][lane] = live ? a[k] : 0.f;
        rowsH[warp * kEpiRowsPerWarp + k][lane] = live ? ah : 0.f;
    }
    inner = warp_sum_f(inner);
    if (lane == 0) winner[warp] = inner;
    __syncthreads();

    // per-CTA partial Grams (FP32 over this CTA's rows), <M, A>, and sum(V (*) G_cta)
    const int rr = r * r;
    double quad = 0.0;
    for (int q = threadIdx.x; q < rr; q += blockDim.x) {
        const int p = q / r, c = q % r;
        float sa = 0.f, sh = 0.f;
#pragma unroll
        for (int i = 0; i < kEpiRows; ++i) {
            sa = fmaf(rowsA[i][p], rowsA[i][c], sa);
            sh = fmaf(rowsH[i][p], rowsH[i][c], sh);
        }
        P.gpart[((int64_t)blockIdx.x * 2 + 0) * rr + q] = sa;
        if (her) P.gpart[((int64_t)blockIdx.x * 2 + 1) * rr + q] = sh;
        if (P.last) quad = fma(P.V[q], (double)sa, quad);
    }
    if (P.last) {
        quad = warp_sum_dd(quad);
        if (lane == 0) dred[warp] = quad;
    }
    __syncthreads();
    if (warp == 0) {
        // the CTA's sums over its 8 warps: 3-level butterflies on lanes 0..7
        double s = lane < kEpiWarps ? (double)winner[lane] : 0.0;
        double qs = (P.last && lane < kEpiWarps) ? dred[lane] : 0.0;
#pragma unroll
        for (int off = kEpiWarps / 2; off > 0; off >>= 1) {
            s += __shfl_xor_sync(0xffffffffu, s, off);
            qs += __shfl_xor_sync(0xffffffffu, qs, off);
        }
        if (lane == 0) {
            P.ipart[blockIdx.x] = s;
            if (P.last) P.qpart[blockIdx.x] = qs;
        }
    }
    if (!P.last) return;

    // end of the iteration, in the CTA that finishes last (its partials and every
    // other CTA's are visible after the fence / counter handshake)
    __shared__ int is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = atomicAdd(P.ticket, 1) == (int)gridDim.x - 1;
    __syncthreads();
    if (!is_last || warp != 0) return;
    __threadfence();
    double isum = 0.0, qsum = 0.0;
    for (int b = lane; b < (int)gridDim.x; b += 32) {
        isum += __ldcg(P.ipart + b);
        qsum += __ldcg(P.qpart + b);
    }
    isum = warp_sum_dd(isum);
    qsum = warp_sum_dd(qsum);
    if (lane != 0) return;
    *P.ticket = 0;
    const double fhat = *P.tnorm - 2.0 * isum + qsum;
    *P.fhat_out = fhat;
    *P.iters_out += 1;
    if (!P.her) return;
    // Alg. 2: restart if F_hat_k > F_hat_{k-1}; a non-finite F_hat restarts and is flagged
    ntf_her_state* hs = P.her;
    const double b0 = hs->beta, bb = hs->beta_bar;
    const bool finite = isfinite(fhat);
    const int restart = (!finite || fhat > hs->f_hat_prev) ? 1 : 0;
    if (restart) {
        hs->beta_bar = b0;
        hs->beta = b0 / hs->eta;
    } else {
        hs->beta_bar = fmin(1.0, hs->gamma_bar * bb);
        hs->beta = fmin(bb, hs->gamma * b0);
        // keep the extrapolated sequence: A_k <- A_hat_k for every block
        for (int l = 0; l < P.order; ++l) P.B.cur[l] = 1 - P.B.cur[l];
    }
    hs->f_hat_prev = fhat;
    hs->iters += 1;
    hs->restarts += restart;
    hs->last_restart = restart;
    if (!finite) hs->numeric_error = 1;
}

int epilogue_blocks(int64_t rows) { return (int)((rows + kEpiRows - 1) / kEpiRows); }

cudaError_t launch_epilogue(const EpiParams& P, cudaStream_t st) {
    k_epilogue<<<epilogue_blocks(P.rows), kEpiWarps * 32, 0, st>>>(P);
    count_launch();
    return cudaGetLastError();
}

}  // namespace ntf
