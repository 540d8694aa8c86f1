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

// Epilogue CTA: 4 rows of mode n, 8 warps.  Output M(j, p) of row j is the sum of
// two pieces of the stream's partials, taken by warp j and warp j + 4 (lane p);
// the HALS sweep of row j then runs on warp j alone.
constexpr int kEpiWarps = 8;
constexpr int kEpiRows = 4;                              // rows per CTA
constexpr int kEpiPieces = kEpiWarps / kEpiRows;         // partial-sum pieces per output

// Element (row i, column nn of 2 RPH) of the 3xTF32 operand: 32-row chunks of 2 RPH rows x
// 128 B, 16-byte groups swizzled as a 128-byte-swizzled TMA box; columns [0, RPH) hold tf32(x),
// [RPH, 2 RPH) hold tf32(x - tf32(x)).  (FP32 word index.)
__device__ __forceinline__ int64_t packed_index_tf32(int64_t i, int nn, int rph) {
    const int N = 2 * rph;
    const int64_t kc = i >> 5;
    const int kl = (int)(i & 31);
    return ((kc * N + nn) * 128 + (((kl >> 2) ^ (nn & 7)) << 4) + (kl & 3) * 4) / 4;
}

// write row `row`, column `lane` of the next stream's operand (bf16 hi | lo or TF32 hi | lo)
__device__ __forceinline__ void pack_store(__nv_bfloat16* dst, int64_t row, int lane, int rph, int tf32, float x) {
    if (tf32) {
        float* f = reinterpret_cast<float*>(dst);
        const float hi = tf32_rna(x);
        f[packed_index_tf32(row, lane, rph)] = hi;
        f[packed_index_tf32(row, rph + lane, rph)] = tf32_rna(x - hi);
    } else {
        const __nv_bfloat16 hi = __float2bfloat16_rn(x);
        dst[packed_index(row, lane, rph)] = hi;
        dst[packed_index(row, rph + lane, rph)] = __float2bfloat16_rn(x - __bfloat162float(hi));
    }
}

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

// pairing factor A_hat_l as seen by the update of mode n (eq. NNLS_her_exact):
// modes already updated in this iteration use their extrapolated buffer;
// cbuf holds the current buffer index of every mode
__device__ __forceinline__ const float* pairing_factor_c(const FusedBufs& B, int l, int n, const int* cbuf) {
    const int c = cbuf[l];
    return (B.her && l < n) ? B.X[l][1 - c] : B.X[l][c];
}

// ---------------------------------------------------------------------------
// prep
// ---------------------------------------------------------------------------
__global__ void k_prep(const PrepParams P) {
    pdl_wait();
    pdl_trigger();
    const int rr = P.r * P.r;
    const int n = P.mode;
    const FusedBufs& B = P.B;
    if (P.sched && blockIdx.x == 0 && threadIdx.x == 0) *P.sched = 0u;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // Control words first, all loads in flight together: the current buffer of
    // every mode (lane l holds mode l's), the iteration count and the last decision.
    const int cur_l = lane < P.order ? B.cur[lane] : 0;
    const int iters = *B.iters;
    const int last_restart = P.her ? P.her->last_restart : 1;
    int cbuf[NTF_MAX_ORDER];
#pragma unroll
    for (int l = 0; l < NTF_MAX_ORDER; ++l) cbuf[l] = __shfl_sync(0xffffffffu, cur_l, l);
    // Gram finishing for fin_mode; at mode 0 only once an iteration has completed
    const bool end_of_iter = n == 0;
    const bool fin = P.fin_mode >= 0 && (!end_of_iter || iters > 0);
    const bool two = fin && !end_of_iter && B.her;     // mid-iteration with HER: Grams of A and A_hat
    // at the end of an iteration the kept Gram of the last mode: A_hat's after an accept, else A's
    const bool keep_hat = end_of_iter && B.her && last_restart == 0;

    // (1) the finished Grams of fin_mode and V_n: one warp per entry q, the
    // warps of different blocks first.  The partials of both Grams and both
    // buffers of every other mode's Gram are loaded before anything is chosen.
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    for (int q = blockIdx.x + gridDim.x * warp; q < rr; q += nwarps) {
        float pa = 0.f, ph = 0.f;
        const float* base = P.gpart + q;
        for (int b = lane; b < P.fin_blocks; b += 32) {
            pa += base[(int64_t)(2 * b) * rr];
            if (B.her) ph += base[(int64_t)(2 * b + 1) * rr];
        }
        // lane 2l + k: entry q of the Gram held in buffer k of mode l
        const int gl_mode = lane >> 1, gl_buf = lane & 1;
        const double gq = (gl_mode < P.order && gl_mode != n) ? B.GB[gl_mode][gl_buf][q] : 0.0;
        pa = warp_allsum_f(pa);
        ph = warp_allsum_f(ph);
        double gsel[NTF_MAX_ORDER];
#pragma unroll
        for (int l = 0; l < NTF_MAX_ORDER; ++l) {
            // the pairing buffer of mode l (eq. NNLS_her_exact): A_hat for modes already updated
            const int k = (B.her && l < n) ? 1 - cbuf[l] : cbuf[l];
            const double g0 = __shfl_sync(0xffffffffu, gq, 2 * l);
            const double g1 = __shfl_sync(0xffffffffu, gq, 2 * l + 1);
            gsel[l] = k ? g1 : g0;
        }
        if (lane == 0) {
            double v = 1.0;
#pragma unroll
            for (int l = 0; l < NTF_MAX_ORDER; ++l) {
                if (l >= P.order || l == n) continue;
                double gl = gsel[l];
                if (fin && l == P.fin_mode) {
                    const int c = cbuf[l];
                    const double gA = (double)((end_of_iter && keep_hat) ? ph : pa);
                    B.GB[l][c][q] = gA;   // the kept factor (end of iteration) or A_{n-1}
                    gl = gA;
                    if (two) {
                        gl = (double)ph;   // A_hat_{n-1} pairs with mode n
                        B.GB[l][1 - c][q] = gl;
                    }
                }
                v *= gl;
            }
            P.V[q] = v;
            P.Vf[q] = (float)v;
        }
    }
    // (2) packed factors and weights
    const float* src_fc = P.Fc ? pairing_factor_c(B, P.order - 1, n, cbuf)
                               : P.FcT ? pairing_factor_c(B, P.fct_mode, n, cbuf) : nullptr;
    const float* src_fi = P.Fi ? pairing_factor_c(B, P.order - 2, n, cbuf) : nullptr;
    const int64_t nFc = P.Fc ? P.Fc_rows_out * P.RP : P.FcT ? (int64_t)P.n_kc * 2 * P.RPH * (P.fct_tf32 ? 32 : 64) : 0;
    const int64_t nFi = P.Fi ? P.Ii * P.RP : 0;
    const int64_t nW = P.W ? P.n_o * P.RP : 0;
    const int64_t total = nFc + nFi + nW;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t k = idx;
        if (k < nFc) {
            if (P.Fc) {
                const float* src = src_fc;
                const int64_t i = k / P.RP;
                const int p = (int)(k % P.RP);
                P.Fc[k] = (i < P.C && p < P.r) ? src[i * P.r + p] : 0.f;
            } else if (P.fct_tf32) {
                // 3xTF32 B operand: F_hi | F_lo = tf32(F), tf32(F - F_hi) as FP32 words, 32-row chunks of 128-byte rows
                const float* src = src_fc;
                const int N = 2 * P.RPH;
                const int kl = (int)(k % 32);
                const int nn = (int)((k / 32) % N);
                const int64_t kc = k / (32 * (int64_t)N);
                const int64_t i = kc * 32 + kl;
                const int p = nn < P.RPH ? nn : nn - P.RPH;
                const float x = (i < P.fct_rows && p < P.r) ? src[i * P.r + p] : 0.f;
                const float hi = tf32_rna(x);
                reinterpret_cast<float*>(P.FcT)[((kc * N + nn) * 128 + (((kl >> 2) ^ (nn & 7)) << 4) + (kl & 3) * 4) / 4] =
                    nn < P.RPH ? hi : tf32_rna(x - hi);
            } else {
                // tensor-core B operand: bf16 hi | lo columns, 128-byte rows, swizzled like a TMA box
                const float* src = src_fc;
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
            const float* src = src_fi;
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
#pragma unroll
                for (int l = NTF_MAX_ORDER - 3; l >= 0; --l) {
                    if (l > P.order - 3) continue;
                    const int64_t il = rem % P.dims[l];
                    rem /= P.dims[l];
                    if (l != P.skip) w *= pairing_factor_c(B, l, n, cbuf)[il * P.r + p];
                }
            }
            P.W[k] = w;
        }
    }
}

cudaError_t launch_prep(const PrepParams& P, cudaStream_t st, bool pdl) {
    const int64_t total = (int64_t)32 * P.r * P.r +
                          (P.Fc ? P.Fc_rows_out * P.RP : P.FcT ? (int64_t)P.n_kc * 2 * P.RPH * (P.fct_tf32 ? 32 : 64) : 0) +
                          (P.Fi ? P.Ii * P.RP : 0) + (P.W ? P.n_o * P.RP : 0);
    int64_t g = (total + 255) / 256;
    if (g > 2 * num_sms()) g = 2 * num_sms();
    if (g < 8) g = 8;
    cudaError_t e = launch_kernel(k_prep, dim3((unsigned)g), dim3(256), 0, st, pdl, P);
    count_launch();
    return e;
}

// ---------------------------------------------------------------------------
// epilogue
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kEpiWarps * 32) k_epilogue(const EpiParams P) {
    __shared__ float Vs[32 * 33];
    __shared__ float rinv[32];
    __shared__ float rowsA[kEpiRows][32];
    __shared__ float rowsH[kEpiRows][32];
    __shared__ float mpiece[kEpiPieces - 1][kEpiRows][32];
    __shared__ float winner[kEpiWarps];
    __shared__ double dred[kEpiWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = P.r, n = P.mode;
    const bool her = P.B.her != 0;
    const int rw = warp % kEpiRows, piece = warp / kEpiRows;
    const int64_t row = (int64_t)blockIdx.x * kEpiRows + rw;
    const bool live = row < P.rows && lane < r;
    // Read before the wait for the stream: the current buffer index, the factor row,
    // V and beta.  They were written two or more launches back, and this launch starts
    // only after the stream's own wait has seen those launches complete -- or, after an
    // early stream (TcParams::early), while the epilogue two launches back may still run,
    // which the host allows only where that epilogue writes none of them.  Loads go to
    // L2 (ld.global.cg), never to a possibly older L1 copy.
    const int cn = __ldcg(P.B.cur + n);
    float* A = P.B.X[n][cn];                      // in: A_{k-1}, out: A_k
    float* Ah = her ? P.B.X[n][1 - cn] : nullptr; // out: A_hat_k
    if (!P.v_from_stream) {
        for (int q = threadIdx.x; q < 32 * 32; q += blockDim.x) {
            const int l = q >> 5, c = q & 31;
            Vs[l * 33 + c] = (l < r && c < r) ? __ldcg(P.Vf + l * r + c) : 0.f;
        }
    }
    const float beta = her ? (float)__ldcg(P.beta) : 0.f;
    const float a_old = (live && piece == 0) ? __ldcg(A + row * r + lane) : 0.f;
    pdl_wait();
    pdl_trigger();
    if (P.v_from_stream) {
        // V was formed by the stream this kernel follows: read it only after the wait
        for (int q = threadIdx.x; q < 32 * 32; q += blockDim.x) {
            const int l = q >> 5, c = q & 31;
            Vs[l * 33 + c] = (l < r && c < r) ? __ldcg(P.Vf + l * r + c) : 0.f;
        }
    }

    if (P.sched_next && blockIdx.x == 0 && threadIdx.x == 0) *P.sched_next = 0u;
    // M row pieces from the stream's partial sums
    float m = live ? reduce_piece(P.red, row, lane, piece, kEpiPieces) : 0.f;
    if (piece > 0) mpiece[piece - 1][rw][lane] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        const float d = Vs[threadIdx.x * 33 + threadIdx.x];
        rinv[threadIdx.x] = (threadIdx.x < r && d > 0.f) ? 1.f / d : 0.f;
    }
    float a = a_old, ah = 0.f, inner = 0.f;
    if (piece == 0) {
#pragma unroll
        for (int k = 0; k < kEpiPieces - 1; ++k) m += mpiece[k][rw][lane];
    }
    __syncthreads();
    if (piece == 0) {
        // residual g_p = M_p - sum_l a_l V(l,p), lane p
        float g = m;
        for (int l = 0; l < r; ++l) g = fmaf(-__shfl_sync(0xffffffffu, a, l), Vs[l * 33 + lane], g);
        // one HALS sweep: a_j <- max(0, M_j - sum_{l != j} a_l V_lj) / V_jj = max(0, g_j + a_j V_jj) / V_jj
        for (int jj = 0; jj < r; ++jj) {
            const float vjj = Vs[jj * 33 + jj];
            const float rj = rinv[jj];
            float delta = 0.f;
            if (lane == jj && rj > 0.f) {
                const float nv = fmaxf(fmaf(a, vjj, g), 0.f) * rj;
                delta = nv - a;
                a = nv;
            }
            delta = __shfl_sync(0xffffffffu, delta, jj);
            g = fmaf(-delta, Vs[jj * 33 + lane], g);
        }
        ah = a;
        if (live) {
            A[row * r + lane] = a;
            if (her) {
                ah = fmaxf(fmaf(beta, a - a_old, a), 0.f);
                Ah[row * r + lane] = ah;
            }
            inner = m * a;
            // the next stream's tensor-core operand: hi | lo of this row
            __nv_bfloat16* pa = P.packA[cn];
            __nv_bfloat16* ph = her ? P.packH[1 - cn] : nullptr;
            if (pa) pack_store(pa, row, lane, P.pack_rph, P.pack_tf32, a);
            if (ph) pack_store(ph, row, lane, P.pack_rph, P.pack_tf32, ah);
        }
        rowsA[rw][lane] = live ? a : 0.f;
        rowsH[rw][lane] = live ? ah : 0.f;
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
    // everything the decision reads is loaded before anything is stored, so the
    // loads are in flight together
    double isum = 0.0, qsum = 0.0;
    for (int b = lane; b < (int)gridDim.x; b += 32) {
        isum += __ldcg(P.ipart + b);
        qsum += __ldcg(P.qpart + b);
    }
    const double tn = __ldcg(P.tnorm);
    const int it = __ldcg(P.iters_out);
    const int cl = lane < P.order ? __ldcg(P.B.cur + lane) : 0;
    ntf_her_state hs{};
    if (P.her) {
        hs.beta = __ldcg(&P.her->beta);
        hs.beta_bar = __ldcg(&P.her->beta_bar);
        hs.f_hat_prev = __ldcg(&P.her->f_hat_prev);
        hs.gamma = __ldcg(&P.her->gamma);
        hs.gamma_bar = __ldcg(&P.her->gamma_bar);
        hs.eta = __ldcg(&P.her->eta);
        hs.iters = __ldcg(&P.her->iters);
        hs.restarts = __ldcg(&P.her->restarts);
    }
    isum = warp_sum_dd(isum);
    qsum = warp_sum_dd(qsum);
    const double fhat = tn - 2.0 * isum + qsum;
    // Alg. 2: restart if F_hat_k > F_hat_{k-1}; a non-finite F_hat restarts and is flagged
    const bool finite = isfinite(fhat);
    const int restart = (!finite || fhat > hs.f_hat_prev) ? 1 : 0;
    if (P.her && !restart && lane < P.order) P.B.cur[lane] = 1 - cl;   // keep A_hat_k: A_k <- A_hat_k
    if (lane != 0) return;
    *P.ticket = 0;
    *P.fhat_out = fhat;
    *P.iters_out = it + 1;
    if (!P.her) return;
    ntf_her_state* out = P.her;
    if (restart) {
        out->beta_bar = hs.beta;
        out->beta = hs.beta / hs.eta;
    } else {
        out->beta_bar = fmin(1.0, hs.gamma_bar * hs.beta_bar);
        out->beta = fmin(hs.beta_bar, hs.gamma * hs.beta);
    }
    out->f_hat_prev = fhat;
    out->iters = hs.iters + 1;
    out->restarts = hs.restarts + restart;
    out->last_restart = restart;
    if (!finite) out->numeric_error = 1;
}

int epilogue_blocks(int64_t rows) { return (int)((rows + kEpiRows - 1) / kEpiRows); }

cudaError_t launch_epilogue(const EpiParams& P, cudaStream_t st, bool pdl) {
    cudaError_t e = launch_kernel(k_epilogue, dim3((unsigned)epilogue_blocks(P.rows)), dim3(kEpiWarps * 32), 0, st,
                                  pdl, P);
    count_launch();
    return e;
}

}  // namespace ntf
