// Device pieces shared by the solver's fused kernels (epilogue.cu, mttkrp_tc.cu):
// finishing a mode's Grams from the epilogue CTAs' partials and forming
// V_n = Hadamard product of the pairing Grams (Appendix A), and the packed
// bf16 hi | lo layout of a factor as the tensor-core kernels read it.
#pragma once

#include "ntf_common.cuh"

namespace ntf {

// Grams of fin_mode finished from the partials of fin_blocks epilogue CTAs, and V of
// `mode` (the update whose pairing factors they are).  At the end of an iteration
// (mode 0) the last mode's kept Gram is A_hat's after an accept, else A's.
struct GramJob {
    int rr;                     // r * r entries; 0: no job
    int order, mode, fin_mode, fin_blocks, her;
    const float* gpart;         // [blocks][2][r*r]: partial Grams of A and A_hat
    double* GB[NTF_MAX_ORDER][2];
    double* V;                  // r x r
    float* Vf;                  // r x r, FP32 copy
    const int* cur;             // current buffer of every mode
    const int* iters;           // outer iterations completed
    const ntf_her_state* hs;    // the last decision (nullptr without HER)
};

#ifdef __CUDACC__
__device__ __forceinline__ float warp_allsum(float v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// One warp per entry q: warp `widx` of `nw` participating warps.  The partials of both
// Grams and both buffers of every other mode's Gram are loaded before anything is
// chosen; sums are FP32 butterflies in a fixed order (Gram entries of nonnegative
// factors are sums of nonnegative terms), the product V is FP64.
__device__ __forceinline__ void gram_job_run(const GramJob& J, int widx, int nw) {
    if (J.rr == 0) return;
    const int lane = threadIdx.x & 31;
    const int n = J.mode, rr = J.rr;
    const int cur_l = lane < J.order ? __ldcg(J.cur + lane) : 0;
    const int iters = __ldcg(J.iters);
    const int last_restart = J.hs ? __ldcg(&J.hs->last_restart) : 1;
    int cbuf[NTF_MAX_ORDER];
#pragma unroll
    for (int l = 0; l < NTF_MAX_ORDER; ++l) cbuf[l] = __shfl_sync(0xffffffffu, cur_l, l);
    const bool end_of_iter = n == 0;
    const bool fin = J.fin_mode >= 0 && (!end_of_iter || iters > 0);
    const bool two = fin && !end_of_iter && J.her;     // mid-iteration with HER: Grams of A and A_hat
    const bool keep_hat = end_of_iter && J.her && last_restart == 0;
    for (int q = widx; q < rr; q += nw) {
        float pa = 0.f, ph = 0.f;
        if (fin) {
            const float* base = J.gpart + q;
            for (int b = lane; b < J.fin_blocks; b += 32) {
                pa += __ldcg(base + (int64_t)(2 * b) * rr);
                if (J.her) ph += __ldcg(base + (int64_t)(2 * b + 1) * rr);
            }
        }
        // lane 2l + k: entry q of the Gram held in buffer k of mode l
        const int gl_mode = lane >> 1, gl_buf = lane & 1;
        const double gq = (gl_mode < J.order && gl_mode != n) ? __ldcg(J.GB[gl_mode][gl_buf] + q) : 0.0;
        pa = warp_allsum(pa);
        ph = warp_allsum(ph);
        double gsel[NTF_MAX_ORDER];
#pragma unroll
        for (int l = 0; l < NTF_MAX_ORDER; ++l) {
            // the pairing buffer of mode l (eq. NNLS_her_exact): A_hat for modes already updated
            const int k = (J.her && l < n) ? 1 - cbuf[l] : cbuf[l];
            const double g0 = __shfl_sync(0xffffffffu, gq, 2 * l);
            const double g1 = __shfl_sync(0xffffffffu, gq, 2 * l + 1);
            gsel[l] = k ? g1 : g0;
        }
        if (lane == 0) {
            double v = 1.0;
#pragma unroll
            for (int l = 0; l < NTF_MAX_ORDER; ++l) {
                if (l >= J.order || l == n) continue;
                double gl = gsel[l];
                if (fin && l == J.fin_mode) {
                    const int c = cbuf[l];
                    const double gA = (double)((end_of_iter && keep_hat) ? ph : pa);
                    J.GB[l][c][q] = gA;   // the kept factor (end of iteration) or A_{n-1}
                    gl = gA;
                    if (two) {
                        gl = (double)ph;   // A_hat_{n-1} pairs with mode n
                        J.GB[l][1 - c][q] = gl;
                    }
                }
                v *= gl;
            }
            J.V[q] = v;
            J.Vf[q] = (float)v;
        }
    }
}

// Element (row i, column nn of 2 RPH) of the tensor-core operand: 64-row chunks of
// 2 RPH rows x 128 B each, 16-byte groups swizzled as a 128-byte-swizzled TMA box;
// columns [0, RPH) hold bf16(x), columns [RPH, 2 RPH) hold bf16(x - bf16(x)).
__device__ __forceinline__ int64_t packed_index(int64_t i, int nn, int rph) {
    const int N = 2 * rph;
    const int64_t kc = i >> 6;
    const int kl = (int)(i & 63);
    return ((kc * N + nn) * 128 + (((kl >> 3) ^ (nn & 7)) << 4) + (kl & 7) * 2) / 2;
}
#endif

}  // namespace ntf
