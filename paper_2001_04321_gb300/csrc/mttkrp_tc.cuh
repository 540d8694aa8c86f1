// tcgen05 MTTKRP kernels for bf16 tensor storage (see mttkrp_tc.cu).
#pragma once

#include "fused.cuh"

#include "ntf_common.cuh"

namespace ntf {

struct TcParams {
    int64_t C, Ii, n_o;
    int I_T, O_T;
    int64_t nb, n_ot, n_tiles;      // n_tiles: scheduled units (see n_whole)
    int n_kc;
    int n_cs, kc_per;                // column segments (output slots) per row tile, chunks per segment
    int64_t n_whole;                 // units below n_whole are whole row tiles, the rest single segments
    int RP, r;
    int Smax;
    int64_t Cpad;
    const unsigned char* FcT;   // rows kernel: A_{N-1} per 64-row chunk; last kernel: A_{N-2} per 128-row
                                // block; N rows x 128 B per 64 rows, swizzled bf16 hi|lo
    const float* Fi;            // A_{N-2} rows (fp32), row stride ldw
    const float* W;             // n_o weight rows (fp32), row stride ldw
    int ldw;                    // RP for packed tables, r when W / Fi are factor rows
    float* part;                // rows kernels: one slot per tile; last kernel: one per CTA
    unsigned int* sched;        // rows kernels: next tile to hand out (0 before every launch)
    int* err;
    // fused solver path: operands chosen on the device from the current-buffer indices
    // (cur == nullptr: FcT, Fi and W are used as given)
    const int* cur;
    const unsigned char* FcTb[2];   // FcT = FcTb[cur[fct_sel]]
    const float* Fib[2];            // Fi = Fib[cur[fi_sel] ^ fi_flip]
    const float* Wb[2];             // W = Wb[cur[w_sel] ^ w_flip]
    int fct_sel, fi_sel, fi_flip, w_sel, w_flip;
    GramJob job;                    // Grams + V for the epilogue after this stream (job.rr == 0: none)
    // rows kernels: the producer and MMA warps read nothing the kernel before this one writes
    // (its operands and tile counter were written two or more kernels back), so only the
    // epilogue warps wait for it and the tensor streams in while it finishes
    int early;
};

size_t tc_rows_smem(int rph);
int tc_rows_ctas_per_sm();          // CTAs of the bf16 rows kernel that share an SM's tensor memory
size_t tc_last_smem(int rph);
size_t tc_last_b_bytes(int rph);
size_t tf32_rows_smem(int rph);
// TF32 rows kernels for FP32 tensors (kind 0 inner, 1 outer); FcT holds F_hi | F_lo
// as FP32 words in 32-row chunks (N rows x 128 B each, swizzled)
cudaError_t launch_stream_tf32(int kind, int rph, dim3 grid, size_t smem, cudaStream_t st, const CUtensorMap& map,
                               const TcParams& P, bool pdl = false);
cudaError_t launch_stream_tc(int kind, int rph, dim3 grid, size_t smem, cudaStream_t st, const CUtensorMap& map,
                             const TcParams& P, bool pdl = false);

}  // namespace ntf
