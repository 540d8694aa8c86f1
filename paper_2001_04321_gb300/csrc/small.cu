// Kernels of steps a2-a8 other than the MTTKRP stream: Grams and their
// Hadamard product (a2), HALS / projected-gradient block updates (a3), the HER
// extrapolation (a4), the objective by reuse (a5), the restart decision (a6),
// the explicit residual (a7), the bf16 cast (a8) and ||T||^2.
//
// GB300 runs FP64 at a small fraction of its FP32 rate, so every per-element
// product here is FP32; FP64 only combines short FP32 partial sums and holds
// the r x r Grams, the objective terms and the HER scalars.
#include "small.cuh"
#include "block_reduce.cuh"

#include <cmath>

namespace ntf {


// ---------------------------------------------------------------------------
// a2: Gram A^T A.  Rows are staged in shared memory in blocks (zero-padded to 4T columns,
// T = ceil(r / 4)).  Thread (tp, grp) owns the 4 x 4 tile pair tp = (a, b), a <= b, of the upper
// triangle and rows grp, grp + ngrp, ... of the block (at most 32 of them): 16 FP32 accumulators,
// two 16-byte shared loads per row.  The ngrp row groups are then added per entry in FP64 in
// group order, and the blocks in FP64 in block order.  Deterministic, no workspace.
// ---------------------------------------------------------------------------
constexpr int kGramThreads = 1024;

__host__ __device__ __forceinline__ int gram_tiles(int r) { return (r + 3) / 4; }
__host__ __device__ __forceinline__ int gram_tile_pairs(int r) { return gram_tiles(r) * (gram_tiles(r) + 1) / 2; }
__host__ __device__ __forceinline__ int gram_groups(int r) {
    const int g = kGramThreads / gram_tile_pairs(r);
    return g < 1 ? 1 : g;
}
// rows of one staged block: at most 32 per row group
__host__ __device__ __forceinline__ int gram_blk_rows(int r) {
    const int b = gram_groups(r) * 32;
    return b > 1024 ? 1024 : b;
}
__host__ __device__ __forceinline__ int gram_stride(int r) { return 4 * gram_tiles(r) + 4; }

__device__ __forceinline__ void pair_of(int q, int r, int& p, int& c) {
    p = 0;
    int rem = q;
    while (rem >= r - p) {
        rem -= r - p;
        ++p;
    }
    c = p + rem;
}

// acc[q] += entry q (upper triangle, row-major pair order) of the Gram of rows [r0, r0 + n) of
// A, n <= gram_blk_rows(r); sA holds max(n * stride, ngrp * ntp * 16) floats
__device__ void gram_chunk(const float* __restrict__ A, int64_t r0, int n, int r, float* sA, double* acc) {
    const int T = gram_tiles(r), S = gram_stride(r), ntp = gram_tile_pairs(r), ngrp = gram_groups(r);
    __syncthreads();
    for (int t = threadIdx.x; t < n * S; t += blockDim.x) {
        const int i = t / S, j = t - i * S;
        sA[t] = j < r ? A[(r0 + i) * r + j] : 0.f;
    }
    __syncthreads();
    const int tid = threadIdx.x;
    float x16[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) x16[e] = 0.f;
    const bool active = tid < ntp * ngrp;
    const int tp = tid % ntp, grp = tid / ntp;
    if (active) {
        int a, b;
        pair_of(tp, T, a, b);
        for (int i = grp; i < n; i += ngrp) {
            const float4 u = *reinterpret_cast<const float4*>(sA + i * S + 4 * a);
            const float4 v = *reinterpret_cast<const float4*>(sA + i * S + 4 * b);
            const float uu[4] = {u.x, u.y, u.z, u.w}, vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int e = 0; e < 16; ++e) x16[e] = fmaf(uu[e >> 2], vv[e & 3], x16[e]);
        }
    }
    __syncthreads();                       // sA is reused for the row-group partials
    if (active)
#pragma unroll
        for (int e = 0; e < 16; ++e) sA[(grp * ntp + tp) * 16 + e] = x16[e];
    __syncthreads();
    for (int idx = tid; idx < ntp * 16; idx += blockDim.x) {
        const int t2 = idx >> 4, e = idx & 15;
        int a, b;
        pair_of(t2, T, a, b);
        const int p = 4 * a + (e >> 2), c = 4 * b + (e & 3);
        if (p >= r || c >= r || p > c) continue;
        double s = 0.0;
        for (int g0 = 0; g0 < ngrp; g0 += 16) {          // FP32 over 16 groups, FP64 across
            float f = 0.f;
            const int g1 = g0 + 16 < ngrp ? g0 + 16 : ngrp;
            for (int g = g0; g < g1; ++g) f += sA[(g * ntp + t2) * 16 + e];
            s += (double)f;
        }
        acc[p * r - p * (p - 1) / 2 + (c - p)] += s;
    }
}

// shared memory of the Gram kernels: 2080 FP64 entries (r = 64) and the staged block / partials
size_t gram_smem(int r) {
    const size_t stage = (size_t)gram_blk_rows(r) * gram_stride(r);
    const size_t red = (size_t)gram_groups(r) * gram_tile_pairs(r) * 16;
    return sizeof(double) * 2080 + sizeof(float) * (stage > red ? stage : red);
}

// the whole Gram in one CTA (any number of rows)
__device__ void gram_cta(const float* __restrict__ A, int64_t rows, int r, float* sA, double* acc) {
    const int npairs = r * (r + 1) / 2;
    for (int q = threadIdx.x; q < npairs; q += blockDim.x) acc[q] = 0.0;
    const int blk = gram_blk_rows(r);
    for (int64_t r0 = 0; r0 < rows; r0 += blk) gram_chunk(A, r0, (int)(rows - r0 < blk ? rows - r0 : blk), r, sA, acc);
    __syncthreads();
}

__global__ void __launch_bounds__(kGramThreads) k_gram(const float* __restrict__ A, int64_t rows, int r,
                                                       double* __restrict__ G) {
    extern __shared__ __align__(16) unsigned char gram_smem_raw[];
    double* acc = reinterpret_cast<double*>(gram_smem_raw);
    float* sA = reinterpret_cast<float*>(gram_smem_raw + sizeof(double) * 2080);
    gram_cta(A, rows, r, sA, acc);
    const int npairs = r * (r + 1) / 2;
    for (int q = threadIdx.x; q < npairs; q += blockDim.x) {
        int p, c;
        pair_of(q, r, p, c);
        G[p * r + c] = acc[q];
        G[c * r + p] = acc[q];
    }
}


// Many-row Grams: one CTA per row block writes its entries to its own slot of partials;
// k_gram_sum adds the slots in block order.
__global__ void __launch_bounds__(kGramThreads) k_gram_part(const float* __restrict__ A, int64_t rows, int r,
                                                            double* __restrict__ parts) {
    extern __shared__ __align__(16) unsigned char gram_smem_raw[];
    double* acc = reinterpret_cast<double*>(gram_smem_raw);
    float* sA = reinterpret_cast<float*>(gram_smem_raw + sizeof(double) * 2080);
    const int blk = gram_blk_rows(r);
    const int npairs = r * (r + 1) / 2;
    for (int q = threadIdx.x; q < npairs; q += blockDim.x) acc[q] = 0.0;
    const int64_t r0 = (int64_t)blockIdx.x * blk;
    gram_chunk(A, r0, (int)(rows - r0 < blk ? rows - r0 : blk), r, sA, acc);
    __syncthreads();
    for (int q = threadIdx.x; q < npairs; q += blockDim.x) parts[(int64_t)blockIdx.x * npairs + q] = acc[q];
}

__global__ void k_gram_sum(const double* __restrict__ parts, int nblk, int r, double* __restrict__ G) {
    const int npairs = r * (r + 1) / 2;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= npairs) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += parts[(int64_t)b * npairs + q];
    int p, c;
    pair_of(q, r, p, c);
    G[p * r + c] = s;
    G[c * r + p] = s;
}

// the dynamic shared memory of the Gram and objective kernels (above 48 KB), set once
static cudaError_t configure_gram_kernels() {
    static bool done = false;
    if (done) return cudaSuccess;
    int bytes = 0;
    for (int r = 1; r <= NTF_MAX_RANK; ++r) bytes = (int)gram_smem(r) > bytes ? (int)gram_smem(r) : bytes;
    cudaError_t e = cudaFuncSetAttribute(k_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gram_part, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done = true;
    return e;
}

cudaError_t launch_gram(const float* A, int64_t rows, int r, double* G, cudaStream_t st) {
    cudaError_t e = configure_gram_kernels();
    if (e != cudaSuccess) return e;
    k_gram<<<1, kGramThreads, gram_smem(r), st>>>(A, rows, r, G);
    count_launch();
    return cudaGetLastError();
}

size_t gram_parts_bytes(int64_t rows, int r) {
    return sizeof(double) * (size_t)((rows + gram_blk_rows(r) - 1) / gram_blk_rows(r)) * (size_t)(r * (r + 1) / 2);
}

cudaError_t launch_gram_parts(const float* A, int64_t rows, int r, double* G, double* parts, cudaStream_t st) {
    const int blk = gram_blk_rows(r);
    if (!parts || rows <= 2 * (int64_t)blk) return launch_gram(A, rows, r, G, st);
    cudaError_t e = configure_gram_kernels();
    if (e != cudaSuccess) return e;
    const int nblk = (int)((rows + blk - 1) / blk);
    k_gram_part<<<nblk, kGramThreads, gram_smem(r), st>>>(A, rows, r, parts);
    count_launch();
    const int npairs = r * (r + 1) / 2;
    k_gram_sum<<<(npairs + 255) / 256, 256, 0, st>>>(parts, nblk, r, G);
    count_launch();
    return cudaGetLastError();
}

// V = Hadamard product of grams[l], l != skip
__global__ void k_hadamard(GramPtrs P, int order, int skip, int r, double* __restrict__ V) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < r * r; q += gridDim.x * blockDim.x) {
        double v = 1.0;
        for (int l = 0; l < order; ++l)
            if (l != skip) v *= P.g[l][q];
        V[q] = v;
    }
}

cudaError_t launch_hadamard(const GramPtrs& P, int order, int skip, int r, double* V, cudaStream_t st) {
    k_hadamard<<<(r * r + 255) / 256, 256, 0, st>>>(P, order, skip, r, V);
    count_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// gradient of (1/2)||T - X||^2 with respect to one factor (Sec. 2, eq. def:grad
// with Appendix A's Hadamard product): out = scale (A V - M), one row per thread
// ---------------------------------------------------------------------------
__global__ void k_block_gradient(const float* __restrict__ A, int64_t rows, int r, const float* __restrict__ M,
                                 const double* __restrict__ V, const double* __restrict__ scale_dev, double scale,
                                 float* __restrict__ out) {
    __shared__ float Vs[NTF_MAX_RANK * NTF_MAX_RANK];
    for (int q = threadIdx.x; q < r * r; q += blockDim.x) Vs[q] = (float)V[q];
    __syncthreads();
    const float sc = (float)(scale_dev ? *scale_dev * scale : scale);
    // one thread per entry (i, j): g = sum_l A(i,l) V(l,j) - M(i,j); the threads of a row read
    // A(i,:) together (broadcast) and consecutive columns of V
    const int64_t n = rows * r;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / r;
        const int j = (int)(idx - i * r);
        const float* a = A + i * r;
        float g = -M[idx];
        for (int l = 0; l < r; ++l) g = fmaf(a[l], Vs[l * r + j], g);
        out[idx] = sc * g;
    }
}

cudaError_t launch_block_gradient(const float* A, int64_t rows, int r, const float* M, const double* V,
                                  const double* scale_dev, double scale, float* out, cudaStream_t st) {
    int64_t g = (rows * r + 255) / 256;
    if (g > 1024) g = 1024;
    if (g < 1) g = 1;
    k_block_gradient<<<(int)g, 256, 0, st>>>(A, rows, r, M, V, scale_dev, scale, out);
    count_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// check of the bounded-wait path: one thread waits on an mbarrier that nothing
// arrives on, gives up after limit_ns, records the time-out code and returns
// ---------------------------------------------------------------------------
__global__ void k_wait_check(int64_t limit_ns, int* err) {
    __shared__ uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    fence_mbar_init();
    const uint64_t t0 = global_timer_ns();
    for (;;) {
        if (mbar_try_wait(&bar, 0)) return;                 // cannot happen: nothing arrives
        if (global_timer_ns() - t0 > (uint64_t)limit_ns) {
            record_device_error(err, kErrWaitFull);
            return;
        }
    }
}

cudaError_t launch_wait_check(int64_t limit_ns, int* err, cudaStream_t st) {
    k_wait_check<<<1, 32, 0, st>>>(limit_ns, err);
    count_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// a4: extrapolation  A_hat = max(0, A + beta (A - A_prev))
// ---------------------------------------------------------------------------
__global__ void k_extrapolate(const float* __restrict__ A, const float* __restrict__ Ap,
                              const double* __restrict__ beta, int64_t n, float* __restrict__ Ah) {
    const float b = (float)*beta;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float a = A[i];
        Ah[i] = fmaxf(fmaf(b, a - Ap[i], a), 0.f);
    }
}

cudaError_t launch_extrapolate(const float* A, const float* Ap, const double* beta, int64_t n, float* Ah,
                               cudaStream_t st) {
    int64_t g = (n + 255) / 256;
    if (g > 1024) g = 1024;
    if (g < 1) g = 1;
    k_extrapolate<<<(int)g, 256, 0, st>>>(A, Ap, beta, n, Ah);
    count_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// a5: objective by reuse:  ||T||^2 - 2 <M, A> + sum(V (*) A^T A)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kGramThreads) k_objective(const double* __restrict__ tn, const float* __restrict__ M,
                                                            const float* __restrict__ A, int64_t rows, int r,
                                                            const double* __restrict__ V, const double* __restrict__ G_in,
                                                            double* __restrict__ out, double* __restrict__ G_out) {
    extern __shared__ __align__(16) unsigned char gram_smem_raw[];
    __shared__ double sbuf[33];
    double* acc = reinterpret_cast<double*>(gram_smem_raw);
    float* sA = reinterpret_cast<float*>(gram_smem_raw + sizeof(double) * 2080);
    // <M, A>: thread t sums entries t, t + T, ... (coalesced), FP32 over 32 of them, then FP64
    const int64_t n = rows * r;
    const int64_t T = blockDim.x;
    double inner = 0.0;
    for (int64_t b = threadIdx.x; b < n; b += 32 * T) {
        float s = 0.f;
#pragma unroll 8
        for (int k = 0; k < 32; ++k) {
            const int64_t i = b + k * T;
            if (i < n) s = fmaf(M[i], A[i], s);
        }
        inner += (double)s;
    }
    inner = block_sum_d(inner, sbuf);
    // sum_pq V(p,q) G(p,q), G = A^T A: given (the caller's Gram of A) or formed here
    const int npairs = r * (r + 1) / 2;
    double quad = 0.0;
    if (G_in) {
        for (int q = threadIdx.x; q < r * r; q += blockDim.x) quad += V[q] * G_in[q];
    } else {
        gram_cta(A, rows, r, sA, acc);
        for (int q = threadIdx.x; q < npairs; q += blockDim.x) {
            int p, c;
            pair_of(q, r, p, c);
            quad += (p == c ? V[p * r + p] : V[p * r + c] + V[c * r + p]) * acc[q];
            if (G_out) {
                G_out[p * r + c] = acc[q];
                G_out[c * r + p] = acc[q];
            }
        }
    }
    quad = block_sum_d(quad, sbuf);
    if (threadIdx.x == 0) *out = *tn - 2.0 * inner + quad;
}

cudaError_t launch_objective(const double* tn, const float* M, const float* A, int64_t rows, int r, const double* V,
                             double* out, double* G_out, cudaStream_t st, const double* G_in) {
    const size_t smem = G_in ? 0 : gram_smem(r);
    static size_t set_bytes = 0;
    if (set_bytes == 0) {
        size_t most = 0;
        for (int q = 1; q <= NTF_MAX_RANK; ++q) most = gram_smem(q) > most ? gram_smem(q) : most;
        cudaError_t e = cudaFuncSetAttribute(k_objective, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most);
        if (e != cudaSuccess) return e;
        e = configure_gram_kernels();
        if (e != cudaSuccess) return e;
        set_bytes = most;
    }
    if (!M) return cudaSuccess;   // configuration only
    k_objective<<<1, kGramThreads, smem, st>>>(tn, M, A, rows, r, V, G_in, out, G_out);
    count_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// ||T||^2 and the explicit residual ||T - X||^2 (multi-CTA partials + final sum)
// ---------------------------------------------------------------------------
constexpr int kStreamRedThreads = 256;

// 16-byte vector of the stored type, unpacked to FP32 (bf16 -> f32 is exact)
template <typename TE>
struct Vec16;
template <>
struct Vec16<float> {
    static constexpr int n = 4;
    __device__ __forceinline__ static void unpack(const uint4& u, float* x) {
        x[0] = __uint_as_float(u.x);
        x[1] = __uint_as_float(u.y);
        x[2] = __uint_as_float(u.z);
        x[3] = __uint_as_float(u.w);
    }
};
template <>
struct Vec16<__nv_bfloat16> {
    static constexpr int n = 8;
    __device__ __forceinline__ static void unpack(const uint4& u, float* x) {
        const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            x[2 * k] = __uint_as_float(w[k] << 16);
            x[2 * k + 1] = __uint_as_float(w[k] & 0xffff0000u);
        }
    }
};

// ||T||^2: warp per row, 16-byte loads, four per lane in flight; the padding
// between C and ld is never summed
template <typename TE>
__global__ void __launch_bounds__(kStreamRedThreads) k_norm_sq(const TE* __restrict__ T, int64_t rows, int64_t C,
                                                               int64_t ld, double* __restrict__ parts) {
    __shared__ double sbuf[33];
    constexpr int E = Vec16<TE>::n;
    const int lane = threadIdx.x & 31;
    const int64_t warp_g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nv = (C + E - 1) / E;          // 16-byte vectors holding the row's C values
    double acc = 0.0;
    for (int64_t row = warp_g; row < rows; row += nwarps) {
        const uint4* rp = reinterpret_cast<const uint4*>(T + row * ld);
        for (int64_t v0 = lane; v0 < nv; v0 += 128) {
            uint4 u[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) u[k] = (v0 + 32 * k < nv) ? __ldg(rp + v0 + 32 * k) : make_uint4(0, 0, 0, 0);
            float s = 0.f;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                float x[E];
                Vec16<TE>::unpack(u[k], x);
                const int64_t c0 = (v0 + 32 * k) * E;
#pragma unroll
                for (int j = 0; j < E; ++j) s = (c0 + j < C) ? fmaf(x[j], x[j], s) : s;
            }
            acc += (double)s;
        }
    }
    const double tot = block_sum_d(acc, sbuf);
    if (threadIdx.x == 0) parts[blockIdx.x] = tot;
}

__global__ void k_sum_parts(const double* __restrict__ parts, int n, double* __restrict__ out) {
    __shared__ double sbuf[33];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += parts[i];
    acc = block_sum_d(acc, sbuf);
    if (threadIdx.x == 0) *out = acc;
}

int stream_red_blocks() { return 4 * num_sms(); }

cudaError_t launch_sum_parts(const double* parts, int n, double* out, cudaStream_t st) {
    k_sum_parts<<<1, 256, 0, st>>>(parts, n, out);
    count_launch();
    return cudaGetLastError();
}

// A second layout of a tensor with its trailing modes [split, N) moved to the front:
// D(i_split.., i_{N-1}, i_0.., i_{split-1}) = S(i_0, .., i_{N-1}), rows of D (the last index,
// i_{split-1}) with pitch ld_dst, the padding left as it is.  S is read as an R x C' matrix (R over
// the leading modes, C' over the trailing ones, whose last is pitched by ld) and written
// transposed, through 32 x 32 tiles in shared memory so that both sides are coalesced.
template <typename E>
__global__ void k_permute_split(const E* __restrict__ S, int64_t R, int64_t Cp, int64_t Cb, int64_t ld,
                                int64_t I_in, E* __restrict__ D, int64_t ld_dst) {
    __shared__ E tile[32][33];
    const int64_t c0 = (int64_t)blockIdx.x * 32, r0 = (int64_t)blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;     // 32 x 8 threads
    const int64_t row_stride = (Cp / Cb) * ld;         // one leading index: all trailing entries
    for (int k = ty; k < 32; k += 8) {
        const int64_t row = r0 + k, c = c0 + tx;
        if (row < R && c < Cp) tile[k][tx] = S[row * row_stride + (c / Cb) * ld + (c % Cb)];
    }
    __syncthreads();
    const int64_t R_out = R / I_in;                    // leading modes other than the last one
    for (int k = ty; k < 32; k += 8) {
        const int64_t c = c0 + k, row = r0 + tx;
        if (row < R && c < Cp) {
            const int64_t i0 = row / I_in, i1 = row - i0 * I_in;
            D[(c * R_out + i0) * ld_dst + i1] = tile[tx][k];
        }
    }
}

bool permute_split_fits(const TensorView& v, int split) {
    int64_t R = 1;
    for (int l = 0; l < split; ++l) R *= v.dims[l];
    return split >= 1 && split < v.order && (R + 31) / 32 <= 65535;
}

cudaError_t launch_permute_split(const TensorView& v, int split, void* dst, int64_t ld_dst, cudaStream_t st) {
    int64_t R = 1, Cp = 1;
    for (int l = 0; l < split; ++l) R *= v.dims[l];
    for (int l = split; l < v.order; ++l) Cp *= v.dims[l];
    const int64_t Cb = v.dims[v.order - 1], I_in = v.dims[split - 1];
    const dim3 grid((unsigned)((Cp + 31) / 32), (unsigned)((R + 31) / 32));
    if (v.es == 4)
        k_permute_split<uint32_t><<<grid, dim3(32, 8), 0, st>>>(static_cast<const uint32_t*>(v.data), R, Cp, Cb, v.ld,
                                                               I_in, static_cast<uint32_t*>(dst), ld_dst);
    else
        k_permute_split<uint16_t><<<grid, dim3(32, 8), 0, st>>>(static_cast<const uint16_t*>(v.data), R, Cp, Cb, v.ld,
                                                               I_in, static_cast<uint16_t*>(dst), ld_dst);
    count_launch();
    return cudaGetLastError();
}

// The 3-way tensor with its modes reversed: D(i_2, i_1, i_0) = S(i_0, i_1, i_2), rows of D (the
// i_0 index) with pitch ld_dst, the padding left as it is.  For each i_1 the I_0 x I_2 plane
// is transposed through 32 x 32 tiles in shared memory, so both sides are coalesced.
template <typename E>
__global__ void k_permute_rev3(const E* __restrict__ S, int64_t I0, int64_t I1, int64_t I2, int64_t ld,
                               E* __restrict__ D, int64_t ld_dst) {
    __shared__ E tile[32][33];
    const int64_t c0 = (int64_t)blockIdx.x * 32, r0 = (int64_t)blockIdx.y * 32;   // i_2, i_0 blocks
    const int tx = threadIdx.x, ty = threadIdx.y;                                    // 32 x 8 threads
    for (int64_t i1 = blockIdx.z; i1 < I1; i1 += gridDim.z) {
        for (int k = ty; k < 32; k += 8) {
            const int64_t i0 = r0 + k, i2 = c0 + tx;
            if (i0 < I0 && i2 < I2) tile[k][tx] = S[(i0 * I1 + i1) * ld + i2];
        }
        __syncthreads();
        for (int k = ty; k < 32; k += 8) {
            const int64_t i2 = c0 + k, i0 = r0 + tx;
            if (i0 < I0 && i2 < I2) D[(i2 * I1 + i1) * ld_dst + i0] = tile[tx][k];
        }
        __syncthreads();
    }
}

bool permute_rev3_fits(const TensorView& v) {
    return v.order == 3 && (v.dims[2] + 31) / 32 <= 2147483647 && (v.dims[0] + 31) / 32 <= 65535;
}

cudaError_t launch_permute_rev3(const TensorView& v, void* dst, int64_t ld_dst, cudaStream_t st) {
    const int64_t I0 = v.dims[0], I1 = v.dims[1], I2 = v.dims[2];
    const dim3 grid((unsigned)((I2 + 31) / 32), (unsigned)((I0 + 31) / 32), (unsigned)(I1 < 65535 ? I1 : 65535));
    if (v.es == 4)
        k_permute_rev3<uint32_t><<<grid, dim3(32, 8), 0, st>>>(static_cast<const uint32_t*>(v.data), I0, I1, I2, v.ld,
                                                              static_cast<uint32_t*>(dst), ld_dst);
    else
        k_permute_rev3<uint16_t><<<grid, dim3(32, 8), 0, st>>>(static_cast<const uint16_t*>(v.data), I0, I1, I2, v.ld,
                                                              static_cast<uint16_t*>(dst), ld_dst);
    count_launch();
    return cudaGetLastError();
}

// y += x elementwise (the slab partials of a streamed MTTKRP, summed in slab order)
__global__ void k_add(float* __restrict__ y, const float* __restrict__ x, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] += x[i];
}

cudaError_t launch_add(float* y, const float* x, int64_t n, cudaStream_t st) {
    k_add<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(y, x, n);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_norm_sq(const TensorView& v, double* parts, double* out, cudaStream_t st) {
    const int G = stream_red_blocks();
    if (v.dtype == NTF_F32)
        k_norm_sq<float><<<G, kStreamRedThreads, 0, st>>>(static_cast<const float*>(v.data), v.rows(), v.C, v.ld,
                                                          parts);
    else
        k_norm_sq<__nv_bfloat16><<<G, kStreamRedThreads, 0, st>>>(static_cast<const __nv_bfloat16*>(v.data),
                                                                  v.rows(), v.C, v.ld, parts);
    count_launch();
    k_sum_parts<<<1, 256, 0, st>>>(parts, G, out);
    count_launch();
    return cudaGetLastError();
}

// Explicit residual ||T - X||^2 with X(o, i, c) = sum_p W(o,p) A_{N-2}(i,p) A_{N-1}(c,p).
// A CTA takes blocks of 64 rows (o, i); per chunk of CW columns A_{N-1}^T is staged
// in shared memory, and each lane computes a 4-row x 4-column tile of X (16 FMAs
// per p from one float4 of A_{N-1}^T and one broadcast float4 of the 4 rows'
// Khatri-Rao values), after its 4 x 4 tensor values are already in registers.
constexpr int kResRowsPerWarp = 4;
constexpr int kResGroups = 2;                                    // row groups per warp per chunk
constexpr int kResRows = (kStreamRedThreads / 32) * kResRowsPerWarp * kResGroups;   // 64 rows per block

int residual_chunk(int r) { return r <= 16 ? 512 : r <= 32 ? 256 : 128; }   // r * (CW + 4) * 4 <= 34 KB

template <typename TE>
__device__ __forceinline__ void load4(const TE* p, float* x);
template <>
__device__ __forceinline__ void load4<float>(const float* p, float* x) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    x[0] = v.x, x[1] = v.y, x[2] = v.z, x[3] = v.w;
}
template <>
__device__ __forceinline__ void load4<__nv_bfloat16>(const __nv_bfloat16* p, float* x) {
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(p));
    x[0] = __uint_as_float(v.x << 16), x[1] = __uint_as_float(v.x & 0xffff0000u);
    x[2] = __uint_as_float(v.y << 16), x[3] = __uint_as_float(v.y & 0xffff0000u);
}

template <typename TE>
__global__ void __launch_bounds__(kStreamRedThreads) k_residual_sq(const TE* __restrict__ T, int64_t Ii, int64_t n_o,
                                                                   int64_t C, int64_t ld, int r, int CW, int per,
                                                                   const float* __restrict__ W, int RP,
                                                                   const float* __restrict__ Ai,
                                                                   const float* __restrict__ Ac,
                                                                   double* __restrict__ parts) {
    // Work units: (column chunk, row slice), `per` row slices per chunk.  A block stages its
    // unit's chunk of A_{N-1}^T in shared memory once (coalesced) and streams the slice's rows
    // (64-row blocks slice, slice + per, ...) against it.  With gridDim.x = units, as the host
    // arranges whenever it can, every block has one unit.
    extern __shared__ __align__(16) float AcT[];                 // [r][CW + 4]
    __shared__ __align__(16) float krT[kStreamRedThreads / 32][NTF_MAX_RANK][kResRowsPerWarp];
    __shared__ double sbuf[33];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int CWP = CW + 4;                                       // row pitch: float4-aligned, fewer conflicts
    const int64_t rows = Ii * n_o;
    const int64_t nblk = (rows + kResRows - 1) / kResRows;
    const int64_t n_chunks = (C + CW - 1) / CW;
    double acc = 0.0;
    for (int64_t u = blockIdx.x; u < n_chunks * per; u += gridDim.x) {
        const int64_t cb = (u / per) * CW;
        const int cw = (int)min((int64_t)CW, C - cb);
        __syncthreads();
        for (int q = threadIdx.x; q < r * CW; q += blockDim.x) {
            const int c = q / r, p = q - c * r;                   // consecutive q: consecutive A_{N-1} entries
            AcT[p * CWP + c] = c < cw ? Ac[(cb + c) * r + p] : 0.f;
        }
        __syncthreads();
        for (int64_t blk = u % per; blk < nblk; blk += per) {
            for (int g = 0; g < kResGroups; ++g) {
                const int64_t row0 = blk * kResRows + (int64_t)(g * (kStreamRedThreads / 32) + wl) * kResRowsPerWarp;
                if (row0 >= rows) continue;                        // warp-uniform
                __syncwarp();
                for (int p = lane; p < r; p += 32)
#pragma unroll
                    for (int k = 0; k < kResRowsPerWarp; ++k) {
                        const int64_t row = row0 + k;
                        float kr = 0.f;
                        if (row < rows) {
                            const int64_t o = row / Ii, i = row - o * Ii;
                            kr = W[o * RP + p] * Ai[i * r + p];
                        }
                        krT[wl][p][k] = kr;
                    }
                __syncwarp();
                for (int c0 = 4 * lane; c0 < cw; c0 += 128) {
                    float t[kResRowsPerWarp][4];
#pragma unroll
                    for (int k = 0; k < kResRowsPerWarp; ++k) {
                        if (row0 + k < rows) load4<TE>(T + (row0 + k) * ld + cb + c0, t[k]);
                        else t[k][0] = t[k][1] = t[k][2] = t[k][3] = 0.f;
                    }
                    float x[kResRowsPerWarp][4];
#pragma unroll
                    for (int k = 0; k < kResRowsPerWarp; ++k) x[k][0] = x[k][1] = x[k][2] = x[k][3] = 0.f;
                    for (int p = 0; p < r; ++p) {
                        const float4 a = *reinterpret_cast<const float4*>(&AcT[p * CWP + c0]);
                        const float4 kk = *reinterpret_cast<const float4*>(&krT[wl][p][0]);
                        const float kv[4] = {kk.x, kk.y, kk.z, kk.w};
#pragma unroll
                        for (int k = 0; k < kResRowsPerWarp; ++k) {
                            x[k][0] = fmaf(kv[k], a.x, x[k][0]);
                            x[k][1] = fmaf(kv[k], a.y, x[k][1]);
                            x[k][2] = fmaf(kv[k], a.z, x[k][2]);
                            x[k][3] = fmaf(kv[k], a.w, x[k][3]);
                        }
                    }
                    float s = 0.f;
#pragma unroll
                    for (int k = 0; k < kResRowsPerWarp; ++k)
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const float d = t[k][j] - x[k][j];
                            s = (row0 + k < rows && c0 + j < cw) ? fmaf(d, d, s) : s;
                        }
                    acc += (double)s;
                }
            }
        }
    }
    const double tot = block_sum_d(acc, sbuf);
    if (threadIdx.x == 0) parts[blockIdx.x] = tot;
}

cudaError_t launch_residual_sq(const TensorView& v, int r, const float* W, int RP, const float* Ai, const float* Ac,
                               double* parts, double* out, cudaStream_t st) {
    const int64_t nblk = (v.Ii * v.n_o + kResRows - 1) / kResRows;
    const int CW = residual_chunk(r);
    const int64_t n_chunks = (v.C + CW - 1) / CW;
    // row slices per column chunk; one block per (chunk, slice) unit while they fit in the
    // partial-sum buffer (stream_red_blocks() entries), else blocks loop over units
    const int64_t per = std::max<int64_t>(1, std::min<int64_t>(nblk, stream_red_blocks() / n_chunks));
    const int G = (int)std::min<int64_t>(per * n_chunks, stream_red_blocks());
    const size_t smem = sizeof(float) * (size_t)r * (CW + 4);
    if (v.dtype == NTF_F32)
        k_residual_sq<float><<<G, kStreamRedThreads, smem, st>>>(static_cast<const float*>(v.data), v.Ii, v.n_o, v.C,
                                                                 v.ld, r, CW, (int)per, W, RP, Ai, Ac, parts);
    else
        k_residual_sq<__nv_bfloat16><<<G, kStreamRedThreads, smem, st>>>(
            static_cast<const __nv_bfloat16*>(v.data), v.Ii, v.n_o, v.C, v.ld, r, CW, (int)per, W, RP, Ai, Ac, parts);
    count_launch();
    k_sum_parts<<<1, 256, 0, st>>>(parts, G, out);
    count_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// a8: bf16 cast with row pitch; one thread per 8 destination elements
// ---------------------------------------------------------------------------
__global__ void k_to_bf16(const float* __restrict__ src, int64_t rows, int64_t C, int64_t ld_src,
                          __nv_bfloat16* __restrict__ dst, int64_t ld_dst) {
    const int64_t per_row = ld_dst / 8;
    const int64_t n = rows * per_row;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = idx / per_row, c0 = (idx - row * per_row) * 8;
        const float* sp = src + row * ld_src + c0;
        float x[8];
        // the source row holds C values in a pitch that is a multiple of 4
        float4 a = c0 < C ? __ldg(reinterpret_cast<const float4*>(sp)) : make_float4(0.f, 0.f, 0.f, 0.f);
        float4 b = c0 + 4 < C ? __ldg(reinterpret_cast<const float4*>(sp + 4)) : make_float4(0.f, 0.f, 0.f, 0.f);
        x[0] = a.x, x[1] = a.y, x[2] = a.z, x[3] = a.w, x[4] = b.x, x[5] = b.y, x[6] = b.z, x[7] = b.w;
        uint32_t w[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const __nv_bfloat16 lo = __float2bfloat16_rn(c0 + 2 * k < C ? x[2 * k] : 0.f);
            const __nv_bfloat16 hi = __float2bfloat16_rn(c0 + 2 * k + 1 < C ? x[2 * k + 1] : 0.f);
            w[k] = (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
        }
        *reinterpret_cast<uint4*>(dst + row * ld_dst + c0) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

cudaError_t launch_to_bf16(const float* src, int64_t rows, int64_t C, int64_t ld_src, void* dst, int64_t ld_dst,
                           cudaStream_t st) {
    int64_t g = (rows * (ld_dst / 8) + 255) / 256;
    if (g > 8 * num_sms()) g = 8 * num_sms();
    if (g < 1) g = 1;
    k_to_bf16<<<(int)g, 256, 0, st>>>(src, rows, C, ld_src, static_cast<__nv_bfloat16*>(dst), ld_dst);
    count_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// a6: HER state, decision and the factor copies
// ---------------------------------------------------------------------------
__global__ void k_her_init(ntf_her_state* s, double beta0, double gamma, double gamma_bar, double eta,
                           const double* f0) {
    s->beta = beta0;
    s->beta_bar = 1.0;
    s->f_hat_prev = *f0;
    s->gamma = gamma;
    s->gamma_bar = gamma_bar;
    s->eta = eta;
    s->iters = 0;
    s->restarts = 0;
    s->last_restart = 0;
    s->numeric_error = isfinite(*f0) ? 0 : 1;
}

cudaError_t launch_her_init(ntf_her_state* s, double beta0, double gamma, double gamma_bar, double eta,
                            const double* f0, cudaStream_t st) {
    k_her_init<<<1, 1, 0, st>>>(s, beta0, gamma, gamma_bar, eta, f0);
    count_launch();
    return cudaGetLastError();
}

// Alg. 2, restart test (F-hat_k > F-hat_{k-1}) and eqs. HER_eq:beta_update /
// HER_eq:beta_bar_update.  A non-finite F-hat is treated as a restart and flagged.
__global__ void k_her_decide(ntf_her_state* s, const double* fhat_p) {
    const double fhat = *fhat_p;
    const double beta = s->beta, beta_bar = s->beta_bar;
    const bool finite = isfinite(fhat);
    const bool restart = !finite || fhat > s->f_hat_prev;
    if (restart) {
        s->beta_bar = beta;
        s->beta = beta / s->eta;
    } else {
        s->beta_bar = fmin(1.0, s->gamma_bar * beta_bar);
        s->beta = fmin(beta_bar, s->gamma * beta);
    }
    s->f_hat_prev = fhat;
    s->iters += 1;
    s->restarts += restart ? 1 : 0;
    s->last_restart = restart ? 1 : 0;
    if (!finite) s->numeric_error = 1;
}

// restart: dst = A_hat side gets A (copy A -> A_hat); accept: A gets A_hat.
__global__ void k_her_copy(const ntf_her_state* s, CopyPairs P) {
    const bool restart = s->last_restart != 0;
    for (int q = 0; q < P.count; ++q) {
        float* a = P.a[q];
        float* ah = P.ah[q];
        const int64_t n = P.n[q];
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
             i += (int64_t)gridDim.x * blockDim.x) {
            if (restart) ah[i] = a[i];
            else a[i] = ah[i];
        }
    }
    for (int q = 0; q < P.gcount; ++q) {
        double* g = P.g[q];
        double* gh = P.gh[q];
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.gn; i += gridDim.x * blockDim.x) {
            if (restart) gh[i] = g[i];
            else g[i] = gh[i];
        }
    }
}

cudaError_t launch_her_copy(const ntf_her_state* s, const CopyPairs& P, cudaStream_t st) {
    int64_t maxn = P.gn;
    for (int q = 0; q < P.count; ++q) maxn = P.n[q] > maxn ? P.n[q] : maxn;
    int64_t g = (maxn + 255) / 256;
    if (g > 256) g = 256;
    if (g < 1) g = 1;
    k_her_copy<<<(int)g, 256, 0, st>>>(s, P);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_her_step(ntf_her_state* s, const double* fhat, const CopyPairs& P, cudaStream_t st) {
    k_her_decide<<<1, 1, 0, st>>>(s, fhat);
    count_launch();
    int64_t maxn = P.gn;
    for (int q = 0; q < P.count; ++q) maxn = P.n[q] > maxn ? P.n[q] : maxn;
    int64_t g = (maxn + 255) / 256;
    if (g > 256) g = 256;
    if (g < 1) g = 1;
    k_her_copy<<<(int)g, 256, 0, st>>>(s, P);
    count_launch();
    return cudaGetLastError();
}

}  // namespace ntf
