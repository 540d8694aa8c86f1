// Step a3, the block updates: HALS column sweeps, projected-gradient steps and AO-Nesterov
// steps, one thread per row of A with the row in registers (R >= r wide).  Templates shared by bcd.cu (R <= 24),
// bcd32.cu and bcd64.cu, which instantiate disjoint widths so that they compile in parallel.
#pragma once

#include "block_reduce.cuh"
#include "small.cuh"

namespace ntf {

// ---------------------------------------------------------------------------
// a3: block updates.  One thread owns one row of A (rows are independent in
// both HALS and PGD); R >= r is the register width.
// ---------------------------------------------------------------------------
constexpr int kBcdThreads = 512;

template <int R>
__device__ __forceinline__ void load_row(const float* __restrict__ src, int64_t i, int r, float (&v)[R]) {
#pragma unroll
    for (int p = 0; p < R; ++p) v[p] = p < r ? src[i * r + p] : 0.f;
}

// One HALS sweep (Sec. 2.1.4) of row a against m with V in shared memory
// (Vs row-major R x R, zero padded).  Returns sum of squared changes.
template <int R>
__device__ __forceinline__ float hals_row(float (&a)[R], const float (&m)[R], const float* Vs, int r) {
    float d2 = 0.f;
    // widths up to 32 keep the row in registers (loops unrolled); at 64 the row spills anyway,
    // and unrolling the 64 x 64 sweep only multiplies the compile time
#pragma unroll (R > 32 ? 1 : R)
    for (int j = 0; j < R; ++j) {
        if (j < r) {
            const float vjj = Vs[j * R + j];
            if (vjj > 0.f) {
                // num = M(i,j) - sum_{l != j} a_l V(l,j), in four independent partial sums
                float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
                for (int l = 0; l < R; l += 4) {
                    s0 = fmaf(l + 0 == j ? 0.f : a[l + 0], Vs[(l + 0) * R + j], s0);
                    if (l + 1 < R) s1 = fmaf(l + 1 == j ? 0.f : a[l + 1], Vs[(l + 1) * R + j], s1);
                    if (l + 2 < R) s2 = fmaf(l + 2 == j ? 0.f : a[l + 2], Vs[(l + 2) * R + j], s2);
                    if (l + 3 < R) s3 = fmaf(l + 3 == j ? 0.f : a[l + 3], Vs[(l + 3) * R + j], s3);
                }
                const float num = m[j] - ((s0 + s1) + (s2 + s3));
                const float nv = fmaxf(num, 0.f) / vjj;
                const float d = nv - a[j];
                d2 = fmaf(d, d, d2);
                a[j] = nv;
            }
        }
    }
    return d2;
}

// One projected-gradient step (Sec. 2.2): a <- max(0, a - (a V - m)/L)
template <int R>
__device__ __forceinline__ float pgd_row(float (&a)[R], const float (&m)[R], const float* Vs, int r, float invL) {
    float na[R];
    float d2 = 0.f;
#pragma unroll (R > 32 ? 1 : R)
    for (int j = 0; j < R; ++j) {
        float g = -m[j];
#pragma unroll
        for (int l = 0; l < R; ++l) g = fmaf(a[l], Vs[l * R + j], g);
        const float v = fmaxf(fmaf(-g, invL, a[j]), 0.f);
        na[j] = j < r ? v : 0.f;
    }
#pragma unroll
    for (int j = 0; j < R; ++j) {
        const float d = na[j] - a[j];
        d2 = fmaf(d, d, d2);
        a[j] = na[j];
    }
    return d2;
}

// One AO-Nesterov step (Sec. 2.1, AO-Nesterov): the projected gradient step of eq. projgrad taken
// at the extrapolated point y, then the momentum step with the weight w of the t_k sequence of
// Appendix B:  x_new = max(0, y - (y V - m)/L),  y <- x_new + w (x_new - x),  x <- x_new.
// Returns ||x_new - x||^2.
template <int R>
__device__ __forceinline__ float nesterov_row(float (&x)[R], float (&y)[R], const float (&m)[R], const float* Vs,
                                              int r, float invL, float w) {
    float nx[R];
#pragma unroll (R > 32 ? 1 : R)
    for (int j = 0; j < R; ++j) {
        float g = -m[j];
#pragma unroll
        for (int l = 0; l < R; ++l) g = fmaf(y[l], Vs[l * R + j], g);
        const float v = fmaxf(fmaf(-g, invL, y[j]), 0.f);
        nx[j] = j < r ? v : 0.f;
    }
    float d2 = 0.f;
#pragma unroll
    for (int j = 0; j < R; ++j) {
        const float d = nx[j] - x[j];
        d2 = fmaf(d, d, d2);
        y[j] = fmaf(w, d, nx[j]);
        x[j] = nx[j];
    }
    return d2;
}

// t_s = (1 + sqrt(1 + 4 t_{s-1}^2)) / 2 with t_0 = 1 (Appendix B); the momentum weight after
// step s is (t_{s-1} - 1) / t_s.
__host__ __device__ __forceinline__ double nesterov_t_next(double t) { return 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t)); }

template <int R>
__device__ void stage_V(const double* __restrict__ V, int r, float* Vs) {
    for (int q = threadIdx.x; q < R * R; q += blockDim.x) {
        const int l = q / R, j = q % R;
        Vs[q] = (l < r && j < r) ? (float)V[l * r + j] : 0.f;
    }
}

// Whole inner loop in one CTA (rows <= kBcdThreads).  method 0 = HALS, 1 = PGD, 2 = AO-Nesterov.
template <int R>
__global__ void __launch_bounds__(kBcdThreads) k_bcd_local(int method, float* __restrict__ A, int64_t rows, int r,
                                                           const float* __restrict__ M, const double* __restrict__ V,
                                                           const double* __restrict__ Lptr, int inner_max,
                                                           double tol2, int* __restrict__ sweeps_out) {
    __shared__ float Vs[R * R];
    __shared__ double sbuf[33];
    stage_V<R>(V, r, Vs);
    __syncthreads();
    const int64_t i = threadIdx.x;
    const bool live = i < rows;
    float a[R], m[R];
    if (live) {
        load_row<R>(A, i, r, a);
        load_row<R>(M, i, r, m);
    } else {
#pragma unroll
        for (int p = 0; p < R; ++p) a[p] = m[p] = 0.f;
    }
    const float invL = (method != 0 && Lptr && *Lptr > 0.0) ? (float)(1.0 / *Lptr) : 0.f;
    float y[R];                       // AO-Nesterov: extrapolated point, Y_0 = X_0
#pragma unroll
    for (int p = 0; p < R; ++p) y[p] = a[p];
    double t = 1.0;
    double delta1 = 0.0;
    int s = 0;
    for (;;) {
        ++s;
        float d2 = 0.f;
        if (method == 2) {
            const double tn = nesterov_t_next(t);
            const float w = (float)((t - 1.0) / tn);
            t = tn;
            if (live) d2 = nesterov_row<R>(a, y, m, Vs, r, invL, w);
        } else if (live) {
            d2 = method == 0 ? hals_row<R>(a, m, Vs, r) : pgd_row<R>(a, m, Vs, r, invL);
        }
        const double tot = block_sum_d((double)d2, sbuf);
        if (s == 1) delta1 = tot;
        if (s >= inner_max || tot <= tol2 * delta1) break;
    }
    if (live)
#pragma unroll
        for (int p = 0; p < R; ++p)
            if (p < r) A[i * r + p] = a[p];
    if (threadIdx.x == 0 && sweeps_out) *sweeps_out = s;
}

// One sweep/step across many CTAs.  Sweep s (1-based) first decides, from the
// partial sums of sweeps 1 and s-1, whether the inner loop has stopped.
// parts: [2][gridDim] doubles (by sweep parity) + [gridDim] for sweep 1; flag: stopped.
// AO-Nesterov keeps its extrapolated point in Y (rows x r; read from A at s = 1) and takes
// the momentum weight w of step s from the host.
template <int R>
__global__ void __launch_bounds__(kBcdThreads) k_bcd_sweep(int method, float* __restrict__ A, int64_t rows, int r,
                                                           const float* __restrict__ M, const double* __restrict__ V,
                                                           const double* __restrict__ Lptr, int s, double tol2,
                                                           double* __restrict__ parts, int* __restrict__ stopped,
                                                           float* __restrict__ Y, float w) {
    __shared__ float Vs[R * R];
    __shared__ double sbuf[33];
    __shared__ int stop_sh;
    const int G = gridDim.x;
    if (threadIdx.x == 0) {
        int stop = (s == 1) ? 0 : *stopped;
        if (s > 1 && !stop) {
            double d1 = 0.0, dp = 0.0;
            for (int g = 0; g < G; ++g) {
                d1 += parts[2 * G + g];
                dp += parts[((s - 1) & 1) * G + g];
            }
            if (dp <= tol2 * d1) stop = 1;
        }
        stop_sh = stop;
    }
    stage_V<R>(V, r, Vs);
    __syncthreads();
    if (stop_sh) {
        if (blockIdx.x == 0 && threadIdx.x == 0) *stopped = 1;
        return;
    }
    if (s == 1 && blockIdx.x == 0 && threadIdx.x == 0) *stopped = 0;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float d2 = 0.f;
    if (i < rows) {
        float a[R], m[R];
        load_row<R>(A, i, r, a);
        load_row<R>(M, i, r, m);
        const float invL = (method != 0 && Lptr && *Lptr > 0.0) ? (float)(1.0 / *Lptr) : 0.f;
        if (method == 2) {
            float y[R];
            load_row<R>(s == 1 ? A : Y, i, r, y);
            d2 = nesterov_row<R>(a, y, m, Vs, r, invL, w);
#pragma unroll
            for (int p = 0; p < R; ++p)
                if (p < r) Y[i * r + p] = y[p];
        } else {
            d2 = method == 0 ? hals_row<R>(a, m, Vs, r) : pgd_row<R>(a, m, Vs, r, invL);
        }
#pragma unroll
        for (int p = 0; p < R; ++p)
            if (p < r) A[i * r + p] = a[p];
    }
    const double tot = block_sum_d((double)d2, sbuf);
    if (threadIdx.x == 0) {
        parts[(s & 1) * G + blockIdx.x] = tot;
        if (s == 1) parts[2 * G + blockIdx.x] = tot;
    }
}

// L = lambda_max(V) of the symmetric nonnegative r x r matrix V: FP32 power
// iteration to a relative change below 1e-7 (at most 500 steps), then one
// FP64 Rayleigh quotient.  One warp.
static __global__ void k_lambda_max(const double* __restrict__ V, int r, double* __restrict__ L) {
    __shared__ float Vs[NTF_MAX_RANK * NTF_MAX_RANK];
    __shared__ float x[NTF_MAX_RANK];
    const int lane = threadIdx.x;
    for (int q = lane; q < r * r; q += 32) Vs[q] = (float)V[q];
    for (int j = lane; j < r; j += 32) x[j] = 1.f + 0.01f * j;
    __syncwarp();
    float lam = 0.f;
    for (int it = 0; it < 500; ++it) {
        float y0 = 0.f, y1 = 0.f;
        if (lane < r)
            for (int l = 0; l < r; ++l) y0 = fmaf(Vs[lane * r + l], x[l], y0);
        if (lane + 32 < r)
            for (int l = 0; l < r; ++l) y1 = fmaf(Vs[(lane + 32) * r + l], x[l], y1);
        float nrm = y0 * y0 + y1 * y1;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, off);
        nrm = sqrtf(nrm);
        __syncwarp();
        if (nrm > 0.f) {
            if (lane < r) x[lane] = y0 / nrm;
            if (lane + 32 < r) x[lane + 32] = y1 / nrm;
        }
        __syncwarp();
        const bool done = fabsf(nrm - lam) <= 1e-7f * nrm;
        lam = nrm;
        if (done || nrm == 0.f) break;
    }
    // Rayleigh quotient x^T V x / x^T x in FP64
    double num = 0.0, den = 0.0;
    for (int j = lane; j < r; j += 32) {
        double y = 0.0;
        for (int l = 0; l < r; ++l) y += V[j * r + l] * (double)x[l];
        num += (double)x[j] * y;
        den += (double)x[j] * (double)x[j];
    }
    num = warp_sum_d(num);
    den = warp_sum_d(den);
    if (lane == 0) *L = den > 0.0 ? num / den : 0.0;
}

template <int R>
static cudaError_t bcd_impl(int method, float* A, int64_t rows, int r, const float* M, const double* V,
                            int inner_max, double tol, double* L, double* parts, int* stopped, float* Y,
                            cudaStream_t st) {
    if (method != 0) {
        k_lambda_max<<<1, 32, 0, st>>>(V, r, L);
        count_launch();
    }
    const double tol2 = tol * tol;
    if (rows <= kBcdThreads) {
        k_bcd_local<R><<<1, kBcdThreads, 0, st>>>(method, A, rows, r, M, V, L, inner_max, tol2, nullptr);
        count_launch();
        return cudaGetLastError();
    }
    const int G = (int)((rows + kBcdThreads - 1) / kBcdThreads);
    double t = 1.0;
    for (int s = 1; s <= inner_max; ++s) {
        const double tn = nesterov_t_next(t);
        const float w = (float)((t - 1.0) / tn);
        t = tn;
        k_bcd_sweep<R><<<G, kBcdThreads, 0, st>>>(method, A, rows, r, M, V, L, s, tol2, parts, stopped, Y, w);
        count_launch();
    }
    return cudaGetLastError();
}

cudaError_t launch_bcd_r32(int method, float* A, int64_t rows, int r, const float* M, const double* V,
                           int inner_max, double tol, double* L, double* parts, int* stopped, float* Y,
                           cudaStream_t st);
cudaError_t launch_bcd_r64(int method, float* A, int64_t rows, int r, const float* M, const double* V,
                           int inner_max, double tol, double* L, double* parts, int* stopped, float* Y,
                           cudaStream_t st);

}  // namespace ntf
