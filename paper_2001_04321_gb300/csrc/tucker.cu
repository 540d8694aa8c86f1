// Tucker-format data (Appendix A): MTTKRP and norm of (U_0 (x) ... (x) U_{N-1}) G through the
// core, and their C-ABI entry points.
//
// The gradient formula of Appendix A gives the MTTKRP of the Tucker-format tensor as
//   M_n = U_n G_[n] (Khatri-Rao of U_p^T A_p, p != n) = U_n MTTKRP(G, {W_p = U_p^T A_p}, n),
// so one MTTKRP costs N-1 projections (n_p x r_p by n_p x r), one MTTKRP of the small core
// (the library's MTTKRP kernels on the r_0 x ... x r_{N-1} tensor) and one expansion
// (n_n x r_n by r_n x r).  ||T||^2 = <G, G x_0 Q_0 ... x_{N-1} Q_{N-1}> with Q_p = U_p^T U_p.
// Every sum is in a fixed order (FP32 over 64-row chunks, chunks combined in FP64), so the
// results are bitwise reproducible.
#include "tucker.cuh"
#include "block_reduce.cuh"

#include <string>

namespace ntf {

constexpr int kProjRows = 64;      // rows of U_p and A_p staged per CTA
constexpr int kProjThreads = 256;

static inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }
static inline unsigned grid_of(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// part[c][q r + j] = sum over the rows i of chunk c of U(i, q) A(i, j)   (FP32, rows in order)
__global__ void __launch_bounds__(kProjThreads) k_project(const float* __restrict__ U, int64_t n, int rp,
                                                          const float* __restrict__ A, int r,
                                                          float* __restrict__ part) {
    __shared__ float sU[kProjRows * kTuckerMaxRank];
    __shared__ float sA[kProjRows * NTF_MAX_RANK];
    const int64_t i0 = (int64_t)blockIdx.x * kProjRows;
    const int nrow = (int)(n - i0 < kProjRows ? n - i0 : kProjRows);
    for (int t = threadIdx.x; t < nrow * rp; t += blockDim.x) sU[t] = U[i0 * rp + t];
    for (int t = threadIdx.x; t < nrow * r; t += blockDim.x) sA[t] = A[i0 * r + t];
    __syncthreads();
    float* out = part + (int64_t)blockIdx.x * rp * r;
    for (int o = threadIdx.x; o < rp * r; o += blockDim.x) {
        const int q = o / r, j = o - q * r;
        float s = 0.f;
        for (int i = 0; i < nrow; ++i) s = fmaf(sU[i * rp + q], sA[i * r + j], s);
        out[o] = s;
    }
}

// out[o] = sum over chunks c of part[c][o] in FP64: one warp per output, lane l takes chunks
// l, l + 32, ... in order, then a fixed butterfly (independent loads, same order every run)
__global__ void k_project_sum(const float* __restrict__ part, int nchunks, int n_out, float* __restrict__ outf,
                              double* __restrict__ outd) {
    const int o = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (o >= n_out) return;   // whole warps leave together
    double s = 0.0;
    for (int c = lane; c < nchunks; c += 32) s += (double)part[(int64_t)c * n_out + o];
    s = warp_sum_d(s);
    if (lane == 0) {
        if (outf) outf[o] = (float)s;
        if (outd) outd[o] = s;
    }
}

// out(i, j) = sum_q U(i, q) Y(q, j): one warp per row, lanes over columns j (and j + 32)
__global__ void __launch_bounds__(256) k_expand(const float* __restrict__ U, int64_t n, int rp,
                                                const float* __restrict__ Y, int r, float* __restrict__ out) {
    __shared__ float sY[kTuckerMaxRank * NTF_MAX_RANK];
    for (int t = threadIdx.x; t < rp * r; t += blockDim.x) sY[t] = Y[t];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += nwarps) {
        const float u0 = lane < rp ? U[i * rp + lane] : 0.f;
        const float u1 = lane + 32 < rp ? U[i * rp + lane + 32] : 0.f;
        float s0 = 0.f, s1 = 0.f;
        for (int q = 0; q < rp; ++q) {
            const float uq = __shfl_sync(0xffffffffu, q < 32 ? u0 : u1, q & 31);
            if (lane < r) s0 = fmaf(uq, sY[q * r + lane], s0);
            if (lane + 32 < r) s1 = fmaf(uq, sY[q * r + lane + 32], s1);
        }
        if (lane < r) out[i * r + lane] = s0;
        if (lane + 32 < r) out[i * r + lane + 32] = s1;
    }
}

struct CoreDims {
    int64_t d[NTF_MAX_ORDER];
};

// Z (dense C order, FP64) <- the core G (row pitch ld)
__global__ void k_core_to_f64(const float* __restrict__ G, int64_t rows, int64_t C, int64_t ld, double* __restrict__ Z) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= rows * C) return;
    const int64_t row = t / C, c = t - row * C;
    Z[t] = (double)G[row * ld + c];
}

// Zout = Zin x_p Q: every mode-p fibre z of Zin becomes Q z (FP64)
__global__ void k_mode_product(const double* __restrict__ Zin, const double* __restrict__ Q, double* __restrict__ Zout,
                               CoreDims D, int order, int p, int64_t total) {
    const int64_t lin = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (lin >= total) return;
    int64_t stride = 1;
    for (int l = order - 1; l > p; --l) stride *= D.d[l];
    const int64_t rp = D.d[p];
    const int64_t a = (lin / stride) % rp;
    const int64_t base = lin - a * stride;
    double s = 0.0;
    for (int64_t b = 0; b < rp; ++b) s += Q[a * rp + b] * Zin[base + b * stride];
    Zout[lin] = s;
}

// *out = <G, Z> in FP64, one CTA, fixed order
__global__ void __launch_bounds__(1024) k_core_dot(const float* __restrict__ G, int64_t rows, int64_t C, int64_t ld,
                                                   const double* __restrict__ Z, double* __restrict__ out) {
    __shared__ double sbuf[33];
    double s = 0.0;
    for (int64_t t = threadIdx.x; t < rows * C; t += blockDim.x) {
        const int64_t row = t / C, c = t - row * C;
        s += (double)G[row * ld + c] * Z[t];
    }
    s = block_sum_d(s, sbuf);
    if (threadIdx.x == 0) *out = s;
}

ntf_status make_tucker_view(const ntf_tucker* X, TuckerView* v) {
    if (!X) return fail(NTF_EINVAL, "Tucker data is NULL");
    ntf_status s = make_view(&X->core, &v->core);
    if (s != NTF_OK) return s;
    if (v->core.dtype != NTF_F32) return fail(NTF_EINVAL, "the Tucker core must be NTF_F32");
    v->order = v->core.order;
    for (int p = 0; p < v->order; ++p) {
        if (v->core.dims[p] > kTuckerMaxRank) return fail(NTF_EINVAL, "Tucker ranks (core dims) must be <= 64");
        if (X->dims[p] < 1 || X->dims[p] > (int64_t(1) << 31)) return fail(NTF_EINVAL, "Tucker dims must be in [1, 2^31]");
        if (!X->U[p]) return fail(NTF_EINVAL, "Tucker basis U_p is NULL");
        v->dims[p] = X->dims[p];
        v->U[p] = X->U[p];
    }
    return NTF_OK;
}

static int64_t proj_chunks(int64_t n) { return (n + kProjRows - 1) / kProjRows; }

ntf_status plan_tucker_mttkrp(const TuckerView& v, int rank, int mode, TuckerPlan* P) {
    if (rank < 1 || rank > NTF_MAX_RANK) return fail(NTF_EINVAL, "rank must be in [1, 64]");
    if (mode < 0 || mode >= v.order) return fail(NTF_EINVAL, "mode out of range");
    P->mode = mode;
    P->rank = rank;
    ntf_status s = plan_mttkrp(v.core, rank, mode, &P->core);
    if (s != NTF_OK) return s;
    size_t off = 0, part = 0;
    for (int p = 0; p < v.order; ++p) {
        P->off_W[p] = off;
        if (p == mode) continue;
        off += align256(sizeof(float) * (size_t)v.core.dims[p] * rank);
        part = std::max(part, sizeof(float) * (size_t)proj_chunks(v.dims[p]) * v.core.dims[p] * rank);
    }
    P->off_part = off;
    off += align256(part);
    P->off_Y = off;
    off += align256(sizeof(float) * (size_t)v.core.dims[mode] * rank);
    P->off_core = off;
    off += align256(P->core.total);
    P->total = off;
    return NTF_OK;
}

// W = U^T A (r_p x r) through the chunked partial sums
static cudaError_t project(const float* U, int64_t n, int rp, const float* A, int r, float* part, float* Wf,
                           double* Wd, cudaStream_t st) {
    const int64_t nc = proj_chunks(n);
    k_project<<<(unsigned)nc, kProjThreads, 0, st>>>(U, n, rp, A, r, part);
    count_launch();
    k_project_sum<<<grid_of((int64_t)rp * r * 32, 256), 256, 0, st>>>(part, (int)nc, rp * r, Wf, Wd);
    count_launch();
    return cudaGetLastError();
}

ntf_status run_tucker_mttkrp(const TuckerView& v, const TuckerPlan& P, const float* const* factors, float* out,
                             void* workspace, cudaStream_t st, TmapCache* cache) {
    unsigned char* ws = static_cast<unsigned char*>(workspace);
    const int n = P.mode, r = P.rank;
    float* part = reinterpret_cast<float*>(ws + P.off_part);
    const float* W[NTF_MAX_ORDER] = {nullptr};
    for (int p = 0; p < v.order; ++p) {
        if (p == n) continue;
        float* Wp = reinterpret_cast<float*>(ws + P.off_W[p]);
        cudaError_t e = project(v.U[p], v.dims[p], (int)v.core.dims[p], factors[p], r, part, Wp, nullptr, st);
        if (e != cudaSuccess) return cuda_fail(e, "Tucker projection U_p^T A_p");
        W[p] = Wp;
    }
    float* Y = reinterpret_cast<float*>(ws + P.off_Y);
    ntf_status s = run_mttkrp(v.core, P.core, W, Y, ws + P.off_core, st, cache, nullptr);
    if (s != NTF_OK) return s;
    const int64_t rows = v.dims[n];
    const unsigned blocks = (unsigned)std::min<int64_t>((rows + 7) / 8, 4 * num_sms());
    k_expand<<<blocks, 256, 0, st>>>(v.U[n], rows, (int)v.core.dims[n], Y, r, out);
    NTF_LAUNCH_CHECK("Tucker expansion U_n Y");
    return NTF_OK;
}

size_t tucker_norm_workspace(const TuckerView& v) {
    const int64_t ctot = v.core.numel();
    size_t part = 0;
    for (int p = 0; p < v.order; ++p)
        part = std::max(part, sizeof(float) * (size_t)proj_chunks(v.dims[p]) * v.core.dims[p] * v.core.dims[p]);
    return align256(part) + align256(sizeof(double) * kTuckerMaxRank * kTuckerMaxRank) +
           2 * align256(sizeof(double) * (size_t)ctot);
}

ntf_status run_tucker_norm_sq(const TuckerView& v, double* out, void* workspace, cudaStream_t st) {
    unsigned char* ws = static_cast<unsigned char*>(workspace);
    const int64_t ctot = v.core.numel();
    size_t part_b = 0;
    for (int p = 0; p < v.order; ++p)
        part_b = std::max(part_b, sizeof(float) * (size_t)proj_chunks(v.dims[p]) * v.core.dims[p] * v.core.dims[p]);
    float* part = reinterpret_cast<float*>(ws);
    double* Q = reinterpret_cast<double*>(ws + align256(part_b));
    double* Z[2];
    Z[0] = reinterpret_cast<double*>(ws + align256(part_b) + align256(sizeof(double) * kTuckerMaxRank * kTuckerMaxRank));
    Z[1] = reinterpret_cast<double*>(reinterpret_cast<unsigned char*>(Z[0]) + align256(sizeof(double) * (size_t)ctot));
    const TensorView& c = v.core;
    k_core_to_f64<<<grid_of(ctot, 256), 256, 0, st>>>(static_cast<const float*>(c.data), c.rows(), c.C, c.ld, Z[0]);
    NTF_LAUNCH_CHECK("Tucker core to FP64");
    CoreDims D{};
    for (int p = 0; p < v.order; ++p) D.d[p] = c.dims[p];
    int cur = 0;
    for (int p = 0; p < v.order; ++p) {
        const int rp = (int)c.dims[p];
        cudaError_t e = project(v.U[p], v.dims[p], rp, v.U[p], rp, part, nullptr, Q, st);
        if (e != cudaSuccess) return cuda_fail(e, "Tucker Gram U_p^T U_p");
        k_mode_product<<<grid_of(ctot, 256), 256, 0, st>>>(Z[cur], Q, Z[cur ^ 1], D, v.order, p, ctot);
        NTF_LAUNCH_CHECK("Tucker mode product");
        cur ^= 1;
    }
    k_core_dot<<<1, 1024, 0, st>>>(static_cast<const float*>(c.data), c.rows(), c.C, c.ld, Z[cur], out);
    NTF_LAUNCH_CHECK("Tucker core inner product");
    return NTF_OK;
}

static ntf_status check_tucker_ptrs(const TuckerView& v) {
    ntf_status s = check_device_ptr(v.core.data, "Tucker core data");
    for (int p = 0; p < v.order && s == NTF_OK; ++p) s = check_device_ptr(v.U[p], "Tucker basis U_p");
    return s;
}

}  // namespace ntf

using namespace ntf;

extern "C" {

size_t ntf_tucker_mttkrp_workspace_bytes(const ntf_tucker* X, int rank, int mode) {
    TuckerView v;
    TuckerPlan P;
    if (make_tucker_view(X, &v) != NTF_OK || plan_tucker_mttkrp(v, rank, mode, &P) != NTF_OK) return 0;
    return P.total;
}

ntf_status ntf_tucker_mttkrp(const ntf_tucker* X, const float* const* factors, int rank, int mode, float* out,
                             void* workspace, size_t ws_bytes, void* stream) {
    TuckerView v;
    ntf_status s = make_tucker_view(X, &v);
    if (s != NTF_OK) return s;
    TuckerPlan P;
    if ((s = plan_tucker_mttkrp(v, rank, mode, &P)) != NTF_OK) return s;
    if ((s = check_tucker_ptrs(v)) != NTF_OK) return s;
    if (!factors) return fail(NTF_EINVAL, "factors is NULL");
    for (int l = 0; l < v.order; ++l)
        if (l != mode && (s = check_device_ptr(factors[l], "factor")) != NTF_OK) return s;
    if ((s = check_device_ptr(out, "out")) != NTF_OK) return s;
    if (!workspace || reinterpret_cast<uintptr_t>(workspace) % 256)
        return fail(NTF_EINVAL, "workspace must be a 256-byte aligned device buffer");
    if (ws_bytes < P.total) return fail(NTF_EINVAL, "workspace too small: need " + std::to_string(P.total) + " bytes");
    return run_tucker_mttkrp(v, P, factors, out, workspace, static_cast<cudaStream_t>(stream), nullptr);
}

size_t ntf_tucker_norm_workspace_bytes(const ntf_tucker* X) {
    TuckerView v;
    if (make_tucker_view(X, &v) != NTF_OK) return 0;
    return tucker_norm_workspace(v);
}

ntf_status ntf_tucker_norm_sq(const ntf_tucker* X, double* out_dev, void* workspace, size_t ws_bytes, void* stream) {
    TuckerView v;
    ntf_status s = make_tucker_view(X, &v);
    if (s != NTF_OK) return s;
    if ((s = check_tucker_ptrs(v)) != NTF_OK) return s;
    if ((s = check_device_ptr(out_dev, "out_dev")) != NTF_OK) return s;
    if (!workspace || reinterpret_cast<uintptr_t>(workspace) % 256)
        return fail(NTF_EINVAL, "workspace must be a 256-byte aligned device buffer");
    if (ws_bytes < tucker_norm_workspace(v)) return fail(NTF_EINVAL, "workspace too small");
    return run_tucker_norm_sq(v, out_dev, workspace, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
