// extern "C" entry points of libntf: argument validation, error reporting and
// the single-step calls (steps a1-a8).  The solver lives in solver.cu.
#include "small.cuh"

#include <atomic>
#include <cmath>
#include <mutex>
#include <string>

namespace ntf {

static thread_local std::string g_last_error;
static std::atomic<int64_t> g_launches{0};

void set_error(const std::string& msg) { g_last_error = msg; }
ntf_status fail(ntf_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}
ntf_status cuda_fail(cudaError_t e, const char* where) {
    g_last_error = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return NTF_ECUDA;
}
void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// One error word per device, in a static device variable (no allocation).
__device__ int g_device_error_word;

int* device_error_word() {
    static int* addr[64] = {nullptr};
    static std::mutex mu;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_device_error_word) == cudaSuccess) addr[dev] = static_cast<int*>(p);
    }
    return addr[dev];
}

ntf_status check_device_ptr(const void* p, const char* what) {
    if (!p) return fail(NTF_EINVAL, std::string(what) + " is NULL");
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(NTF_EINVAL, std::string(what) + " is not a CUDA pointer");
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
        return fail(NTF_EINVAL, std::string(what) + " must be device memory");
    return NTF_OK;
}

static ntf_status check_rank(int rank) {
    if (rank < 1 || rank > NTF_MAX_RANK) return fail(NTF_EINVAL, "rank must be in [1, 64]");
    return NTF_OK;
}

#define NTF_TRY(expr)                     \
    do {                                  \
        ntf_status _s = (expr);           \
        if (_s != NTF_OK) return _s;      \
    } while (0)

}  // namespace ntf

using namespace ntf;

extern "C" {

const char* ntf_last_error(void) { return g_last_error.c_str(); }

int64_t ntf_launch_count(void) { return g_launches.load(); }

ntf_status ntf_device_status(void* stream) {
    NTF_CUDA_TRY(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    int* w = device_error_word();
    if (!w) return fail(NTF_ECUDA, "device error word unavailable");
    int v = 0;
    NTF_CUDA_TRY(cudaMemcpy(&v, w, sizeof(int), cudaMemcpyDeviceToHost));
    if (v != 0) {
        const int zero = 0;
        NTF_CUDA_TRY(cudaMemcpy(w, &zero, sizeof(int), cudaMemcpyHostToDevice));
        return fail(NTF_ETIMEOUT, "a kernel gave up a bounded wait (code " + std::to_string(v) + ")");
    }
    return NTF_OK;
}

ntf_status ntf_check_wait_timeout(int64_t limit_ns, void* stream) {
    if (limit_ns < 1000 || limit_ns > 2000000000ll) return fail(NTF_EINVAL, "limit_ns must be in [1e3, 2e9]");
    int* w = device_error_word();
    if (!w) return fail(NTF_ECUDA, "device error word unavailable");
    cudaError_t e = launch_wait_check(limit_ns, w, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "ntf_check_wait_timeout");
    return ntf_device_status(stream);
}

void ntf_opts_default(ntf_opts* o) {
    if (!o) return;
    o->her = 1;
    o->method = NTF_HALS;
    o->inner_max = 1;
    o->inner_tol = 1e-2;
    o->max_iters = 100;
    o->beta0 = 0.5;
    o->gamma = 1.05;
    o->gamma_bar = 1.01;
    o->eta = 1.5;
    o->compute_dtype = NTF_F32;
    o->report_every = 0;
    o->use_graph = 0;
    o->max_seconds = 0.0;
    o->rel_tol = 0.0;
    o->check_every = 10;
}

int64_t ntf_bf16_ld(const ntf_tensor* T) {
    if (!T || T->order < 2 || T->order > NTF_MAX_ORDER) return 0;
    return round_up(T->dims[T->order - 1], 8);
}

ntf_status ntf_tensor_to_bf16(const ntf_tensor* T, void* dst, int64_t dst_ld, void* stream) {
    TensorView v;
    NTF_TRY(make_view(T, &v));
    if (v.dtype != NTF_F32) return fail(NTF_EINVAL, "ntf_tensor_to_bf16: source must be NTF_F32");
    if (!dst || reinterpret_cast<uintptr_t>(dst) % 16) return fail(NTF_EINVAL, "dst must be 16-byte aligned");
    if (dst_ld < v.C || (dst_ld * 2) % 16) return fail(NTF_EINVAL, "dst_ld must be >= dims[N-1] and a multiple of 8");
    NTF_TRY(check_device_ptr(v.data, "tensor data"));
    NTF_TRY(check_device_ptr(dst, "dst"));
    cudaError_t e = launch_to_bf16(static_cast<const float*>(v.data), v.rows(), v.C, v.ld, dst, dst_ld,
                                   static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "ntf_tensor_to_bf16");
    return NTF_OK;
}

size_t ntf_norm_workspace_bytes(void) { return sizeof(double) * (size_t)stream_red_blocks(); }

ntf_status ntf_tensor_norm_sq(const ntf_tensor* T, double* out_dev, void* workspace, size_t ws_bytes,
                              void* stream) {
    TensorView v;
    NTF_TRY(make_view(T, &v));
    NTF_TRY(check_device_ptr(v.data, "tensor data"));
    NTF_TRY(check_device_ptr(out_dev, "out_dev"));
    if (!workspace || ws_bytes < ntf_norm_workspace_bytes()) return fail(NTF_EINVAL, "workspace too small");
    cudaError_t e = launch_norm_sq(v, static_cast<double*>(workspace), out_dev, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "ntf_tensor_norm_sq");
    return NTF_OK;
}

size_t ntf_mttkrp_workspace_bytes(const ntf_tensor* T, int rank, int mode) {
    TensorView v;
    MttkrpPlan P;
    if (make_view(T, &v) != NTF_OK || plan_mttkrp(v, rank, mode, &P) != NTF_OK) return 0;
    return P.total;
}

ntf_status ntf_mttkrp(const ntf_tensor* T, const float* const* factors, int rank, int mode, float* out,
                      void* workspace, size_t ws_bytes, void* stream) {
    TensorView v;
    NTF_TRY(make_view(T, &v));
    NTF_TRY(check_rank(rank));
    if (mode < 0 || mode >= v.order) return fail(NTF_EINVAL, "mode out of range");
    if (!factors) return fail(NTF_EINVAL, "factors is NULL");
    NTF_TRY(check_device_ptr(v.data, "tensor data"));
    for (int l = 0; l < v.order; ++l)
        if (l != mode) NTF_TRY(check_device_ptr(factors[l], "factor"));
    NTF_TRY(check_device_ptr(out, "out"));
    MttkrpPlan P;
    NTF_TRY(plan_mttkrp(v, rank, mode, &P));
    if (!workspace || reinterpret_cast<uintptr_t>(workspace) % 256)
        return fail(NTF_EINVAL, "workspace must be a 256-byte aligned device buffer");
    if (ws_bytes < P.total)
        return fail(NTF_EINVAL, "workspace too small: need " + std::to_string(P.total) + " bytes");
    return run_mttkrp(v, P, factors, out, workspace, static_cast<cudaStream_t>(stream), nullptr, nullptr);
}

ntf_status ntf_gram(const float* A, int64_t rows, int rank, double* G, void* stream) {
    NTF_TRY(check_rank(rank));
    if (rows < 1) return fail(NTF_EINVAL, "rows must be >= 1");
    NTF_TRY(check_device_ptr(A, "A"));
    NTF_TRY(check_device_ptr(G, "G"));
    cudaError_t e = launch_gram(A, rows, rank, G, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "ntf_gram");
    return NTF_OK;
}

ntf_status ntf_hadamard_grams(const double* const* grams, int order, int skip, int rank, double* V, void* stream) {
    NTF_TRY(check_rank(rank));
    if (order < 1 || order > NTF_MAX_ORDER) return fail(NTF_EINVAL, "order must be in [1, 8]");
    if (skip < -1 || skip >= order) return fail(NTF_EINVAL, "skip out of range");
    if (!grams) return fail(NTF_EINVAL, "grams is NULL");
    GramPtrs P{};
    for (int l = 0; l < order; ++l) {
        if (l != skip) NTF_TRY(check_device_ptr(grams[l], "gram"));
        P.g[l] = grams[l];
    }
    NTF_TRY(check_device_ptr(V, "V"));
    cudaError_t e = launch_hadamard(P, order, skip, rank, V, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "ntf_hadamard_grams");
    return NTF_OK;
}

size_t ntf_bcd_workspace_bytes(int64_t rows, int rank) {
    return (rows < 1 || rank < 1 || rank > NTF_MAX_RANK) ? 0 : bcd_workspace(rows, rank);
}

ntf_status ntf_bcd_update(ntf_method method, float* A, int64_t rows, int rank, const float* M, const double* V,
                          int inner_max, double inner_tol, void* workspace, size_t ws_bytes, void* stream) {
    NTF_TRY(check_rank(rank));
    if (method != NTF_HALS && method != NTF_PGD && method != NTF_NESTEROV) return fail(NTF_EINVAL, "unknown method");
    if (rows < 1) return fail(NTF_EINVAL, "rows must be >= 1");
    if (inner_max < 1) return fail(NTF_EINVAL, "inner_max must be >= 1");
    if (!(inner_tol >= 0.0)) return fail(NTF_EINVAL, "inner_tol must be >= 0");
    NTF_TRY(check_device_ptr(A, "A"));
    NTF_TRY(check_device_ptr(M, "M"));
    NTF_TRY(check_device_ptr(V, "V"));
    NTF_TRY(check_device_ptr(workspace, "workspace"));
    if (ws_bytes < bcd_workspace(rows, rank)) return fail(NTF_EINVAL, "workspace too small");
    cudaError_t e = launch_bcd((int)method, A, rows, rank, M, V, inner_max, inner_tol, workspace,
                               static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "ntf_bcd_update");
    return NTF_OK;
}

ntf_status ntf_block_gradient(const float* A, int64_t rows, int rank, const float* M, const double* V,
                              const double* scale_dev, double scale, float* out, void* stream) {
    NTF_TRY(check_rank(rank));
    if (rows < 1) return fail(NTF_EINVAL, "rows must be >= 1");
    NTF_TRY(check_device_ptr(A, "A"));
    NTF_TRY(check_device_ptr(M, "M"));
    NTF_TRY(check_device_ptr(V, "V"));
    NTF_TRY(check_device_ptr(out, "out"));
    if (scale_dev) NTF_TRY(check_device_ptr(scale_dev, "scale_dev"));
    cudaError_t e = launch_block_gradient(A, rows, rank, M, V, scale_dev, scale, out,
                                          static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "ntf_block_gradient");
    return NTF_OK;
}

ntf_status ntf_her_extrapolate(const float* A, const float* A_prev, const double* beta_dev, int64_t n, float* A_hat,
                               void* stream) {
    if (n < 1) return fail(NTF_EINVAL, "n must be >= 1");
    NTF_TRY(check_device_ptr(A, "A"));
    NTF_TRY(check_device_ptr(A_prev, "A_prev"));
    NTF_TRY(check_device_ptr(beta_dev, "beta_dev"));
    NTF_TRY(check_device_ptr(A_hat, "A_hat"));
    cudaError_t e = launch_extrapolate(A, A_prev, beta_dev, n, A_hat, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "ntf_her_extrapolate");
    return NTF_OK;
}

ntf_status ntf_objective(const double* tnorm_sq_dev, const float* M, const float* A, int64_t rows, int rank,
                         const double* V, double* out_dev, void* stream) {
    NTF_TRY(check_rank(rank));
    if (rows < 1) return fail(NTF_EINVAL, "rows must be >= 1");
    NTF_TRY(check_device_ptr(tnorm_sq_dev, "tnorm_sq_dev"));
    NTF_TRY(check_device_ptr(M, "M"));
    NTF_TRY(check_device_ptr(A, "A"));
    NTF_TRY(check_device_ptr(V, "V"));
    NTF_TRY(check_device_ptr(out_dev, "out_dev"));
    cudaError_t e = launch_objective(tnorm_sq_dev, M, A, rows, rank, V, out_dev, nullptr,
                                     static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "ntf_objective");
    return NTF_OK;
}

size_t ntf_residual_workspace_bytes(const ntf_tensor* T, int rank) {
    TensorView v;
    if (make_view(T, &v) != NTF_OK || rank < 1 || rank > NTF_MAX_RANK) return 0;
    const size_t w = ((sizeof(float) * (size_t)v.n_o * (size_t)round_up(rank, 4)) + 255) & ~size_t(255);
    return w + sizeof(double) * (size_t)stream_red_blocks();
}

ntf_status ntf_residual_sq(const ntf_tensor* T, const float* const* factors, int rank, double* out_dev,
                           void* workspace, size_t ws_bytes, void* stream) {
    TensorView v;
    NTF_TRY(make_view(T, &v));
    NTF_TRY(check_rank(rank));
    if (!factors) return fail(NTF_EINVAL, "factors is NULL");
    NTF_TRY(check_device_ptr(v.data, "tensor data"));
    for (int l = 0; l < v.order; ++l) NTF_TRY(check_device_ptr(factors[l], "factor"));
    NTF_TRY(check_device_ptr(out_dev, "out_dev"));
    NTF_TRY(check_device_ptr(workspace, "workspace"));
    if (reinterpret_cast<uintptr_t>(workspace) % 256) return fail(NTF_EINVAL, "workspace must be 256-byte aligned");
    if (ws_bytes < ntf_residual_workspace_bytes(T, rank)) return fail(NTF_EINVAL, "workspace too small");
    const int RP = (int)round_up(rank, 4);
    float* W = static_cast<float*>(workspace);
    const size_t woff = ((sizeof(float) * (size_t)v.n_o * RP) + 255) & ~size_t(255);
    double* parts = reinterpret_cast<double*>(static_cast<unsigned char*>(workspace) + woff);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = launch_weights_all(v, factors, rank, RP, W, st);
    if (e != cudaSuccess) return cuda_fail(e, "ntf_residual_sq(weights)");
    e = launch_residual_sq(v, rank, W, RP, factors[v.order - 2], factors[v.order - 1], parts, out_dev, st);
    if (e != cudaSuccess) return cuda_fail(e, "ntf_residual_sq");
    return NTF_OK;
}

ntf_status ntf_her_state_init(ntf_her_state* state_dev, double beta0, double gamma, double gamma_bar, double eta,
                              const double* f_hat0_dev, void* stream) {
    if (!(beta0 > 0.0 && beta0 < 1.0)) return fail(NTF_EINVAL, "beta0 must be in (0, 1) (Alg. 2)");
    if (!(1.0 < gamma_bar && gamma_bar <= gamma && gamma <= eta && std::isfinite(eta)))
        return fail(NTF_EINVAL, "need 1 < gamma_bar <= gamma <= eta (Sec. 3.1, eq. HER:relation)");
    NTF_TRY(check_device_ptr(state_dev, "state_dev"));
    NTF_TRY(check_device_ptr(f_hat0_dev, "f_hat0_dev"));
    cudaError_t e = launch_her_init(state_dev, beta0, gamma, gamma_bar, eta, f_hat0_dev,
                                    static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "ntf_her_state_init");
    return NTF_OK;
}

ntf_status ntf_her_step(ntf_her_state* state_dev, float* const* A, float* const* A_hat, int order,
                        const int64_t* rows, int rank, const double* f_hat_dev, void* stream) {
    NTF_TRY(check_rank(rank));
    if (order < 1 || order > NTF_MAX_ORDER) return fail(NTF_EINVAL, "order must be in [1, 8]");
    if (!A || !A_hat || !rows) return fail(NTF_EINVAL, "A, A_hat and rows must not be NULL");
    NTF_TRY(check_device_ptr(state_dev, "state_dev"));
    NTF_TRY(check_device_ptr(f_hat_dev, "f_hat_dev"));
    CopyPairs P;
    P.count = order;
    for (int l = 0; l < order; ++l) {
        if (rows[l] < 1) return fail(NTF_EINVAL, "rows must be >= 1");
        NTF_TRY(check_device_ptr(A[l], "A[l]"));
        NTF_TRY(check_device_ptr(A_hat[l], "A_hat[l]"));
        P.a[l] = A[l];
        P.ah[l] = A_hat[l];
        P.n[l] = rows[l] * rank;
    }
    P.gcount = 0;
    P.gn = 0;
    cudaError_t e = launch_her_step(state_dev, f_hat_dev, P, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "ntf_her_step");
    return NTF_OK;
}

}  // extern "C"
