// Tensor in host memory, streamed by slabs of mode 0 (see stream_host.cuh), and the
// ntf_mttkrp_streamed entry point.
//
// Slab s covers mode-0 indices [s S, min(I_0, (s+1) S)).  It is a tensor of the same order
// with dims[0] = its length, so the library's MTTKRP, norm and residual kernels run on it
// unchanged; mode 0's factor enters through a row offset.  For mode 0 the slab's MTTKRP is
// the output's rows of that slab; for every other mode it is a partial sum, added to the
// output in slab order (fixed order, bitwise reproducible).
#include "stream_host.cuh"

#include <string>

namespace ntf {

static inline size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

static size_t residual_ws(const TensorView& v, int r) {
    return al256(sizeof(float) * (size_t)v.n_o * (size_t)round_up(r, 4)) + sizeof(double) * (size_t)stream_red_blocks();
}

ntf_status slab_layout(const TensorView& host, int rank, int mode, int64_t slab_rows, SlabLayout* L) {
    const int N = host.order;
    L->per_index = host.ld;
    for (int l = 1; l < N - 1; ++l) L->per_index *= host.dims[l];
    const int64_t I0 = host.dims[0];
    if (slab_rows <= 0) slab_rows = std::max<int64_t>(1, (int64_t(64) << 20) / (L->per_index * host.es));
    L->slab = std::min<int64_t>(slab_rows, I0);
    L->nslabs = ceil_div(I0, L->slab);
    L->stage_bytes = (size_t)L->slab * (size_t)L->per_index * (size_t)host.es;
    size_t ws = 0, mrows = 0;
    for (int n = 0; n < N; ++n) {
        if (mode >= 0 && n != mode) continue;
        for (int k = 0; k < 2; ++k) {
            TensorView v = host;
            v.dims[0] = k == 0 ? L->slab : I0 - (L->nslabs - 1) * L->slab;
            if (N == 2) v.Ii = v.dims[0];
            else v.n_o = host.n_o / host.dims[0] * v.dims[0];
            ntf_status s = plan_mttkrp(v, rank, n, &L->plan[n][k]);
            if (s != NTF_OK) return s;
            ws = std::max(ws, L->plan[n][k].total);
            ws = std::max(ws, residual_ws(v, rank));
        }
        mrows = std::max<size_t>(mrows, (size_t)host.dims[n]);
    }
    ws = std::max(ws, sizeof(double) * (size_t)stream_red_blocks());
    size_t off = 0;
    L->off_stage[0] = off;
    off += al256(L->stage_bytes);
    L->off_stage[1] = off;
    off += al256(L->stage_bytes);
    L->off_M = off;
    off += al256(sizeof(float) * mrows * (size_t)rank);
    L->off_scal = off;
    off += al256(sizeof(double) * (size_t)L->nslabs);
    L->off_ws = off;
    off += al256(ws);
    L->total = off;
    return NTF_OK;
}

SlabStreamer::~SlabStreamer() {
    if (cst) cudaStreamDestroy(cst);
    if (ev_start) cudaEventDestroy(ev_start);
    for (int b = 0; b < 2; ++b) {
        if (copied[b]) cudaEventDestroy(copied[b]);
        if (freed[b]) cudaEventDestroy(freed[b]);
    }
}

ntf_status SlabStreamer::init(const TensorView& host_view, int r, int mode, int64_t slab_rows, void* workspace) {
    host = host_view;
    rank = r;
    ntf_status s = slab_layout(host, rank, mode, slab_rows, &L);
    if (s != NTF_OK) return s;
    ws = static_cast<unsigned char*>(workspace);
    NTF_CUDA_TRY(cudaStreamCreateWithFlags(&cst, cudaStreamNonBlocking));
    NTF_CUDA_TRY(cudaEventCreateWithFlags(&ev_start, cudaEventDisableTiming));
    for (int b = 0; b < 2; ++b) {
        NTF_CUDA_TRY(cudaEventCreateWithFlags(&copied[b], cudaEventDisableTiming));
        NTF_CUDA_TRY(cudaEventCreateWithFlags(&freed[b], cudaEventDisableTiming));
    }
    for (int n = 0; n < host.order; ++n) {
        if (mode >= 0 && n != mode) continue;
        for (int k = 0; k < 2; ++k) {
            TensorView v = slab_view(k == 0 ? 0 : L.nslabs - 1, 0);
            if ((s = configure_mttkrp(v, L.plan[n][k])) != NTF_OK) return s;
        }
    }
    return NTF_OK;
}

TensorView SlabStreamer::slab_view(int64_t s, int b) const {
    TensorView v = host;
    v.dims[0] = std::min(L.slab, host.dims[0] - s * L.slab);
    if (host.order == 2) v.Ii = v.dims[0];
    else v.n_o = host.n_o / host.dims[0] * v.dims[0];
    v.data = ws + L.off_stage[b];
    return v;
}

ntf_status SlabStreamer::fetch(int64_t s, cudaStream_t st) {
    const int b = (int)(s & 1);
    if (s == 0) {
        // the staging buffers may still be read by earlier work on st
        NTF_CUDA_TRY(cudaEventRecord(ev_start, st));
        NTF_CUDA_TRY(cudaStreamWaitEvent(cst, ev_start, 0));
    } else if (s >= 2) {
        NTF_CUDA_TRY(cudaStreamWaitEvent(cst, freed[b], 0));
    }
    const int64_t rows = std::min(L.slab, host.dims[0] - s * L.slab);
    const unsigned char* src = static_cast<const unsigned char*>(host.data) + (size_t)(s * L.slab) * L.per_index * host.es;
    NTF_CUDA_TRY(cudaMemcpyAsync(ws + L.off_stage[b], src, (size_t)rows * L.per_index * host.es,
                                 cudaMemcpyHostToDevice, cst));
    NTF_CUDA_TRY(cudaEventRecord(copied[b], cst));
    NTF_CUDA_TRY(cudaStreamWaitEvent(st, copied[b], 0));
    return NTF_OK;
}

ntf_status SlabStreamer::release(int64_t s, cudaStream_t st) {
    NTF_CUDA_TRY(cudaEventRecord(freed[s & 1], st));
    return NTF_OK;
}

ntf_status SlabStreamer::mttkrp(const float* const* factors, int mode, float* out, cudaStream_t st) {
    const int r = rank;
    float* Mslab = reinterpret_cast<float*>(ws + L.off_M);
    for (int64_t s = 0; s < L.nslabs; ++s) {
        ntf_status e = fetch(s, st);
        if (e != NTF_OK) return e;
        const TensorView v = slab_view(s, (int)(s & 1));
        const float* fac[NTF_MAX_ORDER];
        for (int l = 0; l < host.order; ++l) fac[l] = factors[l];
        if (mode != 0) fac[0] = factors[0] + s * L.slab * r;
        float* target = mode == 0 ? out + s * L.slab * r : (s == 0 ? out : Mslab);
        const MttkrpPlan& P = L.plan[mode][s == L.nslabs - 1 && L.nslabs > 1 ? 1 : 0];
        e = run_mttkrp(v, P, fac, target, ws + L.off_ws, st, nullptr, nullptr);
        if (e != NTF_OK) return e;
        if (mode != 0 && s > 0) {
            cudaError_t c = launch_add(out, Mslab, host.dims[mode] * r, st);
            if (c != cudaSuccess) return cuda_fail(c, "streamed MTTKRP: slab sum");
        }
        if ((e = release(s, st)) != NTF_OK) return e;
    }
    return NTF_OK;
}

ntf_status SlabStreamer::norm_sq(double* out, cudaStream_t st) {
    double* scal = reinterpret_cast<double*>(ws + L.off_scal);
    double* parts = reinterpret_cast<double*>(ws + L.off_ws);
    for (int64_t s = 0; s < L.nslabs; ++s) {
        ntf_status e = fetch(s, st);
        if (e != NTF_OK) return e;
        cudaError_t c = launch_norm_sq(slab_view(s, (int)(s & 1)), parts, scal + s, st);
        if (c != cudaSuccess) return cuda_fail(c, "streamed norm");
        if ((e = release(s, st)) != NTF_OK) return e;
    }
    cudaError_t c = launch_sum_parts(scal, (int)L.nslabs, out, st);
    return c == cudaSuccess ? NTF_OK : cuda_fail(c, "streamed norm: slab sum");
}

ntf_status SlabStreamer::residual_sq(const float* const* factors, double* out, cudaStream_t st) {
    const int r = rank, RP = (int)round_up(r, 4);
    double* scal = reinterpret_cast<double*>(ws + L.off_scal);
    for (int64_t s = 0; s < L.nslabs; ++s) {
        ntf_status e = fetch(s, st);
        if (e != NTF_OK) return e;
        const TensorView v = slab_view(s, (int)(s & 1));
        const float* fac[NTF_MAX_ORDER];
        for (int l = 0; l < host.order; ++l) fac[l] = factors[l];
        fac[0] = factors[0] + s * L.slab * r;
        float* W = reinterpret_cast<float*>(ws + L.off_ws);
        double* parts = reinterpret_cast<double*>(ws + L.off_ws + al256(sizeof(float) * (size_t)v.n_o * RP));
        cudaError_t c = launch_weights_all(v, fac, r, RP, W, st);
        if (c == cudaSuccess)
            c = launch_residual_sq(v, r, W, RP, fac[host.order - 2], fac[host.order - 1], parts, scal + s, st);
        if (c != cudaSuccess) return cuda_fail(c, "streamed residual");
        if ((e = release(s, st)) != NTF_OK) return e;
    }
    cudaError_t c = launch_sum_parts(scal, (int)L.nslabs, out, st);
    return c == cudaSuccess ? NTF_OK : cuda_fail(c, "streamed residual: slab sum");
}

// A view of a host tensor: the usual layout rules, and the data must not be device memory.
ntf_status make_host_view(const ntf_tensor* T, TensorView* v) {
    ntf_status s = make_view(T, v);
    if (s != NTF_OK) return s;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, v->data) != cudaSuccess) {
        cudaGetLastError();
        return NTF_OK;   // unregistered pageable memory on older drivers
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged)
        return fail(NTF_EINVAL, "T_host must be host memory (pinned for full copy speed)");
    return NTF_OK;
}

}  // namespace ntf

using namespace ntf;

extern "C" {

size_t ntf_mttkrp_streamed_workspace_bytes(const ntf_tensor* T_host, int rank, int mode, int64_t slab_rows) {
    TensorView v;
    SlabLayout L;
    if (make_view(T_host, &v) != NTF_OK || rank < 1 || rank > NTF_MAX_RANK || mode < 0 || mode >= v.order) return 0;
    if (slab_layout(v, rank, mode, slab_rows, &L) != NTF_OK) return 0;
    return L.total;
}

ntf_status ntf_mttkrp_streamed(const ntf_tensor* T_host, const float* const* factors, int rank, int mode, float* out,
                               void* workspace, size_t ws_bytes, int64_t slab_rows, void* stream) {
    TensorView v;
    ntf_status s = make_host_view(T_host, &v);
    if (s != NTF_OK) return s;
    if (rank < 1 || rank > NTF_MAX_RANK) return fail(NTF_EINVAL, "rank must be in [1, 64]");
    if (mode < 0 || mode >= v.order) return fail(NTF_EINVAL, "mode out of range");
    if (!factors) return fail(NTF_EINVAL, "factors is NULL");
    for (int l = 0; l < v.order; ++l)
        if (l != mode && (s = check_device_ptr(factors[l], "factor")) != NTF_OK) return s;
    if ((s = check_device_ptr(out, "out")) != NTF_OK) return s;
    if (!workspace || reinterpret_cast<uintptr_t>(workspace) % 256)
        return fail(NTF_EINVAL, "workspace must be a 256-byte aligned device buffer");
    if ((s = check_device_ptr(workspace, "workspace")) != NTF_OK) return s;
    SlabStreamer S;
    if ((s = S.init(v, rank, mode, slab_rows, workspace)) != NTF_OK) return s;
    if (ws_bytes < S.L.total)
        return fail(NTF_EINVAL, "workspace too small: need " + std::to_string(S.L.total) + " bytes");
    // the copy stream and events are released once the queued work completes
    return S.mttkrp(factors, mode, out, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
