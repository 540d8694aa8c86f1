// ntf_mttkrp_noalloc: the MTTKRP of ntf_mttkrp for callers that cannot
// allocate device memory.  Instead of a caller-provided workspace it uses a
// fixed-size scratch array that the library keeps in device memory.
//
// Who cannot allocate: code embedded in a host application that owns all
// device memory through its own allocator (and forbids cudaMalloc behind its
// back), latency-critical loops in which cudaMalloc/cudaFree are not
// acceptable (they can block and synchronise the device), and processes that
// run at their device-memory budget and must not grow it per call.
#include "mttkrp.cuh"

#include <mutex>

namespace ntf {
namespace {

// One scratch array per device, sized NTF_MTTKRP_NOALLOC_SCRATCH_BYTES (16 MiB);
// every GPU that loads the library holds it until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NTF_MTTKRP_NOALLOC_SCRATCH_BYTES];

// In host code `g_noalloc_scratch` names a host-side stand-in, not a device
// address.  The device address is looked up once per device, with that
// device current, on the first call made on it.
ntf_status noalloc_scratch_address(void** out) {
    static void* addr[64] = {nullptr};
    static std::mutex mu;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "ntf_mttkrp_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(NTF_ENOTSUP, "ntf_mttkrp_noalloc: device index above 63");
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(e, "ntf_mttkrp_noalloc: cudaGetSymbolAddress(scratch)");
        addr[dev] = p;
    }
    *out = addr[dev];
    return NTF_OK;
}

ntf_status noalloc_check_device_ptr(const void* p, const char* what) {
    if (!p) return fail(NTF_EINVAL, std::string(what) + " is NULL");
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return fail(NTF_EINVAL, std::string(what) + " is not a CUDA pointer");
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
        return fail(NTF_EINVAL, std::string(what) + " must be device memory");
    return NTF_OK;
}

}  // namespace
}  // namespace ntf

using namespace ntf;

extern "C" ntf_status ntf_mttkrp_noalloc(const ntf_tensor* T, const float* const* factors, int rank, int mode,
                                         float* out, void* stream) {
    TensorView v;
    ntf_status s = make_view(T, &v);
    if (s != NTF_OK) return s;
    if (rank < 1 || rank > NTF_MAX_RANK) return fail(NTF_EINVAL, "rank must be in [1, 64]");
    if (mode < 0 || mode >= v.order) return fail(NTF_EINVAL, "mode out of range");
    if (!factors) return fail(NTF_EINVAL, "factors is NULL");
    if ((s = noalloc_check_device_ptr(v.data, "tensor data")) != NTF_OK) return s;
    for (int l = 0; l < v.order; ++l)
        if (l != mode && (s = noalloc_check_device_ptr(factors[l], "factor")) != NTF_OK) return s;
    if ((s = noalloc_check_device_ptr(out, "out")) != NTF_OK) return s;
    MttkrpPlan P;
    if ((s = plan_mttkrp(v, rank, mode, &P)) != NTF_OK) return s;
    if (P.total > (size_t)NTF_MTTKRP_NOALLOC_SCRATCH_BYTES)
        return fail(NTF_EINVAL, "ntf_mttkrp_noalloc: this tensor, rank and mode need " + std::to_string(P.total) +
                                    " bytes of scratch but the fixed scratch holds " +
                                    std::to_string((size_t)NTF_MTTKRP_NOALLOC_SCRATCH_BYTES) +
                                    " bytes; call ntf_mttkrp with a workspace of ntf_mttkrp_workspace_bytes()");
    void* scratch = nullptr;
    if ((s = noalloc_scratch_address(&scratch)) != NTF_OK) return s;
    // Nothing in the scratch has to start at zero: every byte the kernels read
    // is written earlier in the same call.
    return run_mttkrp(v, P, factors, out, scratch, static_cast<cudaStream_t>(stream), nullptr, nullptr);
}
