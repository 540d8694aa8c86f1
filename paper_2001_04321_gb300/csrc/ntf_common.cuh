// Shared device/host helpers of libntf (CUDA path only; nothing here is used
// by the CPU oracle).  sm_103a: mbarrier, TMA (cp.async.bulk / .tensor) PTX.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stddef.h>

#include <atomic>
#include <string>
#include <utility>

#include "../../include/ntf.h"

namespace ntf {

// ---------------------------------------------------------------------------
// host-side error reporting
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);
ntf_status fail(ntf_status s, const std::string& msg);
ntf_status cuda_fail(cudaError_t e, const char* where);
void count_launch(int n = 1);
// NTF_EINVAL unless p is a non-NULL device (or managed) pointer
ntf_status check_device_ptr(const void* p, const char* what);

#define NTF_CUDA_TRY(expr)                                         \
    do {                                                           \
        cudaError_t _e = (expr);                                   \
        if (_e != cudaSuccess) return ::ntf::cuda_fail(_e, #expr); \
    } while (0)

#define NTF_LAUNCH_CHECK(name)                                     \
    do {                                                           \
        ::ntf::count_launch();                                     \
        cudaError_t _e = cudaGetLastError();                       \
        if (_e != cudaSuccess) return ::ntf::cuda_fail(_e, name);  \
    } while (0)

// Device-side error word shared by every kernel of the library.  Kernels set
// it (never trap) when a bounded wait runs out; the host reads it back.
int* device_error_word();   // device pointer (allocated once per device)

enum DeviceError : int {
    kErrNone = 0,
    kErrWaitFull = 1,    // a consumer gave up waiting for a stage
    kErrWaitEmpty = 2,   // the producer gave up waiting for a free stage
    kErrWaitDrain = 3,   // the producer gave up draining its copies
};

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }

// ---------------------------------------------------------------------------
// device PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Programmatic dependent launch.  A kernel launched with the programmatic
// stream-serialisation attribute may start while its predecessor in the
// stream is still running; pdl_wait() returns once the predecessor has
// completed and its memory operations are visible, so every kernel on the
// fused path calls it before touching anything another kernel wrote.  After
// the wait it lets its own successor launch (pdl_trigger); the successor then
// waits in turn, so at most two consecutive kernels are resident and no
// kernel reads data before its producer has finished.  Without the attribute
// both are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase of the given parity to complete, giving up after about
// two seconds of wall time.  Returns false on time-out (the caller records an
// error and stops); never spins forever.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_timer_ns() - t0 > 2000000000ull) return false;
    }
}

// 3-D tiled TMA load of one box into shared memory, completing on `bar`.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y,
                                            int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}

// Untiled bulk copy global -> shared (16-byte aligned, size multiple of 16).
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void prefetch_tensormap(const CUtensorMap* map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// Orders this thread's ordinary (generic-proxy) reads of shared memory before a later
// async-proxy write of the same bytes.  A warp that reads a TMA-filled buffer with ordinary
// loads runs it before it releases the buffer to the TMA producer: the mbarrier release alone
// let a refill land under loads still in flight (measured as wrong tiles once the compiler
// placed the release ahead of the loads' first use).
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Named barrier among the `count` threads that call it with the same id.
__device__ __forceinline__ void named_bar_sync(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

__device__ __forceinline__ void record_device_error(int* err, int code) {
    if (err) atomicCAS(err, 0, code);
}

// x rounded to TF32 (10 explicit mantissa bits), to nearest with ties away from zero: half a
// TF32 unit in the last place is added to the magnitude bits and the 13 bits below it are
// cleared (a carry runs into the exponent, and values past the largest TF32 number become
// infinity).  Integer arithmetic on the bit pattern: the conversion instruction was measured
// at about 860 cycles per 32 values and thread inside the tensor-core converters.
__device__ __forceinline__ float tf32_rna(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// bf16x2 word -> two floats (exact: a bfloat16 is the top half of a float)
__device__ __forceinline__ float bf16_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

// ---------------------------------------------------------------------------
// host: tensor map encoding through the driver entry point (no -lcuda)
// ---------------------------------------------------------------------------
ntf_status encode_tensor_map_3d(CUtensorMap* map, ntf_dtype dtype, const void* base, uint64_t d0, uint64_t d1,
                                uint64_t d2, uint64_t stride1_bytes, uint64_t stride2_bytes, uint32_t box0,
                                uint32_t box1, uint32_t box2);

#ifdef __CUDACC__
// launch with or without the programmatic stream-serialisation attribute
template <typename... KArgs, typename... Args>
inline cudaError_t launch_kernel(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                 bool pdl, Args&&... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = pdl ? attr : nullptr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}
#endif

}  // namespace ntf
