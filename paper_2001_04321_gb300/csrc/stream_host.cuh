// A tensor that stays in host memory, streamed to the device by slabs of mode 0 (the paper's
// remark in Sec. 4 on data sets too large for its implementation's memory).  Each slab is one
// cudaMemcpyAsync on a copy stream into one of two staging buffers, double-buffered against the
// work on the slab before it.  Internal interface shared by stream_host.cu and the solver.
#pragma once

#include "small.cuh"

namespace ntf {

struct SlabLayout {
    int64_t slab = 0;              // mode-0 indices per slab
    int64_t nslabs = 0;
    int64_t per_index = 0;         // elements (with row padding) per mode-0 index
    size_t stage_bytes = 0;        // one staging buffer
    size_t off_stage[2], off_M, off_scal, off_ws, total;   // device workspace layout
    MttkrpPlan plan[NTF_MAX_ORDER][2];                      // [mode][full slab, last slab]
};

// A view of a host tensor: the usual layout rules, and the data must not be device memory.
ntf_status make_host_view(const ntf_tensor* T, TensorView* v);

// host: a view of host memory (validated like any tensor).  mode < 0 plans every mode.
ntf_status slab_layout(const TensorView& host, int rank, int mode, int64_t slab_rows, SlabLayout* L);

struct SlabStreamer {
    TensorView host;
    int rank = 0;
    SlabLayout L;
    unsigned char* ws = nullptr;   // device workspace of L.total bytes
    cudaStream_t cst = nullptr;    // copy stream
    cudaEvent_t ev_start = nullptr, copied[2] = {nullptr, nullptr}, freed[2] = {nullptr, nullptr};
    ~SlabStreamer();
    ntf_status init(const TensorView& host_view, int rank, int mode, int64_t slab_rows, void* workspace);
    // out (I_mode x rank) <- MTTKRP of `mode`; factors are device pointers
    ntf_status mttkrp(const float* const* factors, int mode, float* out, cudaStream_t st);
    // *out <- ||T||^2
    ntf_status norm_sq(double* out, cudaStream_t st);
    // *out <- ||T - [[A]]||^2, explicit per slab
    ntf_status residual_sq(const float* const* factors, double* out, cudaStream_t st);

   private:
    TensorView slab_view(int64_t s, int b) const;
    ntf_status fetch(int64_t s, cudaStream_t st);   // queue the copy of slab s, make st wait for it
    ntf_status release(int64_t s, cudaStream_t st); // st's work on slab s is queued: its buffer may be refilled
};

}  // namespace ntf
