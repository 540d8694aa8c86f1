// Device-resident solver: Alg. 1 (plain BCD) and Alg. 2 (HER) with HALS or
// projected-gradient block updates.  One outer iteration is a fixed sequence
// of kernels on one stream with no host round trip (the restart decision is
// taken on the device), so it can also be replayed as a CUDA graph.
#include "small.cuh"
#include "epilogue.cuh"
#include "stream_host.cuh"
#include "tucker.cuh"

#include <cstdlib>

#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

namespace ntf {

struct Solver {
    TensorView vu;           // tensor as given (quality is reported against it)
    TensorView vs;           // tensor streamed by the MTTKRP (vu or its bf16 copy)
    void* bf16_copy = nullptr;
    void* owned_T = nullptr; // device copy made by ntf_solve_host
    int N = 0, r = 0;
    ntf_opts o;
    // two buffers per mode (factor and Gram); the fused path flips cur[] on an
    // accepted extrapolation, the general path keeps A in buffer 0 and copies
    float* X[NTF_MAX_ORDER][2] = {{nullptr}};
    double* GB[NTF_MAX_ORDER][2] = {{nullptr}};
    int* cur = nullptr;         // device [NTF_MAX_ORDER]
    int* iters_dev = nullptr;   // device: [0] completed outer iterations, [1] end-of-iteration ticket
    float* A[NTF_MAX_ORDER] = {nullptr};
    float* Ah[NTF_MAX_ORDER] = {nullptr};
    double* G[NTF_MAX_ORDER] = {nullptr};   // Grams of A
    double* Gh[NTF_MAX_ORDER] = {nullptr};  // Grams of A_hat
    float* Aprev = nullptr;
    float* M = nullptr;
    double* V = nullptr;
    float* Vf = nullptr;        // V in FP32 for the fused epilogue
    double* scal = nullptr;  // [0] ||T_s||^2 [1] F-hat [2] f_true [3] F-hat_0 [4] ||T_u||^2
    ntf_her_state* her = nullptr;
    void* ws_mt = nullptr;
    void* ws_bcd = nullptr;
    void* ws_res = nullptr;
    size_t ws_res_bytes = 0;
    MttkrpPlan plan[NTF_MAX_ORDER];
    TmapCache tm[NTF_MAX_ORDER];
    std::vector<void*> allocs;
    int iters_done = 0;
    double seconds = 0.0;
    // timing of the streaming kernels: every timing_every-th iteration has CUDA
    // events around its streaming launches (0 = off)
    bool timing = false;
    int timing_every = 0;
    int64_t iter_seq = 0;      // iterations issued (eagerly or into the graph being captured)
    bool timed_now = false;    // the iteration being issued is timed
    // programmatic dependent launch on the fused path (off with NTF_PDL=0)
    bool pdl = true;
    std::vector<StreamTimer> ev;
    size_t ev_used = 0;
    // fused main path (HALS, one sweep, rank <= 32)
    bool fused = false;
    float* gpart = nullptr;
    double* ipart = nullptr;
    double* qpart = nullptr;
    unsigned char* wsm[NTF_MAX_ORDER] = {nullptr};   // each mode's MTTKRP workspace (inside ws_mt)
    // 3-way tensor-core path without k_prep
    bool direct = false;
    bool prepped = false;
    __nv_bfloat16* packRows[2] = {nullptr, nullptr};   // packed A_{N-1} of buffer k (row streams)
    __nv_bfloat16* packLast = nullptr;                 // packed pairing factor of the last-mode stream:
                                                       // A_{N-2} (last-mode kernel) or A_0 (perm)
    // second layout of the streamed tensor with its modes reversed, (I_2, I_1, I_0): the last
    // mode's MTTKRP then runs the row-stream kernel (outer mode 0 of that layout)
    bool perm = false;
    TensorView vperm;
    // 4-way tensor-core path: modes 0 and 1 stream the tensor viewed as (I_0, I_1, I_2 I_3)
    // against the packed Khatri-Rao rows of (A_2, A_3); modes 2 and 3 stream a resident copy laid
    // out as (I_2, I_3, I_0 I_1) against those of (A_hat_0, A_hat_1).  Every MTTKRP still reads
    // one full copy, but the contraction runs over I_2 I_3 (or I_0 I_1) columns instead of I_3.
    bool direct4 = false;
    TensorView vmode[NTF_MAX_ORDER];
    void* packKR[2] = {nullptr, nullptr};   // [0]: rows of (A_2, A_3); [1]: rows of (A_hat_0, A_hat_1)
    // graph replay: one graph holds g_iters outer iterations (and, when timing is
    // on, the event records around each MTTKRP stream, read after the replay)
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t gstream = nullptr;
    int g_iters = 0;
    int g_timing = 0;          // timing_every the graph was captured with
    int64_t g_kernels = 0;   // kernel nodes in the graph
    // data term of the general path: a dense tensor in device memory, Tucker-format data
    // (Appendix A), or a dense tensor in host memory streamed by slabs
    enum class Src { Dense, Tucker, Streamed };
    Src src = Src::Dense;
    TuckerView tk;
    TuckerPlan tkp[NTF_MAX_ORDER];
    void* ws_tk = nullptr;
    SlabStreamer* ss = nullptr;
    // objective by the identity (Tucker data): Grams and V at A_k, the last mode's MTTKRP
    double* Grep[NTF_MAX_ORDER] = {nullptr};
    double* Vrep = nullptr;
    float* Mrep = nullptr;
    double* gparts = nullptr;   // partial sums of the many-row Grams of the general path

    ~Solver() {
        delete ss;   // its streams and events; its workspace is one of allocs
        if (gexec) cudaGraphExecDestroy(gexec);
        for (auto& t : ev) {
            if (t.start) cudaEventDestroy(t.start);
            if (t.stop) cudaEventDestroy(t.stop);
        }
        for (void* p : allocs) cudaFree(p);
    }

    ntf_status alloc(void** p, size_t bytes) {
        if (bytes == 0) bytes = 16;
        cudaError_t e = cudaMalloc(p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            *p = nullptr;
            return fail(NTF_ENOMEM, std::string("cudaMalloc(") + std::to_string(bytes) + ") failed");
        }
        allocs.push_back(*p);
        return NTF_OK;
    }

    StreamTimer* next_timer() {
        if (!timing || !timed_now) return nullptr;
        if (ev_used == ev.size()) {
            StreamTimer t;
            if (cudaEventCreate(&t.start) != cudaSuccess || cudaEventCreate(&t.stop) != cudaSuccess) {
                cudaGetLastError();
                return nullptr;
            }
            ev.push_back(t);
        }
        return &ev[ev_used++];
    }

    CopyPairs her_pairs() const {
        CopyPairs P;
        P.count = N;
        P.gcount = N;
        P.gn = r * r;
        for (int l = 0; l < N; ++l) {
            P.a[l] = A[l];
            P.ah[l] = Ah[l];
            P.n[l] = vs.dims[l] * r;
            P.g[l] = G[l];
            P.gh[l] = Gh[l];
        }
        return P;
    }

    FusedBufs fused_bufs() const {
        FusedBufs B{};
        for (int l = 0; l < N; ++l)
            for (int k = 0; k < 2; ++k) {
                B.X[l][k] = X[l][k];
                B.GB[l][k] = GB[l][k];
            }
        B.cur = cur;
        B.iters = iters_dev;
        B.her = o.her;
        return B;
    }

    // preparation of mode n's stream: V_n, the finished Grams of the mode before, and
    // the packed operands in mode n's workspace
    PrepParams make_prep(int n) const {
        const bool use_her = o.her != 0;
        unsigned char* ws = wsm[n];
        const MttkrpPlan& P = plan[n];
        PrepParams pp{};
        pp.B = fused_bufs();
        pp.order = N;
        pp.mode = n;
        pp.skip = P.kind == ModeKind::Outer ? n : -1;
        pp.r = r;
        pp.RP = P.RP;
        pp.C = vs.C;
        pp.Ii = vs.Ii;
        pp.n_o = vs.n_o;
        pp.Fc_rows_out = round_up(vs.C, 64);
        for (int l = 0; l < N; ++l) pp.dims[l] = vs.dims[l];
        pp.V = V;
        pp.Vf = Vf;
        pp.Fc = (P.kind != ModeKind::Last && !P.tc) ? reinterpret_cast<float*>(ws + P.off_Fc) : nullptr;
        pp.FcT = P.tc ? reinterpret_cast<__nv_bfloat16*>(ws + P.off_Fc) : nullptr;
        pp.RPH = P.RPH;
        pp.fct_tf32 = P.tf32 ? 1 : 0;
        if (P.kind == ModeKind::Last) {      // tensor-core last mode: A_{N-2} by row blocks
            pp.fct_mode = N - 2;
            pp.fct_rows = vs.Ii;
            pp.n_kc = (int)(P.tf32 ? P.nb : 2 * P.nb);   // 32-row chunks (tf32) or two 64-row ones
        } else {
            pp.fct_mode = N - 1;
            pp.fct_rows = vs.C;
            pp.n_kc = P.n_kc;
        }
        pp.Fi = (P.kind != ModeKind::Inner && !(P.tc && P.kind == ModeKind::Last))
                    ? reinterpret_cast<float*>(ws + P.off_Fi)
                    : nullptr;
        pp.W = reinterpret_cast<float*>(ws + P.off_W);
        pp.sched = P.tile_slots ? reinterpret_cast<unsigned int*>(ws + P.off_sched) : nullptr;
        pp.fin_mode = n > 0 ? n - 1 : N - 1;
        pp.fin_blocks = epilogue_blocks(vs.dims[pp.fin_mode]);
        pp.gpart = gpart;
        pp.her = use_her ? her : nullptr;
        return pp;
    }

    EpiParams make_epi(int n) const {
        const bool use_her = o.her != 0;
        unsigned char* ws = wsm[n];
        const MttkrpPlan& P = plan[n];
        EpiParams ep{};
        ep.B = fused_bufs();
        ep.red = make_reduce_params(stream_view(n), P, reinterpret_cast<const float*>(ws + P.off_part),
                                    reinterpret_cast<const float*>(ws + P.off_W));
        ep.mode = n;
        ep.order = N;
        ep.rows = vs.dims[n];
        ep.r = r;
        ep.last = n == N - 1 ? 1 : 0;
        ep.beta = &her->beta;
        ep.V = V;
        ep.Vf = Vf;
        ep.gpart = gpart;
        ep.ipart = ipart;
        ep.qpart = qpart;
        ep.ticket = iters_dev + 1;
        ep.tnorm = &scal[0];
        ep.fhat_out = &scal[1];
        ep.iters_out = iters_dev;
        ep.her = use_her ? her : nullptr;
        return ep;
    }

    // The 3-way tensor-core path runs without k_prep: the stream kernels read W and
    // A_{N-2} straight from the factor buffers (chosen on the device from cur[]), take
    // their packed operand from buffers the epilogues write, and finish the Grams and V
    // for the epilogue that follows them in their idle epilogue warps.  k_prep runs once,
    // before the first stream.
    ntf_status ensure_prepped(cudaStream_t st) {
        if (!direct || prepped) return NTF_OK;
        PrepParams pp = make_prep(0);
        pp.FcT = packRows[0];            // cur is 0 before the first decision
        pp.fin_mode = -1;
        cudaError_t e = launch_prep(pp, st, false);
        if (e != cudaSuccess) return cuda_fail(e, "prep");
        prepped = true;
        return NTF_OK;
    }

    // the tensor layout mode n's MTTKRP streams
    const TensorView& stream_view(int n) const {
        if (direct4) return vmode[n];
        return (perm && n == N - 1) ? vperm : vs;
    }

    TcParams direct4_stream(int n) const {
        const bool use_her = o.her != 0;
        TcParams T = direct_stream(n);
        const unsigned char* pk = reinterpret_cast<const unsigned char*>(packKR[n / 2]);
        T.FcTb[0] = T.FcTb[1] = pk;
        T.fct_sel = 0;
        T.early = 0;
        const int lead = n < 2 ? 0 : 2;     // the view's outer mode
        // outer kind (n = 0, 2): its rows are mode lead + 1, not yet updated this iteration
        T.Fib[0] = X[lead + 1][0];
        T.Fib[1] = X[lead + 1][1];
        T.fi_sel = lead + 1;
        T.fi_flip = 0;
        // inner kind (n = 1, 3): its outer index is mode lead, updated: the pairing A_hat
        T.Wb[0] = X[lead][0];
        T.Wb[1] = X[lead][1];
        T.w_sel = lead;
        T.w_flip = use_her ? 1 : 0;
        return T;
    }

    // one outer iteration on the 4-way tensor-core path: two Khatri-Rao operand packs, and per
    // mode a stream and an epilogue (the last epilogue takes F_hat, the decision and the flip)
    ntf_status iterate_direct4(cudaStream_t st) {
        const bool use_her = o.her != 0;
        for (int n = 0; n < N; ++n) {
            if (n == 0 || n == 2) {
                // n = 0: (A_2, A_3) as the last decision left them; n = 2: the pairing A_hat of
                // modes 0 and 1 (eq. NNLS_her_exact).  Launched in plain stream order.
                KrPack K{};
                const int a = n == 0 ? 2 : 0, b = a + 1;
                K.a[0] = X[a][0];
                K.a[1] = X[a][1];
                K.b[0] = X[b][0];
                K.b[1] = X[b][1];
                K.cur = cur;
                K.sel_a = a;
                K.sel_b = b;
                K.flip_a = K.flip_b = (n == 2 && use_her) ? 1 : 0;
                K.Ia = vs.dims[a];
                K.Ib = vs.dims[b];
                K.r = r;
                K.RPH = plan[n].RPH;
                K.n_kc = plan[n].n_kc;
                K.tf32 = plan[n].tf32 ? 1 : 0;
                K.out = packKR[n / 2];
                cudaError_t e = launch_pack_kr(K, st);
                if (e != cudaSuccess) return cuda_fail(e, "Khatri-Rao operand");
            }
            StreamTimer* timer = next_timer();
            const TcParams T = direct4_stream(n);
            ntf_status s = run_mttkrp_stream(vmode[n], plan[n], wsm[n], st, &tm[n], timer, pdl, &T);
            if (s != NTF_OK) return s;
            EpiParams ep = make_epi(n);
            const int nx = (n + 2) % N;
            ep.sched_next = plan[nx].tile_slots ? reinterpret_cast<unsigned int*>(wsm[nx] + plan[nx].off_sched) : nullptr;
            ep.v_from_stream = 1;
            cudaError_t e = launch_epilogue(ep, st, pdl && !timer);
            if (e != cudaSuccess) return cuda_fail(e, "epilogue");
        }
        return NTF_OK;
    }

    // Whether stream n may run ahead of the epilogue before it (TcParams::early).  Its producer
    // and MMA warps then skip the programmatic-launch wait and trigger the launch of the
    // epilogue after the stream while epilogue n-1 may still run.  That next epilogue reads
    // cur[n], its factor row in X[n][cur], beta and V (when not formed by the stream) before
    // its own wait, and the stream reads its packed operand and tile counter without waiting;
    // so epilogue n-1 must write none of these.  The last mode's epilogue writes cur, beta,
    // F-hat and the rows streams' packed operand (n = 0 excluded).  The packed operand of the
    // last-mode stream comes from epilogue N-2 for the last-mode kernel (n = N-1 excluded) and
    // from epilogue 0 on the reversed copy (allowed: two launches back).  Every other epilogue
    // writes only its own factor buffers, Gram partials and objective partials.  Every tile
    // counter is reset by the epilogue two launches ahead of its stream.
    bool early_stream_ok(int n) const { return n >= 1 && (n < N - 1 || (perm && n == N - 1 && N == 3)); }

    TcParams direct_stream(int n) const {
        const bool use_her = o.her != 0;
        TcParams T{};
        T.ldw = r;
        T.cur = cur;
        if (n < N - 1) {
            T.FcTb[0] = reinterpret_cast<const unsigned char*>(packRows[0]);
            T.FcTb[1] = reinterpret_cast<const unsigned char*>(packRows[1]);
            T.fct_sel = N - 1;
        } else if (perm) {
            // last mode = outer mode 0 of the (I_2, I_1, I_0) layout: it contracts the I_0 index
            // with the packed pairing A_0 and weights its I_1 rows by the pairing A_1
            T.FcTb[0] = T.FcTb[1] = reinterpret_cast<const unsigned char*>(packLast);
            T.fct_sel = 0;
        } else {
            T.FcTb[0] = T.FcTb[1] = reinterpret_cast<const unsigned char*>(packLast);
            T.fct_sel = 0;
        }
        // 3-way: the outer mode's row weights are A_1 (not yet updated), the inner and last
        // modes' W is A_0's pairing factor (A_hat_0 with HER)
        T.Fib[0] = X[1][0];
        T.Fib[1] = X[1][1];
        T.fi_sel = 1;
        T.fi_flip = 0;
        T.Wb[0] = X[0][0];
        T.Wb[1] = X[0][1];
        T.w_sel = 0;
        T.w_flip = (use_her && n > 0) ? 1 : 0;
        if (perm && n == N - 1) {
            T.fi_flip = use_her ? 1 : 0;    // rows I_1: the pairing A_hat_1
        }
        // mode 1's packed operand and buffer index come from the previous iteration's last
        // epilogue, and (on the reversed copy) mode 2's from the mode-0 epilogue; their tile
        // counters are reset two launches ahead: these tensors can stream in while the epilogue
        // before them runs
        T.early = early_stream_ok(n) ? 1 : 0;
        GramJob& J = T.job;
        J.rr = r * r;
        J.order = N;
        J.mode = n;
        J.fin_mode = n > 0 ? n - 1 : N - 1;
        J.fin_blocks = epilogue_blocks(vs.dims[J.fin_mode]);
        J.her = use_her ? 1 : 0;
        J.gpart = gpart;
        for (int l = 0; l < N; ++l)
            for (int k = 0; k < 2; ++k) J.GB[l][k] = GB[l][k];
        J.V = V;
        J.Vf = Vf;
        J.cur = cur;
        J.iters = iters_dev;
        J.hs = use_her ? her : nullptr;
        return T;
    }

    // one outer iteration on the fused path: per mode (prep ->) stream -> epilogue;
    // the last epilogue also takes F_hat, the decision and the buffer flip
    ntf_status iterate_fused(cudaStream_t st) {
        if (direct && !prepped) return fail(NTF_EINVAL, "internal: fused iteration before its first preparation");
        const bool use_her = o.her != 0;
        for (int n = 0; n < N; ++n) {
            const MttkrpPlan& P = plan[n];
            if (!direct) {
                cudaError_t e = launch_prep(make_prep(n), st, pdl);
                if (e != cudaSuccess) return cuda_fail(e, "prep");
            }
            // a kernel right after an event record is launched without the PDL attribute
            StreamTimer* timer = next_timer();
            ntf_status s;
            if (direct) {
                const TcParams T = direct_stream(n);
                s = run_mttkrp_stream(stream_view(n), P, wsm[n], st, &tm[n], timer, pdl, &T);
            } else {
                s = run_mttkrp_stream(vs, P, wsm[n], st, &tm[n], timer, pdl);
            }
            if (s != NTF_OK) return s;
            EpiParams ep = make_epi(n);
            if (direct) {
                // the tile counter of the stream after next (two kernels before its launch, so
                // that an early stream does not depend on the epilogue right before it)
                const int nx = (n + 2) % N;
                const MttkrpPlan& Q = plan[nx];
                ep.sched_next = Q.tile_slots ? reinterpret_cast<unsigned int*>(wsm[nx] + Q.off_sched) : nullptr;
                ep.v_from_stream = 1;
                if (n == N - 1) {
                    // the next iteration's row streams read A_{N-1} (or A_hat_{N-1} after an accept)
                    ep.packA[0] = ep.packH[0] = packRows[0];
                    ep.packA[1] = ep.packH[1] = packRows[1];
                    ep.pack_rph = plan[0].RPH;
                    ep.pack_tf32 = plan[0].tf32 ? 1 : 0;
                } else if (perm ? n == 0 : n == N - 2) {
                    // the last-mode stream reads the pairing factor of mode N-2, or of mode 0 on
                    // the reversed copy
                    if (use_her) ep.packH[0] = ep.packH[1] = packLast;
                    else ep.packA[0] = ep.packA[1] = packLast;
                    ep.pack_rph = plan[N - 1].RPH;
                    ep.pack_tf32 = plan[N - 1].tf32 ? 1 : 0;
                }
            }
            cudaError_t e = launch_epilogue(ep, st, pdl && !timer);
            if (e != cudaSuccess) return cuda_fail(e, "epilogue");
        }
        return NTF_OK;
    }

    // device pointers of the current factors A_k (synchronises `st`)
    ntf_status current_factors(cudaStream_t st, float** out) {
        int h[NTF_MAX_ORDER] = {0};
        NTF_CUDA_TRY(cudaMemcpyAsync(h, cur, sizeof(int) * NTF_MAX_ORDER, cudaMemcpyDeviceToHost, st));
        NTF_CUDA_TRY(cudaStreamSynchronize(st));
        for (int l = 0; l < N; ++l) out[l] = X[l][h[l] & 1];
        return NTF_OK;
    }

    // one outer iteration of Alg. 2 (or Alg. 1 when her == 0)
    ntf_status iterate(cudaStream_t st) {
        timed_now = timing_every > 0 && (iter_seq % timing_every) == 0;
        ++iter_seq;
        if (direct4) return iterate_direct4(st);
        if (fused) return iterate_fused(st);
        const bool use_her = o.her != 0;
        for (int n = 0; n < N; ++n) {
            const int64_t rows = vs.dims[n];
            GramPtrs gp{};
            for (int l = 0; l < N; ++l) gp.g[l] = Gh[l];
            cudaError_t e = launch_hadamard(gp, N, n, r, V, st);
            if (e != cudaSuccess) return cuda_fail(e, "hadamard");
            const float* fac[NTF_MAX_ORDER];
            for (int l = 0; l < N; ++l) fac[l] = Ah[l];
            ntf_status s = mttkrp_general(n, fac, M, st);
            if (s != NTF_OK) return s;
            if (use_her) NTF_CUDA_TRY(cudaMemcpyAsync(Aprev, A[n], sizeof(float) * rows * r, cudaMemcpyDeviceToDevice, st));
            e = launch_bcd((int)o.method, A[n], rows, r, M, V, o.inner_max, o.inner_tol, ws_bcd, st);
            if (e != cudaSuccess) return cuda_fail(e, "block update");
            if (use_her) {
                e = launch_extrapolate(A[n], Aprev, &her->beta, rows * r, Ah[n], st);
                if (e != cudaSuccess) return cuda_fail(e, "extrapolate");
                e = launch_gram_parts(A[n], rows, r, G[n], gparts, st);
                if (e != cudaSuccess) return cuda_fail(e, "gram");
            }
            e = launch_gram_parts(Ah[n], rows, r, Gh[n], gparts, st);
            if (e != cudaSuccess) return cuda_fail(e, "gram");
        }
        // F-hat_k = ||T||^2 - 2 <M_{N-1}, A_{N-1}> + sum(V_{N-1} (*) G(A_{N-1}))   (Alg. 2, restart test)
        const int last = N - 1;
        // the Gram of A_{N-1} was just formed (into G with HER, else into Gh, the same factor)
        cudaError_t e = launch_objective(&scal[0], M, A[last], vs.dims[last], r, V, &scal[1], nullptr, st,
                                         use_her ? G[last] : Gh[last]);
        if (e != cudaSuccess) return cuda_fail(e, "objective");
        if (use_her) {
            CopyPairs P;
            P.count = N;
            P.gcount = N;
            P.gn = r * r;
            for (int l = 0; l < N; ++l) {
                P.a[l] = A[l];
                P.ah[l] = Ah[l];
                P.n[l] = vs.dims[l] * r;
                P.g[l] = G[l];
                P.gh[l] = Gh[l];
            }
            e = launch_her_step(her, &scal[1], P, st);
            if (e != cudaSuccess) return cuda_fail(e, "her step");
        }
        return NTF_OK;
    }

    // M_n against `fac` by the data term of this solver (the general path)
    ntf_status mttkrp_general(int n, const float* const* fac, float* out, cudaStream_t st) {
        if (src == Src::Tucker) return run_tucker_mttkrp(tk, tkp[n], fac, out, ws_tk, st, &tm[n]);
        if (src == Src::Streamed) return ss->mttkrp(fac, n, out, st);
        return run_mttkrp(vs, plan[n], fac, out, ws_mt, st, &tm[n], next_timer());
    }

    // ||T - [[A_k]]||^2 at the current factors: explicit for dense data (in device memory or
    // streamed); for Tucker data by the identity of the restart test with a fresh MTTKRP
    ntf_status residual(const TensorView& v, double* out, cudaStream_t st) {
        if (src != Src::Dense) {
            float* facs[NTF_MAX_ORDER];
            ntf_status s = current_factors(st, facs);
            if (s != NTF_OK) return s;
            const float* fac[NTF_MAX_ORDER];
            for (int l = 0; l < N; ++l) fac[l] = facs[l];
            if (src == Src::Streamed) return ss->residual_sq(fac, out, st);
            GramPtrs gp{};
            for (int l = 0; l < N; ++l) {
                cudaError_t e = launch_gram_parts(fac[l], vu.dims[l], r, Grep[l], gparts, st);
                if (e != cudaSuccess) return cuda_fail(e, "gram");
                gp.g[l] = Grep[l];
            }
            cudaError_t e = launch_hadamard(gp, N, N - 1, r, Vrep, st);
            if (e != cudaSuccess) return cuda_fail(e, "hadamard");
            s = run_tucker_mttkrp(tk, tkp[N - 1], fac, Mrep, ws_tk, st, &tm[N - 1]);
            if (s != NTF_OK) return s;
            e = launch_objective(&scal[0], Mrep, fac[N - 1], vu.dims[N - 1], r, Vrep, out, nullptr, st, Grep[N - 1]);
            return e == cudaSuccess ? NTF_OK : cuda_fail(e, "objective");
        }
        const int RP = (int)round_up(r, 4);
        float* W = static_cast<float*>(ws_res);
        const size_t woff = ((sizeof(float) * (size_t)v.n_o * RP) + 255) & ~size_t(255);
        double* parts = reinterpret_cast<double*>(static_cast<unsigned char*>(ws_res) + woff);
        float* facs[NTF_MAX_ORDER];
        ntf_status s = current_factors(st, facs);
        if (s != NTF_OK) return s;
        const float* fac[NTF_MAX_ORDER];
        for (int l = 0; l < N; ++l) fac[l] = facs[l];
        cudaError_t e = launch_weights_all(v, fac, r, RP, W, st);
        if (e != cudaSuccess) return cuda_fail(e, "residual weights");
        e = launch_residual_sq(v, r, W, RP, fac[N - 2], fac[N - 1], parts, out, st);
        if (e != cudaSuccess) return cuda_fail(e, "residual");
        return NTF_OK;
    }
};

static ntf_status validate_opts(const ntf_opts& o) {
    if (o.her != 0 && o.her != 1) return fail(NTF_EINVAL, "opts.her must be 0 or 1");
    if (o.method != NTF_HALS && o.method != NTF_PGD && o.method != NTF_NESTEROV)
        return fail(NTF_EINVAL, "opts.method unknown");
    if (o.inner_max < 1) return fail(NTF_EINVAL, "opts.inner_max must be >= 1");
    if (!(o.inner_tol >= 0.0)) return fail(NTF_EINVAL, "opts.inner_tol must be >= 0");
    if (o.max_iters < 0) return fail(NTF_EINVAL, "opts.max_iters must be >= 0");
    if (o.compute_dtype != NTF_F32 && o.compute_dtype != NTF_BF16) return fail(NTF_EINVAL, "opts.compute_dtype unknown");
    if (o.her) {
        if (!(o.beta0 > 0.0 && o.beta0 < 1.0)) return fail(NTF_EINVAL, "opts.beta0 must be in (0, 1) (Alg. 2)");
        if (!(1.0 < o.gamma_bar && o.gamma_bar <= o.gamma && o.gamma <= o.eta && std::isfinite(o.eta)))
            return fail(NTF_EINVAL, "need 1 < gamma_bar <= gamma <= eta (Sec. 3.1, eq. HER:relation)");
    }
    if (!(o.max_seconds >= 0.0) || !(o.rel_tol >= 0.0))
        return fail(NTF_EINVAL, "opts.max_seconds and opts.rel_tol must be >= 0");
    return NTF_OK;
}

// Options, factor buffers and HER state shared by every data term.  dims: I_0..I_{N-1}.
static ntf_status setup_common(Solver* S, int N, const int64_t* dims, float* const* factors, int rank,
                               const ntf_opts* opts, cudaStream_t st) {
    if (rank < 1 || rank > NTF_MAX_RANK) return fail(NTF_EINVAL, "rank must be in [1, 64]");
    if (!factors) return fail(NTF_EINVAL, "factors is NULL");
    cudaPointerAttributes pa;
    for (int l = 0; l < N; ++l) {
        if (!factors[l] || cudaPointerGetAttributes(&pa, factors[l]) != cudaSuccess ||
            (pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged)) {
            cudaGetLastError();
            return fail(NTF_EINVAL, "factors must be device memory");
        }
    }
    if (opts) S->o = *opts;
    else ntf_opts_default(&S->o);
    ntf_status s = validate_opts(S->o);
    if (s != NTF_OK) return s;
    {
        const char* e = std::getenv("NTF_PDL");
        S->pdl = !(e && e[0] == '0');
    }
    S->N = N;
    S->r = rank;
    const int r = rank;
    int64_t maxrows = 0;
    for (int l = 0; l < N; ++l) maxrows = std::max(maxrows, dims[l]);
    for (int l = 0; l < N; ++l) {
        const size_t fb = sizeof(float) * (size_t)dims[l] * r;
        for (int k = 0; k < 2; ++k) {
            if ((s = S->alloc((void**)&S->X[l][k], fb)) != NTF_OK) return s;
            NTF_CUDA_TRY(cudaMemcpyAsync(S->X[l][k], factors[l], fb, cudaMemcpyDeviceToDevice, st));  // A_hat_0 = A_0
            if ((s = S->alloc((void**)&S->GB[l][k], sizeof(double) * r * r)) != NTF_OK) return s;
        }
        S->A[l] = S->X[l][0];
        S->G[l] = S->GB[l][0];
        S->Ah[l] = S->o.her ? S->X[l][1] : S->X[l][0];
        S->Gh[l] = S->o.her ? S->GB[l][1] : S->GB[l][0];
    }
    if ((s = S->alloc((void**)&S->cur, sizeof(int) * NTF_MAX_ORDER)) != NTF_OK) return s;
    if ((s = S->alloc((void**)&S->iters_dev, 256)) != NTF_OK) return s;
    NTF_CUDA_TRY(cudaMemsetAsync(S->cur, 0, sizeof(int) * NTF_MAX_ORDER, st));
    NTF_CUDA_TRY(cudaMemsetAsync(S->iters_dev, 0, 256, st));
    if ((s = S->alloc((void**)&S->Aprev, sizeof(float) * maxrows * r)) != NTF_OK) return s;
    if ((s = S->alloc((void**)&S->M, sizeof(float) * maxrows * r)) != NTF_OK) return s;
    if ((s = S->alloc((void**)&S->V, sizeof(double) * r * r)) != NTF_OK) return s;
    if ((s = S->alloc((void**)&S->Vf, sizeof(float) * r * r)) != NTF_OK) return s;
    if ((s = S->alloc((void**)&S->scal, sizeof(double) * 8)) != NTF_OK) return s;
    if ((s = S->alloc((void**)&S->her, sizeof(ntf_her_state))) != NTF_OK) return s;
    if ((s = S->alloc(&S->ws_bcd, bcd_workspace(maxrows, r))) != NTF_OK) return s;
    if ((s = S->alloc((void**)&S->gparts, gram_parts_bytes(maxrows, r))) != NTF_OK) return s;
    if (!device_error_word()) return fail(NTF_ECUDA, "device error word unavailable");
    cudaError_t e0 = launch_objective(nullptr, nullptr, nullptr, 1, r, nullptr, nullptr, nullptr, st);
    if (e0 != cudaSuccess) return cuda_fail(e0, "configure objective kernel");
    return NTF_OK;
}

// Grams of A_0 (= A_hat_0), F-hat_0 = ||T - [[A_0]]||^2 and the HER state.  Needs scal[0] = ||T||^2.
static ntf_status finish_setup(Solver* S, cudaStream_t st) {
    const int N = S->N, r = S->r;
    for (int l = 0; l < N; ++l) {
        cudaError_t e = launch_gram(S->X[l][0], S->vu.dims[l], r, S->GB[l][0], st);
        if (e != cudaSuccess) return cuda_fail(e, "gram");
        NTF_CUDA_TRY(cudaMemcpyAsync(S->GB[l][1], S->GB[l][0], sizeof(double) * r * r, cudaMemcpyDeviceToDevice, st));
    }
    ntf_status s = S->residual(S->vs, &S->scal[3], st);
    if (s != NTF_OK) return s;
    cudaError_t e = launch_her_init(S->her, S->o.beta0, S->o.gamma, S->o.gamma_bar, S->o.eta, &S->scal[3], st);
    if (e != cudaSuccess) return cuda_fail(e, "her init");
    NTF_CUDA_TRY(cudaMemcpyAsync(&S->scal[1], &S->scal[3], sizeof(double), cudaMemcpyDeviceToDevice, st));
    return NTF_OK;
}

// Buffers of the objective by the identity (Tucker data): Grams, V and the last mode's MTTKRP at A_k.
static ntf_status alloc_identity_buffers(Solver* S) {
    const int N = S->N, r = S->r;
    ntf_status s;
    for (int l = 0; l < N; ++l)
        if ((s = S->alloc((void**)&S->Grep[l], sizeof(double) * r * r)) != NTF_OK) return s;
    if ((s = S->alloc((void**)&S->Vrep, sizeof(double) * r * r)) != NTF_OK) return s;
    return S->alloc((void**)&S->Mrep, sizeof(float) * (size_t)S->vu.dims[N - 1] * r);
}

static ntf_status create_solver(Solver** out, const ntf_tensor* T, float* const* factors, int rank,
                                const ntf_opts* opts, cudaStream_t st, void* owned_T) {
    *out = nullptr;
    Solver* S = new Solver();
    S->owned_T = owned_T;
    if (owned_T) S->allocs.push_back(owned_T);
    auto bail = [&](ntf_status s) {
        delete S;
        return s;
    };
    ntf_status s = make_view(T, &S->vu);
    if (s != NTF_OK) return bail(s);
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, S->vu.data) != cudaSuccess ||
        (pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged)) {
        cudaGetLastError();
        return bail(fail(NTF_EINVAL, "tensor data must be device memory"));
    }
    if ((s = setup_common(S, S->vu.order, S->vu.dims, factors, rank, opts, st)) != NTF_OK) return bail(s);
    const int N = S->N, r = rank;

    // streamed tensor
    S->vs = S->vu;
    if (S->o.compute_dtype == NTF_BF16 && S->vu.dtype == NTF_F32) {
        const int64_t ldb = round_up(S->vu.C, 8);
        s = S->alloc(&S->bf16_copy, sizeof(uint16_t) * (size_t)S->vu.rows() * ldb);
        if (s != NTF_OK) return bail(s);
        cudaError_t e = launch_to_bf16(static_cast<const float*>(S->vu.data), S->vu.rows(), S->vu.C, S->vu.ld,
                                       S->bf16_copy, ldb, st);
        if (e != cudaSuccess) return bail(cuda_fail(e, "bf16 cast"));
        S->vs.dtype = NTF_BF16;
        S->vs.es = 2;
        S->vs.ld = ldb;
        S->vs.data = S->bf16_copy;
    }

    int64_t maxrows = 0;
    for (int l = 0; l < N; ++l) maxrows = std::max(maxrows, S->vu.dims[l]);
    for (int n = 0; n < N; ++n) {
        if ((s = plan_mttkrp(S->vs, r, n, &S->plan[n])) != NTF_OK) return bail(s);
        if ((s = configure_mttkrp(S->vs, S->plan[n])) != NTF_OK) return bail(s);
    }
    S->fused = S->o.method == NTF_HALS && S->o.inner_max == 1 && r <= 32;
    // every mode on the tensor cores, all BF16 or all 3xTF32 (the epilogues write one layout)
    S->direct = S->fused && N == 3 && S->plan[0].tc && S->plan[1].tc && S->plan[2].tc &&
                S->plan[0].tf32 == S->plan[2].tf32;
    void* tperm = nullptr;
    size_t tperm_bytes = 0;
    {
        // The last-mode kernel reads its tiles as 32- or 128-row column blocks and is the slowest
        // of the three streams; a resident second copy of the tensor with its modes reversed
        // (I_2 x I_1 x I_0, one more numel x bytes of HBM) lets that MTTKRP run the row-stream
        // kernel instead.  Its rows contract I_0 against the pairing A_0 (A_hat_0 with HER),
        // which the mode-0 epilogue writes two kernels ahead, so this stream too can run
        // ahead of the epilogue before it (early_stream_ok).  Off with NTF_PERM_LAST=0, or when
        // the copy does not fit.
        const char* env = std::getenv("NTF_PERM_LAST");
        const bool want = !(env && env[0] == '0');
        const TensorView& v = S->vs;
        if (S->direct && want && permute_rev3_fits(v)) {
            TensorView vp = v;
            vp.dims[0] = v.dims[2];
            vp.dims[1] = v.dims[1];
            vp.dims[2] = v.dims[0];
            vp.C = v.dims[0];
            vp.ld = round_up(vp.C, 16 / v.es);
            vp.Ii = v.dims[1];
            vp.n_o = v.dims[2];
            MttkrpPlan pp;
            tperm_bytes = (size_t)vp.rows() * vp.ld * vp.es;
            if (plan_mttkrp(vp, r, 0, &pp) == NTF_OK && pp.tc && pp.tf32 == S->plan[0].tf32 &&
                pp.kind == ModeKind::Outer && configure_mttkrp(vp, pp) == NTF_OK &&
                cudaMalloc(&tperm, tperm_bytes) == cudaSuccess) {
                S->allocs.push_back(tperm);
                vp.data = tperm;
                // pp.mode stays 0: the output is mode 0 of the (I_2, I_1, I_0) layout
                S->vperm = vp;
                S->plan[2] = pp;
                S->perm = true;
            } else {
                cudaGetLastError();
            }
        }
    }
    void* t4 = nullptr;
    {
        // 4-way: merged-pair views (see Solver::direct4).  Needs unpadded rows for the merges,
        // every mode on the tensor cores in one form, and room for the second layout; off with
        // NTF_DIRECT4=0.
        const char* env = std::getenv("NTF_DIRECT4");
        const TensorView& v = S->vs;
        if (S->fused && N == 4 && !(env && env[0] == '0') && v.ld == v.dims[3] && (v.dims[1] * v.es) % 16 == 0 &&
            permute_split_fits(v, 2)) {
            auto view3 = [&](int64_t a, int64_t b, int64_t c, const void* data) {
                TensorView w = v;
                w.order = 3;
                w.dims[0] = a;
                w.dims[1] = b;
                w.dims[2] = c;
                for (int l = 3; l < NTF_MAX_ORDER; ++l) w.dims[l] = 0;
                w.C = w.ld = c;
                w.Ii = b;
                w.n_o = a;
                w.data = data;
                return w;
            };
            const int64_t I0 = v.dims[0], I1 = v.dims[1], I2 = v.dims[2], I3 = v.dims[3];
            TensorView w1 = view3(I0, I1, I2 * I3, v.data), w2 = view3(I2, I3, I0 * I1, nullptr);
            MttkrpPlan q[4];
            bool ok = plan_mttkrp(w1, r, 0, &q[0]) == NTF_OK && plan_mttkrp(w1, r, 1, &q[1]) == NTF_OK &&
                      plan_mttkrp(w2, r, 0, &q[2]) == NTF_OK && plan_mttkrp(w2, r, 1, &q[3]) == NTF_OK;
            for (int k = 0; k < 4 && ok; ++k)
                ok = q[k].tc && q[k].tf32 == q[0].tf32 && q[k].kind == (k % 2 ? ModeKind::Inner : ModeKind::Outer);
            const size_t bytes = (size_t)v.numel() * v.es;
            if (ok && configure_mttkrp(w1, q[0]) == NTF_OK && configure_mttkrp(w1, q[1]) == NTF_OK &&
                configure_mttkrp(w2, q[2]) == NTF_OK && configure_mttkrp(w2, q[3]) == NTF_OK &&
                cudaMalloc(&t4, bytes) == cudaSuccess) {
                S->allocs.push_back(t4);
                w2.data = t4;
                for (int k = 0; k < 4; ++k) S->plan[k] = q[k];
                S->vmode[0] = S->vmode[1] = w1;
                S->vmode[2] = S->vmode[3] = w2;
                S->direct4 = true;
                S->prepped = true;     // no preparation kernel on this path
            } else {
                cudaGetLastError();
            }
        }
    }
    // one workspace region per mode: a mode's epilogue still reads its partials while the
    // next mode's operands are being written
    size_t ws = 0, off_mode[NTF_MAX_ORDER];
    for (int n = 0; n < N; ++n) {
        off_mode[n] = ws;
        ws += (S->plan[n].total + 255) & ~size_t(255);
    }
    if ((s = S->alloc(&S->ws_mt, ws)) != NTF_OK) return bail(s);
    for (int n = 0; n < N; ++n) S->wsm[n] = static_cast<unsigned char*>(S->ws_mt) + off_mode[n];
    if (S->perm) {
        NTF_CUDA_TRY(cudaMemsetAsync(tperm, 0, tperm_bytes, st));
        cudaError_t e = launch_permute_rev3(S->vs, tperm, S->vperm.ld, st);
        if (e != cudaSuccess) return bail(cuda_fail(e, "reversed copy"));
        // the outer reduction of a 3-way tensor weights its single outer mode by 1
        std::vector<float> ones((size_t)S->vperm.n_o * S->plan[2].RP, 1.0f);
        NTF_CUDA_TRY(cudaMemcpy(S->wsm[2] + S->plan[2].off_W, ones.data(), sizeof(float) * ones.size(),
                                cudaMemcpyHostToDevice));
    }
    if (S->direct4) {
        // the (I_2, I_3, I_0, I_1) copy, the packed Khatri-Rao operands (zero padded) and the
        // outer reductions' unit weights
        cudaError_t e = launch_permute_split(S->vs, 2, t4, S->vs.dims[1], st);
        if (e != cudaSuccess) return bail(cuda_fail(e, "second layout"));
        for (int k = 0; k < 2; ++k) {
            const MttkrpPlan& P = S->plan[2 * k];
            const size_t b = (size_t)P.n_kc * 2 * P.RPH * 128;
            if ((s = S->alloc(&S->packKR[k], b)) != NTF_OK) return bail(s);
            NTF_CUDA_TRY(cudaMemsetAsync(S->packKR[k], 0, b, st));
            std::vector<float> ones((size_t)S->vmode[2 * k].n_o * P.RP, 1.0f);
            NTF_CUDA_TRY(cudaMemcpy(S->wsm[2 * k] + P.off_W, ones.data(), sizeof(float) * ones.size(),
                                    cudaMemcpyHostToDevice));
        }
    }
    if (S->fused) {
        const int64_t blocks = epilogue_blocks(maxrows);
        if ((s = S->alloc((void**)&S->gpart, sizeof(float) * (size_t)blocks * 2 * r * r)) != NTF_OK) return bail(s);
        if ((s = S->alloc((void**)&S->ipart, sizeof(double) * (size_t)blocks)) != NTF_OK) return bail(s);
        if ((s = S->alloc((void**)&S->qpart, sizeof(double) * (size_t)blocks)) != NTF_OK) return bail(s);
        if (S->direct) {
            // packed operands, zero outside the factor rows and columns
            const size_t rows_b = (size_t)S->plan[0].n_kc * 2 * S->plan[0].RPH * 128;
            const size_t last_b =
                S->perm ? (size_t)S->plan[2].n_kc * 2 * S->plan[2].RPH * 128
                        : (size_t)S->plan[2].nb *
                              (S->plan[2].tf32 ? (size_t)(2 * S->plan[2].RPH) * 128 : tc_last_b_bytes(S->plan[2].RPH));
            for (int k = 0; k < 2; ++k) {
                if ((s = S->alloc((void**)&S->packRows[k], rows_b)) != NTF_OK) return bail(s);
                NTF_CUDA_TRY(cudaMemsetAsync(S->packRows[k], 0, rows_b, st));
            }
            if ((s = S->alloc((void**)&S->packLast, last_b)) != NTF_OK) return bail(s);
            NTF_CUDA_TRY(cudaMemsetAsync(S->packLast, 0, last_b, st));
        }
        if (S->direct || S->direct4) {
            // every epilogue resets the counter of the stream two launches ahead; the first
            // iteration's streams start from these
            for (int n = 0; n < N; ++n)
                if (S->plan[n].tile_slots)
                    NTF_CUDA_TRY(cudaMemsetAsync(S->wsm[n] + S->plan[n].off_sched, 0, sizeof(unsigned int), st));
        }
    }
    S->ws_res_bytes = (((sizeof(float) * (size_t)S->vu.n_o * round_up(r, 4)) + 255) & ~size_t(255)) +
                      sizeof(double) * (size_t)std::max(stream_red_blocks(), 1);
    if ((s = S->alloc(&S->ws_res, S->ws_res_bytes)) != NTF_OK) return bail(s);

    // ||T||^2 of the streamed and of the given tensor
    double* parts = reinterpret_cast<double*>(static_cast<unsigned char*>(S->ws_res) +
                                              ((((sizeof(float) * (size_t)S->vu.n_o * round_up(r, 4)) + 255)) &
                                               ~size_t(255)));
    cudaError_t e = launch_norm_sq(S->vs, parts, &S->scal[0], st);
    if (e != cudaSuccess) return bail(cuda_fail(e, "norm"));
    if (S->vu.data != S->vs.data) {
        e = launch_norm_sq(S->vu, parts, &S->scal[4], st);
        if (e != cudaSuccess) return bail(cuda_fail(e, "norm"));
    } else {
        NTF_CUDA_TRY(cudaMemcpyAsync(&S->scal[4], &S->scal[0], sizeof(double), cudaMemcpyDeviceToDevice, st));
    }
    if ((s = finish_setup(S, st)) != NTF_OK) return bail(s);
    *out = S;
    return NTF_OK;
}

// Tucker-format data (Appendix A): the general iteration with every MTTKRP through the core.
static ntf_status create_solver_tucker(Solver** out, const ntf_tucker* X, float* const* factors, int rank,
                                       const ntf_opts* opts, cudaStream_t st) {
    *out = nullptr;
    Solver* S = new Solver();
    auto bail = [&](ntf_status s) {
        delete S;
        return s;
    };
    ntf_status s = make_tucker_view(X, &S->tk);
    if (s != NTF_OK) return bail(s);
    if ((s = check_device_ptr(S->tk.core.data, "Tucker core data")) != NTF_OK) return bail(s);
    for (int p = 0; p < S->tk.order; ++p)
        if ((s = check_device_ptr(S->tk.U[p], "Tucker basis U_p")) != NTF_OK) return bail(s);
    // the expanded tensor's shape (never formed)
    TensorView& v = S->vu;
    v.order = S->tk.order;
    for (int p = 0; p < v.order; ++p) v.dims[p] = S->tk.dims[p];
    v.dtype = NTF_F32;
    v.es = 4;
    v.C = v.ld = v.dims[v.order - 1];
    v.Ii = v.dims[v.order - 2];
    v.n_o = 1;
    for (int p = 0; p < v.order - 2; ++p) v.n_o *= v.dims[p];
    v.data = nullptr;
    S->vs = v;
    S->src = Solver::Src::Tucker;
    if ((s = setup_common(S, v.order, v.dims, factors, rank, opts, st)) != NTF_OK) return bail(s);
    if (S->o.compute_dtype != NTF_F32) return bail(fail(NTF_EINVAL, "Tucker data needs opts.compute_dtype = NTF_F32"));
    size_t ws = tucker_norm_workspace(S->tk);
    for (int n = 0; n < S->N; ++n) {
        if ((s = plan_tucker_mttkrp(S->tk, rank, n, &S->tkp[n])) != NTF_OK) return bail(s);
        if ((s = configure_mttkrp(S->tk.core, S->tkp[n].core)) != NTF_OK) return bail(s);
        ws = std::max(ws, S->tkp[n].total);
    }
    if ((s = S->alloc(&S->ws_tk, ws)) != NTF_OK) return bail(s);
    if ((s = alloc_identity_buffers(S)) != NTF_OK) return bail(s);
    if ((s = run_tucker_norm_sq(S->tk, &S->scal[0], S->ws_tk, st)) != NTF_OK) return bail(s);
    NTF_CUDA_TRY(cudaMemcpyAsync(&S->scal[4], &S->scal[0], sizeof(double), cudaMemcpyDeviceToDevice, st));
    if ((s = finish_setup(S, st)) != NTF_OK) return bail(s);
    *out = S;
    return NTF_OK;
}

// Tensor in host memory, streamed by slabs of mode 0 for every pass over it.
static ntf_status create_solver_streamed(Solver** out, const ntf_tensor* T_host, float* const* factors, int rank,
                                         const ntf_opts* opts, int64_t slab_rows, cudaStream_t st) {
    *out = nullptr;
    Solver* S = new Solver();
    auto bail = [&](ntf_status s) {
        delete S;
        return s;
    };
    ntf_status s = make_host_view(T_host, &S->vu);
    if (s != NTF_OK) return bail(s);
    S->vs = S->vu;
    S->src = Solver::Src::Streamed;
    if ((s = setup_common(S, S->vu.order, S->vu.dims, factors, rank, opts, st)) != NTF_OK) return bail(s);
    if (S->o.compute_dtype != NTF_F32)
        return bail(fail(NTF_EINVAL, "a streamed tensor is used in its own dtype: opts.compute_dtype = NTF_F32"));
    S->o.use_graph = 0;
    SlabLayout L;
    if ((s = slab_layout(S->vu, rank, -1, slab_rows, &L)) != NTF_OK) return bail(s);
    void* ws = nullptr;
    if ((s = S->alloc(&ws, L.total)) != NTF_OK) return bail(s);
    S->ss = new SlabStreamer();
    if ((s = S->ss->init(S->vu, rank, -1, slab_rows, ws)) != NTF_OK) return bail(s);
    if ((s = S->ss->norm_sq(&S->scal[0], st)) != NTF_OK) return bail(s);
    NTF_CUDA_TRY(cudaMemcpyAsync(&S->scal[4], &S->scal[0], sizeof(double), cudaMemcpyDeviceToDevice, st));
    if ((s = finish_setup(S, st)) != NTF_OK) return bail(s);
    *out = S;
    return NTF_OK;
}

constexpr int kMaxGraphIters = 1024;
constexpr int kGraphChunk = 32;

// Capture `iters` outer iterations into one executable graph.
static ntf_status capture_graph(Solver* S, int iters, cudaStream_t st) {
    if (S->gexec) {
        cudaGraphExecDestroy(S->gexec);
        S->gexec = nullptr;
    }
    ntf_status sp = S->ensure_prepped(st);   // before the capture: the graph holds whole iterations
    if (sp != NTF_OK) return sp;
    S->ev_used = 0;   // the graph's event records use the first timers of the pool
    S->iter_seq = 0;  // the graph's first iteration is timed (when timing is on)
    cudaGraph_t g;
    const int64_t before = ntf_launch_count();
    NTF_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    ntf_status s = NTF_OK;
    for (int k = 0; k < iters && s == NTF_OK; ++k) s = S->iterate(st);
    cudaError_t e = cudaStreamEndCapture(st, &g);
    // capturing launches nothing: the kernels are counted when the graph is replayed
    S->g_kernels = ntf_launch_count() - before;
    count_launch(-(int)S->g_kernels);
    if (s != NTF_OK) return s;
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&S->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    S->gstream = st;
    S->g_iters = iters;
    S->g_timing = S->timing_every;
    return NTF_OK;
}

static ntf_status run_solver(Solver* S, int iters, cudaStream_t st) {
    if (iters < 0) return fail(NTF_EINVAL, "iters must be >= 0");
    if (iters > 0) {
        ntf_status s = S->ensure_prepped(st);
        if (s != NTF_OK) return s;
    }
    const bool graph = S->o.use_graph && st != nullptr;
    if (!graph) {
        for (int k = 0; k < iters; ++k) {
            ntf_status s = S->iterate(st);
            if (s != NTF_OK) return s;
            ++S->iters_done;
        }
        return NTF_OK;
    }
    if (S->timing && iters > kMaxGraphIters)
        return fail(NTF_EINVAL, "timed graph runs are limited to 1024 iterations per call");
    const bool have = S->gexec && S->gstream == st && S->g_timing == S->timing_every;
    if (S->timing || (have && S->g_iters == iters)) {
        // timed runs (and a run matching a prepared graph) replay one graph of all iterations,
        // so that every timed launch belongs to the replay the events are read from
        if (!have || S->g_iters != iters) {
            ntf_status s = capture_graph(S, iters, st);
            if (s != NTF_OK) return s;
        }
        NTF_CUDA_TRY(cudaGraphLaunch(S->gexec, st));
        count_launch((int)S->g_kernels);
        S->iters_done += iters;
        return NTF_OK;
    }
    // otherwise a graph of kGraphChunk iterations is captured once and replayed; the
    // remainder runs eagerly (instantiation time grows with the graph, replay does not)
    int left = iters;
    while (left >= kGraphChunk) {
        if (!S->gexec || S->gstream != st || S->g_iters != kGraphChunk || S->g_timing != S->timing_every) {
            ntf_status s = capture_graph(S, kGraphChunk, st);
            if (s != NTF_OK) return s;
        }
        NTF_CUDA_TRY(cudaGraphLaunch(S->gexec, st));
        count_launch((int)S->g_kernels);
        left -= kGraphChunk;
        S->iters_done += kGraphChunk;
    }
    for (; left > 0; --left) {
        ntf_status s = S->iterate(st);
        if (s != NTF_OK) return s;
        ++S->iters_done;
    }
    return NTF_OK;
}

// ntf_solve*: max_iters outer iterations, or fewer when a stopping rule of opts fires.  The rules
// are tested every check_every iterations on one float64 read back to the host: the wall time
// since t0 (the paper's runs stop at a time budget, Sec. 4.1) and sqrt(F-hat_k) / ||T||_F.
static ntf_status run_until(Solver* S, cudaStream_t st, std::chrono::steady_clock::time_point t0) {
    const ntf_opts& o = S->o;
    if (!(o.max_seconds > 0.0) && !(o.rel_tol > 0.0)) return run_solver(S, o.max_iters, st);
    const int m = o.check_every > 0 ? o.check_every : 10;
    if (o.use_graph && st != nullptr && o.max_iters >= m && m <= kMaxGraphIters) {
        ntf_status s = capture_graph(S, m, st);   // replayed by run_solver for every full chunk
        if (s != NTF_OK) return s;
    }
    double h[2] = {0.0, 0.0};   // ||T_s||^2, F-hat_k
    int done = 0;
    while (done < o.max_iters) {
        const int k = std::min(m, o.max_iters - done);
        ntf_status s = run_solver(S, k, st);
        if (s != NTF_OK) return s;
        done += k;
        NTF_CUDA_TRY(cudaMemcpyAsync(h, S->scal, sizeof(h), cudaMemcpyDeviceToHost, st));
        NTF_CUDA_TRY(cudaStreamSynchronize(st));
        if (o.rel_tol > 0.0 && h[0] > 0.0 && std::sqrt(std::max(h[1], 0.0) / h[0]) <= o.rel_tol) break;
        if (o.max_seconds > 0.0 &&
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() >= o.max_seconds)
            break;
    }
    return NTF_OK;
}

static ntf_status solver_report(Solver* S, ntf_report* rep, cudaStream_t st) {
    ntf_status s = S->residual(S->vu, &S->scal[2], st);
    if (s != NTF_OK) return s;
    double h[8];
    ntf_her_state hs;
    NTF_CUDA_TRY(cudaMemcpyAsync(h, S->scal, sizeof(h), cudaMemcpyDeviceToHost, st));
    NTF_CUDA_TRY(cudaMemcpyAsync(&hs, S->her, sizeof(hs), cudaMemcpyDeviceToHost, st));
    NTF_CUDA_TRY(cudaStreamSynchronize(st));
    if (rep) {
        rep->iters = S->iters_done;
        rep->restarts = S->o.her ? hs.restarts : 0;
        rep->f_hat_last = h[1];
        rep->f_true_last = h[2];
        rep->tnorm_sq = h[4];
        rep->rel_error = h[4] > 0 ? std::sqrt(std::max(h[2], 0.0) / h[4]) : 0.0;
        rep->beta_last = S->o.her ? hs.beta : 0.0;
        rep->beta_bar_last = S->o.her ? hs.beta_bar : 0.0;
        rep->seconds = S->seconds;
    }
    if ((S->o.her && hs.numeric_error) || !std::isfinite(h[1]) || !std::isfinite(h[2]))
        return fail(NTF_ENUMERIC, "non-finite objective encountered");
    return NTF_OK;
}

// Runs a created solver to its stopping rule, copies A_k into `factors`, fills `report`
// and deletes the solver.
static ntf_status solve_and_release(Solver* S, float* const* factors, ntf_report* report, void* stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    ntf_status s = NTF_OK;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) s = cuda_fail(e, "solver set-up");
    auto t0 = std::chrono::steady_clock::now();
    if (s == NTF_OK) s = run_until(S, st, t0);
    if (s == NTF_OK) {
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) s = cuda_fail(e, "solve");
    }
    S->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    float* src[NTF_MAX_ORDER];
    if (s == NTF_OK) s = S->current_factors(st, src);
    for (int l = 0; l < S->N && s == NTF_OK; ++l) {
        e = cudaMemcpyAsync(factors[l], src[l], sizeof(float) * S->vu.dims[l] * S->r, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) s = cuda_fail(e, "copy factors");
    }
    if (s == NTF_OK) s = solver_report(S, report, st);
    delete S;
    if (s == NTF_OK) s = ntf_device_status(stream);
    return s;
}

}  // namespace ntf

using namespace ntf;

struct ntf_solver {
    Solver* s;
};

extern "C" {

ntf_status ntf_solver_create(ntf_solver** out, const ntf_tensor* T, float* const* factors, int rank,
                             const ntf_opts* opts, void* stream) {
    if (!out) return fail(NTF_EINVAL, "out is NULL");
    *out = nullptr;
    Solver* S = nullptr;
    ntf_status s = create_solver(&S, T, factors, rank, opts, static_cast<cudaStream_t>(stream), nullptr);
    if (s != NTF_OK) return s;
    *out = new ntf_solver{S};
    return NTF_OK;
}

ntf_status ntf_solver_run(ntf_solver* h, int iters, void* stream) {
    if (!h || !h->s) return fail(NTF_EINVAL, "solver is NULL");
    return run_solver(h->s, iters, static_cast<cudaStream_t>(stream));
}

ntf_status ntf_solver_get_factors(ntf_solver* h, float* const* factors, void* stream) {
    if (!h || !h->s) return fail(NTF_EINVAL, "solver is NULL");
    if (!factors) return fail(NTF_EINVAL, "factors is NULL");
    Solver* S = h->s;
    float* src[NTF_MAX_ORDER];
    ntf_status s = S->current_factors(static_cast<cudaStream_t>(stream), src);
    if (s != NTF_OK) return s;
    for (int l = 0; l < S->N; ++l) {
        if (!factors[l]) return fail(NTF_EINVAL, "factor pointer is NULL");
        NTF_CUDA_TRY(cudaMemcpyAsync(factors[l], src[l], sizeof(float) * S->vu.dims[l] * S->r,
                                     cudaMemcpyDeviceToDevice, static_cast<cudaStream_t>(stream)));
    }
    return NTF_OK;
}

ntf_status ntf_solver_report(ntf_solver* h, ntf_report* report, void* stream) {
    if (!h || !h->s) return fail(NTF_EINVAL, "solver is NULL");
    return solver_report(h->s, report, static_cast<cudaStream_t>(stream));
}

ntf_status ntf_solver_prepare_graph(ntf_solver* h, int iters, void* stream) {
    if (!h || !h->s) return fail(NTF_EINVAL, "solver is NULL");
    if (iters < 1 || iters > kMaxGraphIters) return fail(NTF_EINVAL, "iters must be in [1, 1024]");
    if (!stream) return fail(NTF_EINVAL, "graph capture needs a non-default stream");
    if (!h->s->o.use_graph) return fail(NTF_EINVAL, "the solver was created without opts.use_graph");
    return capture_graph(h->s, iters, static_cast<cudaStream_t>(stream));
}

ntf_status ntf_solver_set_timing(ntf_solver* h, int on) {
    if (!h || !h->s) return fail(NTF_EINVAL, "solver is NULL");
    h->s->timing_every = on > 0 ? on : 0;
    h->s->timing = on > 0;
    if (!h->s->gexec) h->s->ev_used = 0;
    return NTF_OK;
}

ntf_status ntf_solver_mttkrp_time(ntf_solver* h, double* total_ms, int64_t* launches, double* bytes_per_launch,
                                  void* stream) {
    if (!h || !h->s) return fail(NTF_EINVAL, "solver is NULL");
    Solver* S = h->s;
    NTF_CUDA_TRY(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    double tot = 0.0;
    for (size_t i = 0; i < S->ev_used; ++i) {
        float ms = 0.f;
        NTF_CUDA_TRY(cudaEventElapsedTime(&ms, S->ev[i].start, S->ev[i].stop));
        tot += ms;
    }
    if (total_ms) *total_ms = tot;
    if (launches) *launches = (int64_t)S->ev_used;
    if (bytes_per_launch) *bytes_per_launch = (double)S->vs.numel() * S->vs.es;
    if (!S->gexec) S->ev_used = 0;   // eager timers are reused; a graph keeps its own
    return NTF_OK;
}

void ntf_solver_destroy(ntf_solver* h) {
    if (!h) return;
    delete h->s;
    delete h;
}

ntf_status ntf_solve(const ntf_tensor* T, float* const* factors, int rank, const ntf_opts* opts, ntf_report* report,
                     void* stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Solver* S = nullptr;
    ntf_status s = create_solver(&S, T, factors, rank, opts, st, nullptr);
    if (s != NTF_OK) return s;
    return solve_and_release(S, factors, report, stream);
}

ntf_status ntf_solve_tucker(const ntf_tucker* X, float* const* factors, int rank, const ntf_opts* opts,
                            ntf_report* report, void* stream) {
    Solver* S = nullptr;
    ntf_status s = create_solver_tucker(&S, X, factors, rank, opts, static_cast<cudaStream_t>(stream));
    if (s != NTF_OK) return s;
    return solve_and_release(S, factors, report, stream);
}

ntf_status ntf_solve_streamed(const ntf_tensor* T_host, float* const* factors, int rank, const ntf_opts* opts,
                              ntf_report* report, int64_t slab_rows, void* stream) {
    Solver* S = nullptr;
    ntf_status s = create_solver_streamed(&S, T_host, factors, rank, opts, slab_rows, static_cast<cudaStream_t>(stream));
    if (s != NTF_OK) return s;
    return solve_and_release(S, factors, report, stream);
}

ntf_status ntf_solver_create_tucker(ntf_solver** out, const ntf_tucker* X, float* const* factors, int rank,
                                    const ntf_opts* opts, void* stream) {
    if (!out) return fail(NTF_EINVAL, "out is NULL");
    *out = nullptr;
    Solver* S = nullptr;
    ntf_status s = create_solver_tucker(&S, X, factors, rank, opts, static_cast<cudaStream_t>(stream));
    if (s != NTF_OK) return s;
    *out = new ntf_solver{S};
    return NTF_OK;
}

ntf_status ntf_solver_create_streamed(ntf_solver** out, const ntf_tensor* T_host, float* const* factors, int rank,
                                      const ntf_opts* opts, int64_t slab_rows, void* stream) {
    if (!out) return fail(NTF_EINVAL, "out is NULL");
    *out = nullptr;
    Solver* S = nullptr;
    ntf_status s = create_solver_streamed(&S, T_host, factors, rank, opts, slab_rows, static_cast<cudaStream_t>(stream));
    if (s != NTF_OK) return s;
    *out = new ntf_solver{S};
    return NTF_OK;
}

ntf_status ntf_solve_host(const ntf_tensor* T_host, float* const* factors_host, int rank, const ntf_opts* opts,
                          ntf_report* report, void* stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!T_host || !factors_host) return fail(NTF_EINVAL, "T_host and factors_host must not be NULL");
    if (T_host->order < 2 || T_host->order > NTF_MAX_ORDER) return fail(NTF_EINVAL, "order must be in [2, 8]");
    if (!T_host->data) return fail(NTF_EINVAL, "tensor data is NULL");
    if (rank < 1 || rank > NTF_MAX_RANK) return fail(NTF_EINVAL, "rank must be in [1, 64]");
    ntf_tensor Td = *T_host;
    const int es = T_host->dtype == NTF_F32 ? 4 : 2;
    const int64_t ld = T_host->ld ? T_host->ld : T_host->dims[T_host->order - 1];
    int64_t rows = 1;
    for (int l = 0; l < T_host->order - 1; ++l) rows *= T_host->dims[l];
    // device copy with 16-byte rows
    const int64_t ldd = round_up(T_host->dims[T_host->order - 1], 16 / es);
    void* dT = nullptr;
    cudaError_t e = cudaMalloc(&dT, (size_t)rows * ldd * es);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(NTF_ENOMEM, "cudaMalloc for the tensor failed");
    }
    // one linear copy when the host rows already have the device pitch (no padding), else a pitched copy
    if (ld == ldd)
        e = cudaMemcpyAsync(dT, T_host->data, (size_t)rows * ldd * es, cudaMemcpyHostToDevice, st);
    else
        e = cudaMemcpy2DAsync(dT, ldd * es, T_host->data, ld * es, T_host->dims[T_host->order - 1] * es, rows,
                              cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
        cudaFree(dT);
        return cuda_fail(e, "tensor upload");
    }
    Td.data = dT;
    Td.ld = ldd;
    std::vector<float*> dF(T_host->order, nullptr);
    auto cleanup = [&]() {
        for (float* p : dF) cudaFree(p);
    };
    for (int l = 0; l < T_host->order; ++l) {
        const size_t fb = sizeof(float) * (size_t)T_host->dims[l] * rank;
        if (!factors_host[l]) {
            cleanup();
            cudaFree(dT);
            return fail(NTF_EINVAL, "factor pointer is NULL");
        }
        if (cudaMalloc(&dF[l], fb) != cudaSuccess) {
            cudaGetLastError();
            cleanup();
            cudaFree(dT);
            return fail(NTF_ENOMEM, "cudaMalloc for a factor failed");
        }
        cudaMemcpyAsync(dF[l], factors_host[l], fb, cudaMemcpyHostToDevice, st);
    }
    Solver* S = nullptr;
    ntf_status s = create_solver(&S, &Td, dF.data(), rank, opts, st, dT);  // S owns dT
    if (s != NTF_OK) {
        cleanup();
        cudaFree(dT);
        return s;
    }
    auto t0 = std::chrono::steady_clock::now();
    s = run_until(S, st, t0);
    float* src[NTF_MAX_ORDER];
    if (s == NTF_OK) s = S->current_factors(st, src);
    if (s == NTF_OK) {
        for (int l = 0; l < S->N; ++l)
            cudaMemcpyAsync(factors_host[l], src[l], sizeof(float) * S->vu.dims[l] * rank, cudaMemcpyDeviceToHost, st);
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) s = cuda_fail(e, "solve");
    }
    S->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (s == NTF_OK) s = solver_report(S, report, st);
    delete S;
    cleanup();
    if (s == NTF_OK) s = ntf_device_status(stream);
    return s;
}

}  // extern "C"
