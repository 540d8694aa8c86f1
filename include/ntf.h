/*
 * ntf.h -- C ABI of libntf: block-coordinate descent with heuristic
 * extrapolation with restarts (HER) for dense nonnegative CP factorization
 * (NTF) on one NVIDIA GB300 (sm_103a).
 *
 * Method: Ang, Cohen, Gillis, Hien, "Accelerating Block Coordinate Descent for
 * Nonnegative Tensor Factorization", arXiv 2001.04321.  The problem is eq. NTF
 * (Sec. 1): minimise ||T - sum_p a_p^1 (x) ... (x) a_p^N||_F^2 over
 * nonnegative factors; the solver is Alg. 2 (HER) around the block updates
 * of Sec. 2 (HALS, Sec. 2.1.4; projected gradient, Sec. 2.2).
 *
 * Conventions shared by every entry point
 *   - Modes are 0-based: the paper's mode i is mode i-1 here.
 *   - A tensor of order N (2..8) with dims I_0..I_{N-1} is stored C-order,
 *     last mode fastest.  Rows of the last mode may be padded: element
 *     (i_0,..,i_{N-1}) sits at data[(((i_0*I_1 + i_1)*...)*ld) + i_{N-1}],
 *     with ld >= I_{N-1}.  ld*sizeof(element) must be a multiple of 16 bytes
 *     and data must be 16-byte aligned (the tensor is read with TMA).
 *   - A factor A_l is row-major I_l x rank float32 (rank contiguous), rank in
 *     [1, 64].  Grams and Hadamard products of Grams are rank x rank float64.
 *   - Objectives are ||T - X||_F^2, i.e. twice F of eq. objFun.
 *   - Unless stated otherwise every pointer is a DEVICE pointer, the caller
 *     owns every buffer, and every call is asynchronous on `stream` (a
 *     cudaStream_t passed as void*, NULL = legacy default stream).
 *   - Every call returns a status and never aborts.  On a non-OK status,
 *     ntf_last_error() gives a message (thread-local).  Invalid arguments are
 *     rejected before anything is launched.
 *   - Kernels never trap: a bounded wait that runs out records a device error
 *     word; ntf_device_status() reads (and clears) it and reports NTF_ETIMEOUT.
 */
#ifndef NTF_H_
#define NTF_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define NTF_API __attribute__((visibility("default")))
#else
#define NTF_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NTF_OK = 0,
    NTF_EINVAL = 1,    /* bad shape, rank, mode, pointer, alignment or option */
    NTF_ENOMEM = 2,    /* allocation failed (only ntf_solve* / ntf_solver_* allocate) */
    NTF_ECUDA = 3,     /* a CUDA runtime call failed; message has the CUDA error */
    NTF_ENUMERIC = 4,  /* a non-finite objective appeared; the solver stopped */
    NTF_ETIMEOUT = 5,  /* a kernel gave up a bounded wait (see ntf_device_status) */
    NTF_ENOTSUP = 6    /* valid request that this build does not support */
} ntf_status;

typedef enum { NTF_F32 = 0, NTF_BF16 = 1 } ntf_dtype;
typedef enum { NTF_HALS = 0, NTF_PGD = 1, NTF_NESTEROV = 2 } ntf_method;

#define NTF_MAX_ORDER 8
#define NTF_MAX_RANK 64

/* A dense tensor view (see conventions above).  ld = 0 means ld = dims[N-1]. */
typedef struct {
    int order;
    int64_t dims[NTF_MAX_ORDER];
    ntf_dtype dtype;
    int64_t ld;
    const void* data;
} ntf_tensor;

/* Tucker-format data (Appendix A, eq. objFunTucker): the tensor
 * (U_0 (x) ... (x) U_{N-1}) G with dims[0] x ... x dims[N-1] entries, given by
 * its core G -- an ntf_tensor of order N, NTF_F32, dims r_0 x ... x r_{N-1}
 * with every Tucker rank r_p in [1, 64], laid out like any ntf_tensor -- and
 * its bases U_p, device row-major dims[p] x r_p float32.  The expanded tensor
 * is never formed: every use goes through the core and r_p x rank products. */
typedef struct {
    ntf_tensor core;
    int64_t dims[NTF_MAX_ORDER];
    const float* U[NTF_MAX_ORDER];
} ntf_tucker;

/* Device-resident HER state (Alg. 2 and Table 3).  Allocate sizeof(ntf_her_state)
 * bytes of device memory; initialise with ntf_her_state_init. */
typedef struct {
    double beta;       /* beta_{k-1}: extrapolation weight used by the next sweep */
    double beta_bar;   /* upper bound of beta */
    double f_hat_prev; /* F-hat_{k-1} of the restart test */
    double gamma, gamma_bar, eta;
    int32_t iters;     /* decisions taken */
    int32_t restarts;  /* of which restarts */
    int32_t last_restart; /* 1 if the last decision was a restart */
    int32_t numeric_error; /* 1 if a non-finite F-hat was seen */
} ntf_her_state;

/* Solver options.  ntf_opts_default() fills the paper's defaults:
 * HER on, HALS, inner_max = 1 (plain HALS sweep per block update),
 * inner_tol = 1e-2, beta0 = 0.5, gamma = 1.05, gamma_bar = 1.01, eta = 1.5
 * (Sec. 3.1 remarks; Sec. 4.1 "Parameter set up for HER"), no time or error
 * target.  With HER on, the parameters must satisfy eq. HER:relation:
 * 0 < beta0 < 1 < gamma_bar <= gamma <= eta. */
typedef struct {
    int her;             /* 1: Alg. 2 (HER); 0: Alg. 1 (plain BCD) */
    ntf_method method;   /* block update */
    int inner_max;       /* sweeps (HALS) or steps (PGD) per block update, >= 1 */
    double inner_tol;    /* stop inner loop once ||A_s-A_{s-1}|| <= tol ||A_1-A_0|| (Sec. 4.1) */
    int max_iters;       /* outer iterations (Alg. 2 "repeat") */
    double beta0, gamma, gamma_bar, eta;
    ntf_dtype compute_dtype; /* NTF_BF16: cast T to bfloat16 once and stream that copy */
    int report_every;    /* > 0: explicit ||T - [[A_k]]||^2 every that many iterations */
    int use_graph;       /* 1: replay each outer iteration as a CUDA graph */
    /* Stopping rules of ntf_solve* besides max_iters, tested every check_every
     * iterations by reading one float64 (F-hat_k) back to the host.  The paper
     * stops its runs at a wall-time budget (Sec. 4.1, "Initialization, number
     * of runs and plots"); rel_tol stops at a target relative error instead. */
    double max_seconds;  /* > 0: stop at the first check after this much wall time */
    double rel_tol;      /* > 0: stop at the first check with sqrt(F-hat_k) / ||T||_F <= rel_tol */
    int check_every;     /* iterations between checks; <= 0 means 10 */
} ntf_opts;

/* Host-side summary of a solve. */
typedef struct {
    int iters;
    int restarts;
    double f_hat_last;   /* last F-hat_k (= ||T - X_hat||^2, restart-test surrogate) */
    double f_true_last;  /* ||T - [[A]]||^2 at return, explicit (Sec. 4.1, eq. err_true_def x 2) */
    double rel_error;    /* sqrt(f_true_last) / ||T||_F */
    double tnorm_sq;     /* ||T||^2 of the streamed (possibly bf16) tensor */
    double beta_last, beta_bar_last;
    double seconds;      /* wall time of the iterations (host clock, after a final sync) */
} ntf_report;

/* ----------------------------------------------------------------------- */
/* Library status                                                           */
/* ----------------------------------------------------------------------- */

/* Message for the last non-OK status returned on this thread ("" if none). */
NTF_API const char* ntf_last_error(void);

/* Synchronises `stream`, reads and clears the device error word.  NTF_OK or
 * NTF_ETIMEOUT (a kernel gave up a bounded wait) or NTF_ECUDA. */
NTF_API ntf_status ntf_device_status(void* stream);

/* Check of the failure path (no paper counterpart): launches one kernel whose
 * single thread waits on an mbarrier that nothing arrives on, gives up after
 * `limit_ns` nanoseconds (1e3..2e9) as every bounded wait of this library does,
 * records the time-out in the device error word and returns.  The call then
 * synchronises `stream` and returns ntf_device_status(): NTF_ETIMEOUT when the
 * path works (the word is cleared and the context stays usable). */
NTF_API ntf_status ntf_check_wait_timeout(int64_t limit_ns, void* stream);

/* Number of kernels this library has launched in this process. */
NTF_API int64_t ntf_launch_count(void);

NTF_API void ntf_opts_default(ntf_opts* opts);

/* ----------------------------------------------------------------------- */
/* Step a8: BF16 tensor storage                                             */
/* ----------------------------------------------------------------------- */

/* Row pitch (elements) that libntf uses for a bfloat16 copy of `T`:
 * dims[N-1] rounded up to a multiple of 8 (16-byte rows). */
NTF_API int64_t ntf_bf16_ld(const ntf_tensor* T);

/* dst <- bf16(T) with round-to-nearest-even, row pitch dst_ld (>= dims[N-1],
 * dst_ld*2 % 16 == 0); padding elements are written as 0.  T must be NTF_F32.
 * dst holds prod_{l<N-1} I_l * dst_ld bfloat16 values.  (BF16 storage of the
 * tensor with FP32 accumulation; not in the paper, which works in FP64.) */
NTF_API ntf_status ntf_tensor_to_bf16(const ntf_tensor* T, void* dst, int64_t dst_ld, void* stream);

/* ----------------------------------------------------------------------- */
/* Step a5 helper: ||T||_F^2                                                */
/* ----------------------------------------------------------------------- */

/* Bytes of workspace ntf_tensor_norm_sq needs (one float64 per streaming CTA). */
NTF_API size_t ntf_norm_workspace_bytes(void);

/* *out_dev <- ||T||_F^2 (float64; per-thread FP32 partial sums of at most 64
 * squares, combined in FP64 in a fixed order). */
NTF_API ntf_status ntf_tensor_norm_sq(const ntf_tensor* T, double* out_dev, void* workspace, size_t ws_bytes,
                              void* stream);

/* ----------------------------------------------------------------------- */
/* Step a1: MTTKRP                                                          */
/* ----------------------------------------------------------------------- */

/* Bytes of workspace ntf_mttkrp needs for this tensor, rank and mode. */
NTF_API size_t ntf_mttkrp_workspace_bytes(const ntf_tensor* T, int rank, int mode);

/* out (I_mode x rank, float32) <- MTTKRP of `mode`:
 *   out(j,p) = sum over entries with i_mode = j of T[i] * prod_{l != mode} A_l(i_l, p),
 * i.e. T_[n] B^n of Sec. 2 (def:B, def:grad; the N MTTKRPs per iteration that
 * dominate the run time, Sec. 4.1 footnote).  The Khatri-Rao matrix is never
 * formed: the tensor is streamed once in TMA tiles, contracted with one factor,
 * and the remaining factors enter as per-row weights.  Accumulation in FP32
 * with a fixed reduction order (bitwise reproducible).  Kernels: for rank <= 32
 * the tensor cores (BF16 tensors: bf16 MMAs against the factor split into bf16
 * hi | lo; FP32 tensors: 3xTF32, both operands split into TF32 hi | lo), else
 * FP32 FMAs.  The environment variable NTF_TF32, read once per process, selects
 * the FP32 kernels: unset or 1 = tensor cores for every mode, 2 = for the modes
 * before the last only, 0 = FMAs.
 *   factors: HOST array of `order` device pointers (factors[mode] is unused).
 *   workspace: device buffer of ws_bytes >= ntf_mttkrp_workspace_bytes(), 256-byte aligned.
 * Errors: NTF_EINVAL for bad shape/rank/mode, NULL pointers, misaligned data
 * or pitch, or a too-small workspace. */
NTF_API ntf_status ntf_mttkrp(const ntf_tensor* T, const float* const* factors, int rank, int mode, float* out,
                      void* workspace, size_t ws_bytes, void* stream);

/* Size of the fixed device scratch used by ntf_mttkrp_noalloc (per device). */
#define NTF_MTTKRP_NOALLOC_SCRATCH_BYTES (16u << 20)

/* ntf_mttkrp without a workspace argument and without any allocation.  The
 * paper has no counterpart: this entry exists for callers that cannot
 * allocate device memory -- code inside a host application that owns all
 * device memory through its own allocator, latency-critical loops where
 * cudaMalloc/cudaFree (which can block and synchronise the device) are not
 * acceptable, and processes that must not grow their device footprint per
 * call.  Same arguments, layout, result and errors as ntf_mttkrp, minus the
 * workspace.  Scratch comes from one fixed array of
 * NTF_MTTKRP_NOALLOC_SCRATCH_BYTES (16 MiB) that every GPU loading the library
 * holds until the process exits; requests needing more (see
 * ntf_mttkrp_workspace_bytes) fail with NTF_EINVAL and a message, nothing
 * launched.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls share the one array and it keeps
 * the last call's contents (nothing in it needs to start at zero): calls that
 * overlap on the GPU -- on different streams without ordering, or from
 * several host threads -- race and give wrong results, so order them. */
NTF_API ntf_status ntf_mttkrp_noalloc(const ntf_tensor* T, const float* const* factors, int rank, int mode,
                                      float* out, void* stream);

/* ----------------------------------------------------------------------- */
/* Step a2: Grams and Hadamard product of Grams                              */
/* ----------------------------------------------------------------------- */

/* G (rank x rank, float64) <- A^T A for A (rows x rank, float32).  FP32
 * products summed in FP32 over blocks of 32 rows, blocks combined in FP64.
 * Appendix A: (B^n)^T B^n is the Hadamard product of these Grams. */
NTF_API ntf_status ntf_gram(const float* A, int64_t rows, int rank, double* G, void* stream);

/* V (rank x rank, float64) <- Hadamard product of grams[l] over l != skip
 * (Appendix A).  grams: HOST array of `order` device pointers; skip may be -1. */
NTF_API ntf_status ntf_hadamard_grams(const double* const* grams, int order, int skip, int rank, double* V,
                              void* stream);

/* ----------------------------------------------------------------------- */
/* Step a3: block update (NNLS of one block, eq. NNLS / NNLS_her_exact)      */
/* ----------------------------------------------------------------------- */

/* Bytes of workspace ntf_bcd_update needs. */
NTF_API size_t ntf_bcd_workspace_bytes(int64_t rows, int rank);

/* A (rows x rank, float32, in: A_{k-1}, out: A_k) <- inexact NNLS solution of
 *   min_{A >= 0} ||A B^T - T_[n]||^2  given M = T_[n] B (the MTTKRP) and V = B^T B.
 * NTF_HALS (Sec. 2.1.4): per sweep, columns j = 0..rank-1 in order,
 *   A(:,j) <- max(0, M(:,j) - sum_{l != j} A(:,l) V(l,j)) / V(j,j)
 *   (a column with V(j,j) = 0 is left unchanged).
 * NTF_PGD (Sec. 2.2, eq. projgrad without in-block extrapolation):
 *   A <- max(0, A - (A V - M) / L),  L = lambda_max(V) (FP64 power iteration).
 * NTF_NESTEROV (Sec. 2.1, AO-Nesterov: Nesterov's accelerated gradient on the
 *   block NNLS; the paper names it without a formula, so it takes the
 *   projected gradient step of eq. projgrad and the t_k momentum sequence
 *   printed in Appendix B): with X_0 = Y_0 = A, t_0 = 1,
 *   X_s = max(0, Y_{s-1} - (Y_{s-1} V - M) / L),  t_s = (1 + sqrt(1 + 4 t_{s-1}^2)) / 2,
 *   Y_s = X_s + ((t_{s-1} - 1) / t_s) (X_s - X_{s-1});  A receives the last X_s.
 * Up to inner_max sweeps/steps; after sweep s >= 1 stop if
 * ||A_s - A_{s-1}||_F <= inner_tol ||A_1 - A_0||_F (Sec. 4.1).
 *   M: rows x rank float32; V: rank x rank float64;
 *   workspace: ws_bytes >= ntf_bcd_workspace_bytes(rows, rank). */
NTF_API ntf_status ntf_bcd_update(ntf_method method, float* A, int64_t rows, int rank, const float* M, const double* V,
                          int inner_max, double inner_tol, void* workspace, size_t ws_bytes, void* stream);

/* ----------------------------------------------------------------------- */
/* Step a9 helper: block gradient of the CP loss                             */
/* ----------------------------------------------------------------------- */

/* out (rows x rank, float32) <- s (A V - M), the gradient of (1/2)||T - X||^2
 * with respect to the factor A (Sec. 2, eq. def:grad: (A B^T - T_[n]) B with
 * B^T B = V, the Hadamard product of the other Grams (Appendix A), and
 * T_[n] B = M, the MTTKRP).  s = scale * (*scale_dev) if scale_dev is not
 * NULL (device float64, e.g. an autograd upstream gradient), else scale. */
NTF_API ntf_status ntf_block_gradient(const float* A, int64_t rows, int rank, const float* M, const double* V,
                                      const double* scale_dev, double scale, float* out, void* stream);

/* ----------------------------------------------------------------------- */
/* Step a4: HER extrapolation (Alg. 2, eq. extproj_her)                       */
/* ----------------------------------------------------------------------- */

/* A_hat <- max(0, A + beta (A - A_prev)) elementwise over n floats, with beta
 * read from device memory (*beta_dev, float64) so the call can sit in a graph. */
NTF_API ntf_status ntf_her_extrapolate(const float* A, const float* A_prev, const double* beta_dev, int64_t n,
                               float* A_hat, void* stream);

/* ----------------------------------------------------------------------- */
/* Step a5 / a7: objective                                                    */
/* ----------------------------------------------------------------------- */

/* *out_dev <- ||T||^2 - 2 <M, A> + sum_pq V(p,q) (A^T A)(p,q)   (float64)
 * = ||T - X||^2 where M, V are the MTTKRP and Hadamard-of-Grams of the block
 * A was updated against (Sec. 3.1, restart mechanism: reuse of the last
 * block's products).  M, A: rows x rank float32; V: rank x rank float64;
 * tnorm_sq_dev: device float64. */
NTF_API ntf_status ntf_objective(const double* tnorm_sq_dev, const float* M, const float* A, int64_t rows, int rank,
                         const double* V, double* out_dev, void* stream);

/* Bytes of workspace ntf_residual_sq needs. */
NTF_API size_t ntf_residual_workspace_bytes(const ntf_tensor* T, int rank);

/* *out_dev <- ||T - [[A_0..A_{N-1}]]||_F^2 computed explicitly entry by entry
 * (one pass over T; the true objective f_k of Sec. 4.1, eq. err_true_def, x2).
 * Differences are formed in FP32 and squared sums combined in FP64, so small
 * residuals do not cancel.  factors: HOST array of order device pointers. */
NTF_API ntf_status ntf_residual_sq(const ntf_tensor* T, const float* const* factors, int rank, double* out_dev,
                           void* workspace, size_t ws_bytes, void* stream);

/* ----------------------------------------------------------------------- */
/* Step a6: HER restart test and parameter update (Alg. 2, Table 3)          */
/* ----------------------------------------------------------------------- */

/* state_dev <- {beta0, beta_bar = 1, f_hat_prev = *f_hat0_dev, gamma, gamma_bar,
 * eta, counters 0}.  Requires 0 < beta0 < 1 < gamma_bar <= gamma <= eta (Alg. 2;
 * Sec. 3.1, eq. HER:relation). */
NTF_API ntf_status ntf_her_state_init(ntf_her_state* state_dev, double beta0, double gamma, double gamma_bar, double eta,
                              const double* f_hat0_dev, void* stream);

/* One decision of Alg. 2 on the device, with f_hat = *f_hat_dev (F-hat_k):
 *   F-hat_k > F-hat_{k-1}: A_hat[l] <- A[l] for all l, beta_bar <- beta, beta <- beta/eta;
 *   otherwise:             A[l] <- A_hat[l] for all l, beta_bar <- min(1, gamma_bar beta_bar),
 *                          beta <- min(beta_bar_old, gamma beta);
 * then F-hat_{k-1} <- F-hat_k.  A, A_hat: HOST arrays of `order` device
 * pointers to rows[l] x rank float32 factors; rows: HOST array. */
NTF_API ntf_status ntf_her_step(ntf_her_state* state_dev, float* const* A, float* const* A_hat, int order,
                        const int64_t* rows, int rank, const double* f_hat_dev, void* stream);

/* ----------------------------------------------------------------------- */
/* Tucker-format data (Appendix A)                                           */
/* ----------------------------------------------------------------------- */

/* Bytes of workspace ntf_tucker_mttkrp needs (0 if the arguments are invalid). */
NTF_API size_t ntf_tucker_mttkrp_workspace_bytes(const ntf_tucker* X, int rank, int mode);

/* out (dims[mode] x rank, float32) <- the MTTKRP of the Tucker-format tensor X,
 * by the gradient formula of Appendix A:
 *   out = U_mode * MTTKRP(G, {U_p^T A_p}_{p != mode}, mode),
 * which equals the MTTKRP of the expanded tensor.  Cost: the projections
 * U_p^T A_p (dims[p] x r_p x rank), one MTTKRP of the core, one expansion.
 * Projections and expansion accumulate in FP32 over 64-row chunks combined in
 * FP64 (fixed order).  factors: HOST array of `order` device pointers
 * (factors[mode] unused).  workspace: 256-byte aligned device buffer of
 * ws_bytes >= ntf_tucker_mttkrp_workspace_bytes().  Errors: NTF_EINVAL for an
 * invalid core, Tucker rank > 64, rank, mode, pointer or workspace. */
NTF_API ntf_status ntf_tucker_mttkrp(const ntf_tucker* X, const float* const* factors, int rank, int mode,
                                     float* out, void* workspace, size_t ws_bytes, void* stream);

/* Bytes of workspace ntf_tucker_norm_sq needs. */
NTF_API size_t ntf_tucker_norm_workspace_bytes(const ntf_tucker* X);

/* *out_dev (float64) <- ||(U_0 (x) ... (x) U_{N-1}) G||_F^2 without expanding:
 * <G, G x_0 Q_0 ... x_{N-1} Q_{N-1}> with Q_p = U_p^T U_p, the mode products
 * and the inner product in FP64. */
NTF_API ntf_status ntf_tucker_norm_sq(const ntf_tucker* X, double* out_dev, void* workspace, size_t ws_bytes,
                                      void* stream);

/* ----------------------------------------------------------------------- */
/* Tensor in host memory, streamed by slabs (Sec. 4, remark on data sets   */
/* too large for the implementation's memory)                               */
/* ----------------------------------------------------------------------- */

/* Bytes of device workspace ntf_mttkrp_streamed needs for slabs of slab_rows
 * mode-0 indices (slab_rows <= 0: the default, about 64 MB per slab): two
 * staging buffers, the slab MTTKRP's workspace and one I_mode x rank partial. */
NTF_API size_t ntf_mttkrp_streamed_workspace_bytes(const ntf_tensor* T_host, int rank, int mode, int64_t slab_rows);

/* ntf_mttkrp of a tensor that stays in HOST memory (T_host->data; pinned memory
 * gives full copy speed, pageable memory works but each copy is synchronous).
 * The tensor is cut into slabs of slab_rows indices of mode 0; each slab is
 * copied to the device with one cudaMemcpyAsync on a copy stream of the call,
 * double-buffered against the MTTKRP of the previous slab on `stream`.  Mode 0
 * writes its rows slab by slab; every other mode sums the slabs' partial
 * MTTKRPs in slab order (bitwise reproducible, but summed in another order than
 * ntf_mttkrp, so the two agree to FP32 rounding).  factors, out, workspace:
 * device.  The call returns once everything is queued on `stream`. */
NTF_API ntf_status ntf_mttkrp_streamed(const ntf_tensor* T_host, const float* const* factors, int rank, int mode,
                                       float* out, void* workspace, size_t ws_bytes, int64_t slab_rows, void* stream);

/* ----------------------------------------------------------------------- */
/* Whole solver: Alg. 1 (her = 0) / Alg. 2 (her = 1)                          */
/* ----------------------------------------------------------------------- */

/* Solve from the initial factors in `factors` (HOST array of order device
 * pointers, rows I_l x rank float32), overwriting them with the result.
 * opts = NULL uses ntf_opts_default() with max_iters = 100.  report (host,
 * may be NULL) receives the summary.  Allocates (and frees) its own device
 * state; synchronises `stream` before returning.  Per outer iteration:
 * for each mode n: V_n, M_n against the pairing factors A_hat (eq.
 * NNLS_her_exact), block update, extrapolation (eq. extproj_her); then
 * F-hat_k from the last block's M and V and the restart decision on the
 * device (no host round trip).  F-hat_0 = ||T - [[A_0]]||^2 explicit; the
 * previous F-hat is always replaced by the new one. */
NTF_API ntf_status ntf_solve(const ntf_tensor* T, float* const* factors, int rank, const ntf_opts* opts,
                     ntf_report* report, void* stream);

/* Same as ntf_solve but T->data and factors are HOST pointers (pinned host
 * memory gives full copy speed): copies T and the factors to the device,
 * solves, and copies the factors back, all inside the call. */
NTF_API ntf_status ntf_solve_host(const ntf_tensor* T_host, float* const* factors_host, int rank, const ntf_opts* opts,
                          ntf_report* report, void* stream);

/* ntf_solve on the Tucker-format objective F_t of Appendix A (eq.
 * objFunTucker): every MTTKRP goes through ntf_tucker_mttkrp, ||T||^2 through
 * ntf_tucker_norm_sq, and F-hat_0 and the reported f_true_last are evaluated
 * by the identity ||T||^2 - 2 <M_N, A_N> + sum(V_N (*) G(A_N)) with a fresh
 * MTTKRP (the expanded tensor is never formed).  The general 9-launch
 * iteration is used (no fused path); opts.compute_dtype must be NTF_F32. */
NTF_API ntf_status ntf_solve_tucker(const ntf_tucker* X, float* const* factors, int rank, const ntf_opts* opts,
                                    ntf_report* report, void* stream);

/* ntf_solve with the tensor in HOST memory, streamed by slabs of mode 0 as in
 * ntf_mttkrp_streamed for every MTTKRP, ||T||^2 and explicit residual.
 * factors: HOST array of device pointers.  opts.compute_dtype must be NTF_F32
 * (the host tensor's own dtype is streamed).  Allocates two staging buffers
 * and the solver state on the device. */
NTF_API ntf_status ntf_solve_streamed(const ntf_tensor* T_host, float* const* factors, int rank, const ntf_opts* opts,
                                      ntf_report* report, int64_t slab_rows, void* stream);

/* Stateful form of ntf_solve, for callers that step the solver themselves. */
typedef struct ntf_solver ntf_solver;
NTF_API ntf_status ntf_solver_create(ntf_solver** out, const ntf_tensor* T, float* const* factors, int rank,
                             const ntf_opts* opts, void* stream);
/* Stateful solver on Tucker-format data (see ntf_solve_tucker) or on a tensor
 * streamed from host memory (see ntf_solve_streamed); every other ntf_solver_*
 * call works on them as on ntf_solver_create's solver (graphs are not used
 * for the streamed form). */
NTF_API ntf_status ntf_solver_create_tucker(ntf_solver** out, const ntf_tucker* X, float* const* factors, int rank,
                                            const ntf_opts* opts, void* stream);
NTF_API ntf_status ntf_solver_create_streamed(ntf_solver** out, const ntf_tensor* T_host, float* const* factors,
                                              int rank, const ntf_opts* opts, int64_t slab_rows, void* stream);
/* Run `iters` outer iterations on `stream` (asynchronous).  With opts.use_graph
 * and a non-default stream, a CUDA graph of 32 iterations is captured once and
 * replayed (the remainder runs eagerly); a run whose length matches a graph made
 * by ntf_solver_prepare_graph, or a timed run (at most 1024 iterations), replays
 * one graph of all its iterations. */
NTF_API ntf_status ntf_solver_run(ntf_solver* s, int iters, void* stream);
/* With opts.use_graph: capture `iters` (1..1024) outer iterations into one CUDA
 * graph now, so that a later ntf_solver_run(s, iters, stream) on the same stream
 * only replays it.  With timing on, the graph records the MTTKRP events too. */
NTF_API ntf_status ntf_solver_prepare_graph(ntf_solver* s, int iters, void* stream);
/* Copy the current factors A_k into `factors` (HOST array of device pointers). */
NTF_API ntf_status ntf_solver_get_factors(ntf_solver* s, float* const* factors, void* stream);
/* Synchronise and fill `report` (f_true_last computed explicitly here). */
NTF_API ntf_status ntf_solver_report(ntf_solver* s, ntf_report* report, void* stream);
/* CUDA-event timing of the MTTKRP streaming kernels: every `every`-th outer
 * iteration (counted from the start of each captured graph, or across eager
 * runs) records an event pair around each of its streaming launches; 1 times
 * every iteration, 0 turns timing off.  ntf_solver_mttkrp_time reads the
 * totals (synchronises).  A timed launch and the kernel after it are launched
 * without programmatic dependent launch, so their times carry no overlap with
 * the neighbouring kernels. */
NTF_API ntf_status ntf_solver_set_timing(ntf_solver* s, int every);
NTF_API ntf_status ntf_solver_mttkrp_time(ntf_solver* s, double* total_ms, int64_t* launches, double* bytes_per_launch,
                                  void* stream);
NTF_API void ntf_solver_destroy(ntf_solver* s);

#ifdef __cplusplus
}
#endif

#endif /* NTF_H_ */
