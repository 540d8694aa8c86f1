/*
 * FP64 CPU oracle for block-coordinate descent with heuristic extrapolation
 * with restarts (HER) on dense nonnegative CP factorization (NTF), after
 * Ang, Cohen, Gillis, Hien, "Accelerating Block Coordinate Descent for
 * Nonnegative Tensor Factorization" (arXiv 2001.04321).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * reference that the CUDA path is checked against.  Only the tests, the smoke
 * check and the CPU-baseline leg of the benchmark load it.  It shares no code,
 * header, table or helper with the CUDA library; both receive the same seeded
 * inputs from the generator module and nothing else.
 *
 * Conventions (the paper leaves them open; the CUDA path adopts the same):
 *   - a tensor of order N with dims I_0..I_{N-1} is stored C-order (last mode
 *     fastest); modes are 0-based here (the paper's mode i is our mode i-1);
 *   - a factor A_l is row-major I_l x r (r contiguous);
 *   - the MTTKRP of mode n is M_n(j,p) = sum over all entries with i_n = j of
 *     T[i] * prod_{l != n} A_l(i_l, p), i.e. T_[n] B^n of Sec. 2 (def. of B,
 *     eq. def:grad) under the paper's reverse Khatri-Rao order;
 *   - objectives are returned as ||T - X||_F^2, i.e. 2F of eq. objFun.
 *
 * Every routine is written in plain loops, in the order of the definition or
 * algorithm it follows, with no blocking, fusion or reordering.
 *
 * Parity status per function (what pins it is in tests/test_oracle_*.py):
 *   mttkrp, mttkrp_kr, gram, hadamard_grams, objective_*, hals, pgd,
 *   nesterov, lambda_max, extrapolate, her_decide, solve (including how
 *   Alg. 2 composes its steps), tucker_expand, tucker_mttkrp,
 *   tucker_norm_sq, solve_tucker, round_bf16: pinned.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define MAXORD 8

static int64_t numel_of(int order, const int64_t* dims) {
    int64_t n = 1;
    for (int l = 0; l < order; ++l) n *= dims[l];
    return n;
}

/* Advance a C-order multi-index by one (last mode fastest). */
static void odometer_next(int order, const int64_t* dims, int64_t* idx) {
    for (int l = order - 1; l >= 0; --l) {
        if (++idx[l] < dims[l]) return;
        idx[l] = 0;
    }
}

static int check_shape(int order, const int64_t* dims, int r) {
    if (order < 2 || order > MAXORD || r < 1) return -1;
    for (int l = 0; l < order; ++l)
        if (dims[l] < 1) return -1;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* MTTKRP                                                                    */
/* ------------------------------------------------------------------------ */

/* Direct definition: one pass over every tensor entry.  Sec. 2, eq. def:grad:
 * the term T_[n] B^n, written entrywise so that no unfolding order enters. */
int oracle_mttkrp(int order, const int64_t* dims, const double* T,
                  const double* const* A, int r, int n, double* M) {
    if (check_shape(order, dims, r) || n < 0 || n >= order) return -1;
    memset(M, 0, sizeof(double) * (size_t)dims[n] * (size_t)r);
    int64_t idx[MAXORD] = {0};
    const int64_t total = numel_of(order, dims);
    for (int64_t lin = 0; lin < total; ++lin) {
        const double t = T[lin];
        for (int p = 0; p < r; ++p) {
            double prod = t;
            for (int l = 0; l < order; ++l)
                if (l != n) prod *= A[l][idx[l] * r + p];
            M[idx[n] * r + p] += prod;
        }
        odometer_next(order, dims, idx);
    }
    return 0;
}

/* Brute force with the explicit Khatri-Rao matrix and the explicit unfolding.
 * Sec. 2: B^n = A^N (kr) ... (kr) A^{n+1} (kr) A^{n-1} (kr) ... (kr) A^1
 * (def:B) and the unfolding X_[n] = A^n (kr_{l != n, l = N..1} A^l)^T
 * (eqs. unfold, lrunfold): in both, the factor of the highest mode is the most
 * significant digit of the long index.  Then M_n = T_[n] B^n.  For tiny
 * inputs only (it materialises numel/I_n x r and I_n x numel/I_n matrices). */
int oracle_mttkrp_kr(int order, const int64_t* dims, const double* T,
                     const double* const* A, int r, int n, double* M) {
    if (check_shape(order, dims, r) || n < 0 || n >= order) return -1;
    const int64_t total = numel_of(order, dims);
    const int64_t In = dims[n];
    const int64_t ncols = total / In;
    int modes[MAXORD];
    int nm = 0;
    for (int l = order - 1; l >= 0; --l)       /* N, N-1, ..., 1 without n */
        if (l != n) modes[nm++] = l;
    double* Tn = (double*)malloc(sizeof(double) * (size_t)total);
    double* B = (double*)malloc(sizeof(double) * (size_t)ncols * (size_t)r);
    if (!Tn || !B) { free(Tn); free(B); return -2; }
    /* unfolding T_[n] */
    int64_t idx[MAXORD] = {0};
    for (int64_t lin = 0; lin < total; ++lin) {
        int64_t col = 0;
        for (int m = 0; m < nm; ++m) col = col * dims[modes[m]] + idx[modes[m]];
        Tn[idx[n] * ncols + col] = T[lin];
        odometer_next(order, dims, idx);
    }
    /* Khatri-Rao product: column p is the Kronecker product of the columns p */
    for (int64_t col = 0; col < ncols; ++col) {
        int64_t sub[MAXORD];
        int64_t rem = col;
        for (int m = nm - 1; m >= 0; --m) {
            sub[m] = rem % dims[modes[m]];
            rem /= dims[modes[m]];
        }
        for (int p = 0; p < r; ++p) {
            double v = 1.0;
            for (int m = 0; m < nm; ++m) v *= A[modes[m]][sub[m] * r + p];
            B[col * r + p] = v;
        }
    }
    /* M = T_[n] B */
    for (int64_t i = 0; i < In; ++i)
        for (int p = 0; p < r; ++p) {
            double s = 0.0;
            for (int64_t c = 0; c < ncols; ++c) s += Tn[i * ncols + c] * B[c * r + p];
            M[i * r + p] = s;
        }
    free(Tn);
    free(B);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Grams                                                                     */
/* ------------------------------------------------------------------------ */

/* G = A^T A (r x r). */
int oracle_gram(const double* A, int64_t rows, int r, double* G) {
    for (int p = 0; p < r; ++p)
        for (int q = 0; q < r; ++q) {
            double s = 0.0;
            for (int64_t i = 0; i < rows; ++i) s += A[i * r + p] * A[i * r + q];
            G[p * r + q] = s;
        }
    return 0;
}

/* V = Hadamard product of the Grams G_l over l != skip:
 * (B^n)^T B^n = (*)_{l != n} A_l^T A_l (Appendix A, gradient of F_t). */
int oracle_hadamard_grams(const double* const* G, int order, int skip, int r, double* V) {
    for (int q = 0; q < r * r; ++q) V[q] = 1.0;
    for (int l = 0; l < order; ++l) {
        if (l == skip) continue;
        for (int q = 0; q < r * r; ++q) V[q] *= G[l][q];
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Objective                                                                 */
/* ------------------------------------------------------------------------ */

double oracle_norm_sq(const double* T, int64_t n) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += T[i] * T[i];
    return s;
}

/* ||T - X||_F^2 with X = sum_p (x)_l a^l_p rebuilt entry by entry
 * (eq. NTF; eq. objFun without the 1/2). */
double oracle_objective_explicit(int order, const int64_t* dims, const double* T,
                                 const double* const* A, int r) {
    int64_t idx[MAXORD] = {0};
    const int64_t total = numel_of(order, dims);
    double s = 0.0;
    for (int64_t lin = 0; lin < total; ++lin) {
        double x = 0.0;
        for (int p = 0; p < r; ++p) {
            double prod = 1.0;
            for (int l = 0; l < order; ++l) prod *= A[l][idx[l] * r + p];
            x += prod;
        }
        const double d = T[lin] - x;
        s += d * d;
        odometer_next(order, dims, idx);
    }
    return s;
}

/* Gradient of (1/2)||T - X||^2 with respect to factor `mode` (Sec. 2, eq.
 * def:grad): (A_n (B^n)^T - T_[n]) B^n = (X - T)_[n] B^n, i.e. the MTTKRP of
 * the residual tensor X - T, which is formed entrywise here. */
int oracle_cp_gradient(int order, const int64_t* dims, const double* T, const double* const* A, int r,
                       int mode, double* out) {
    if (check_shape(order, dims, r) || mode < 0 || mode >= order) return 1;
    const int64_t total = numel_of(order, dims);
    double* R = (double*)malloc(sizeof(double) * (size_t)total);
    if (!R) return 2;
    int64_t idx[MAXORD] = {0};
    for (int64_t lin = 0; lin < total; ++lin) {
        double x = 0.0;
        for (int p = 0; p < r; ++p) {
            double prod = 1.0;
            for (int l = 0; l < order; ++l) prod *= A[l][idx[l] * r + p];
            x += prod;
        }
        R[lin] = x - T[lin];
        odometer_next(order, dims, idx);
    }
    const int rc = oracle_mttkrp(order, dims, R, A, r, mode, out);
    free(R);
    return rc;
}

/* ||T - X||^2 = ||T||^2 - 2 <M_n, A_n> + sum_{pq} (V_n (*) A_n^T A_n)_{pq}:
 * the expansion that lets the restart test reuse the last block update's
 * MTTKRP and Gram product (Sec. 3.1, restart mechanism; cost I_N r^{N-1}). */
double oracle_objective_identity(double tnorm_sq, const double* M, const double* A,
                                 int64_t rows, int r, const double* V) {
    double inner = 0.0;
    for (int64_t i = 0; i < rows * r; ++i) inner += M[i] * A[i];
    double* G = (double*)malloc(sizeof(double) * (size_t)r * (size_t)r);
    if (!G) return NAN;
    oracle_gram(A, rows, r, G);
    double quad = 0.0;
    for (int q = 0; q < r * r; ++q) quad += V[q] * G[q];
    free(G);
    return tnorm_sq - 2.0 * inner + quad;
}

/* ------------------------------------------------------------------------ */
/* Block updates                                                             */
/* ------------------------------------------------------------------------ */

static double frob_diff(const double* a, const double* b, int64_t n) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        const double d = a[i] - b[i];
        s += d * d;
    }
    return sqrt(s);
}

/* Inner stopping rule of Sec. 4.1 ("Solving the NNLS problem"): stop after
 * inner_max sweeps or once ||A_s - A_{s-1}|| <= tol ||A_1 - A_0||. */
static int inner_stop(int s, double delta_s, double delta_1, int inner_max, double tol) {
    if (s >= inner_max) return 1;
    return delta_s <= tol * delta_1;
}

/* HALS (Sec. 2.1.4): cyclic exact column updates of the NNLS in block A with
 * M = T_[i] B (the MTTKRP) and V = B^T B.  Column j:
 *   A(:,j) <- max(0, M(:,j) - sum_{l != j} A(:,l) V(l,j)) / V(j,j),
 * using the columns already updated in this sweep (Gauss-Seidel).  A column
 * with V(j,j) = 0 is left unchanged.  Returns the number of sweeps done. */
int oracle_hals(double* A, int64_t rows, int r, const double* M, const double* V,
                int inner_max, double inner_tol) {
    const int64_t n = rows * r;
    double* prev = (double*)malloc(sizeof(double) * (size_t)n);
    if (!prev) return -2;
    double delta_1 = 0.0;
    int s = 0;
    for (;;) {
        ++s;
        memcpy(prev, A, sizeof(double) * (size_t)n);
        for (int j = 0; j < r; ++j) {
            const double vjj = V[j * r + j];
            if (!(vjj > 0.0)) continue;
            for (int64_t i = 0; i < rows; ++i) {
                double num = M[i * r + j];
                for (int l = 0; l < r; ++l)
                    if (l != j) num -= A[i * r + l] * V[l * r + j];
                A[i * r + j] = (num > 0.0 ? num : 0.0) / vjj;
            }
        }
        const double delta = frob_diff(A, prev, n);
        if (s == 1) delta_1 = delta;
        if (inner_stop(s, delta, delta_1, inner_max, inner_tol)) break;
    }
    free(prev);
    return s;
}

/* Largest eigenvalue of the symmetric r x r matrix V by the cyclic Jacobi
 * rotation method (textbook: annihilate each off-diagonal entry in turn until
 * the off-diagonal mass vanishes).  This is the block Lipschitz constant
 * L = ||B^T B||_2 of Sec. 2.2 for a positive semidefinite V. */
double oracle_lambda_max(const double* Vin, int r) {
    double* V = (double*)malloc(sizeof(double) * (size_t)r * (size_t)r);
    if (!V) return NAN;
    memcpy(V, Vin, sizeof(double) * (size_t)r * (size_t)r);
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, diag = 0.0;
        for (int p = 0; p < r; ++p)
            for (int q = 0; q < r; ++q) {
                if (p != q) off += V[p * r + q] * V[p * r + q];
                else diag += V[p * r + q] * V[p * r + q];
            }
        if (off <= 1e-30 * (diag > 0 ? diag : 1.0)) break;
        for (int p = 0; p < r - 1; ++p)
            for (int q = p + 1; q < r; ++q) {
                const double apq = V[p * r + q];
                if (apq == 0.0) continue;
                const double app = V[p * r + p], aqq = V[q * r + q];
                const double theta = (aqq - app) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) /
                                 (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < r; ++k) {            /* V <- V J */
                    const double vkp = V[k * r + p], vkq = V[k * r + q];
                    V[k * r + p] = c * vkp - s * vkq;
                    V[k * r + q] = s * vkp + c * vkq;
                }
                for (int k = 0; k < r; ++k) {            /* V <- J^T V */
                    const double vpk = V[p * r + k], vqk = V[q * r + k];
                    V[p * r + k] = c * vpk - s * vqk;
                    V[q * r + k] = s * vpk + c * vqk;
                }
            }
    }
    double lmax = V[0];
    for (int p = 1; p < r; ++p)
        if (V[p * r + p] > lmax) lmax = V[p * r + p];
    free(V);
    return lmax;
}

/* Projected gradient step (Sec. 2.2; Appendix B, eq. projgrad, without the
 * in-block extrapolation): A <- max(0, A - (A V - M) / L), L = lambda_max(V),
 * repeated under the same inner stopping rule as HALS.  Returns sweeps. */
int oracle_pgd(double* A, int64_t rows, int r, const double* M, const double* V,
               int inner_max, double inner_tol) {
    const int64_t n = rows * r;
    const double L = oracle_lambda_max(V, r);
    double* prev = (double*)malloc(sizeof(double) * (size_t)n);
    if (!prev) return -2;
    if (!(L > 0.0)) { free(prev); return 0; }
    double delta_1 = 0.0;
    int s = 0;
    for (;;) {
        ++s;
        memcpy(prev, A, sizeof(double) * (size_t)n);
        for (int64_t i = 0; i < rows; ++i)
            for (int j = 0; j < r; ++j) {
                double g = -M[i * r + j];
                for (int l = 0; l < r; ++l) g += prev[i * r + l] * V[l * r + j];
                const double v = prev[i * r + j] - g / L;
                A[i * r + j] = v > 0.0 ? v : 0.0;
            }
        const double delta = frob_diff(A, prev, n);
        if (s == 1) delta_1 = delta;
        if (inner_stop(s, delta, delta_1, inner_max, inner_tol)) break;
    }
    free(prev);
    return s;
}

/* ------------------------------------------------------------------------ */
/* HER pieces (Alg. 2)                                                       */
/* ------------------------------------------------------------------------ */

/* Extrapolation step, eq. extproj_her: A_hat = max(0, A + beta (A - A_prev)). */
void oracle_extrapolate(const double* A, const double* A_prev, double beta, int64_t n,
                        double* A_hat) {
    for (int64_t i = 0; i < n; ++i) {
        const double v = A[i] + beta * (A[i] - A_prev[i]);
        A_hat[i] = v > 0.0 ? v : 0.0;
    }
}

/* Restart test and parameter update of Alg. 2 (restart mechanism and
 * eqs. HER_eq:beta_update, HER_eq:beta_bar_update).  state = {beta, beta_bar,
 * f_hat_prev}.  Returns 1 on restart (f_hat > f_hat_prev), 0 on accept.  The
 * previous value is replaced by f_hat in both branches (Alg. 2 compares
 * consecutive F-hat values). */
int oracle_her_decide(double* state, double f_hat, double gamma, double gamma_bar,
                      double eta) {
    const double beta = state[0], beta_bar = state[1], prev = state[2];
    int restart;
    if (f_hat > prev) {
        state[1] = beta;
        state[0] = beta / eta;
        restart = 1;
    } else {
        state[1] = fmin(1.0, gamma_bar * beta_bar);
        state[0] = fmin(beta_bar, gamma * beta);
        restart = 0;
    }
    state[2] = f_hat;
    return restart;
}

/* AO-Nesterov block update (Sec. 2.1, "AO-Nesterov": Nesterov's accelerated
 * gradient method on the block NNLS).  The paper names the method without
 * writing it out; this follows the two ingredients it does print: the
 * projected gradient step with step 1/L of eq. projgrad (L = lambda_max(V),
 * Sec. 2.2) and the momentum sequence t_k of Appendix B (t_0 = 1,
 * t_s = (1 + sqrt(1 + 4 t_{s-1}^2)) / 2, weight (t_{s-1} - 1) / t_s).
 * With X_0 = Y_0 = A:
 *   X_s = max(0, Y_{s-1} - (Y_{s-1} V - M) / L),
 *   Y_s = X_s + w_s (X_s - X_{s-1}),   w_s = (t_{s-1} - 1) / t_s,
 * under the inner stopping rule of Sec. 4.1 applied to ||X_s - X_{s-1}||.
 * A receives the last X_s.  Returns the number of steps. */
int oracle_nesterov(double* A, int64_t rows, int r, const double* M, const double* V,
                    int inner_max, double inner_tol) {
    const int64_t n = rows * r;
    const double L = oracle_lambda_max(V, r);
    double* prev = (double*)malloc(sizeof(double) * (size_t)n);
    double* Y = (double*)malloc(sizeof(double) * (size_t)n);
    if (!prev || !Y) { free(prev); free(Y); return -2; }
    if (!(L > 0.0)) { free(prev); free(Y); return 0; }
    memcpy(Y, A, sizeof(double) * (size_t)n);               /* Y_0 = X_0 */
    double t = 1.0;                                          /* t_0 */
    double delta_1 = 0.0;
    int s = 0;
    for (;;) {
        ++s;
        memcpy(prev, A, sizeof(double) * (size_t)n);         /* X_{s-1} */
        for (int64_t i = 0; i < rows; ++i)
            for (int j = 0; j < r; ++j) {
                double g = -M[i * r + j];
                for (int l = 0; l < r; ++l) g += Y[i * r + l] * V[l * r + j];
                const double v = Y[i * r + j] - g / L;
                A[i * r + j] = v > 0.0 ? v : 0.0;            /* X_s */
            }
        const double t_next = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
        const double w = (t - 1.0) / t_next;
        t = t_next;
        for (int64_t i = 0; i < n; ++i) Y[i] = A[i] + w * (A[i] - prev[i]);
        const double delta = frob_diff(A, prev, n);
        if (s == 1) delta_1 = delta;
        if (inner_stop(s, delta, delta_1, inner_max, inner_tol)) break;
    }
    free(prev);
    free(Y);
    return s;
}

/* ------------------------------------------------------------------------ */
/* Tucker-format data (Appendix A)                                           */
/* ------------------------------------------------------------------------ */

/* The tensor (U_0 (x) ... (x) U_{N-1}) G of Appendix A written out entry by
 * entry: T[i] = sum over core entries q of G[q] prod_p U_p(i_p, q_p).  U_p is
 * row-major dims[p] x cdims[p]; G is C-order with dims cdims.  Tiny inputs. */
int oracle_tucker_expand(int order, const int64_t* dims, const int64_t* cdims, const double* G,
                         const double* const* U, double* T) {
    if (check_shape(order, dims, 1) || check_shape(order, cdims, 1)) return -1;
    const int64_t total = numel_of(order, dims);
    const int64_t ctotal = numel_of(order, cdims);
    int64_t idx[MAXORD] = {0};
    for (int64_t lin = 0; lin < total; ++lin) {
        int64_t q[MAXORD] = {0};
        double s = 0.0;
        for (int64_t c = 0; c < ctotal; ++c) {
            double prod = G[c];
            for (int p = 0; p < order; ++p) prod *= U[p][idx[p] * cdims[p] + q[p]];
            s += prod;
            odometer_next(order, cdims, q);
        }
        T[lin] = s;
        odometer_next(order, dims, idx);
    }
    return 0;
}

/* MTTKRP of the Tucker-format tensor, by the route of the gradient formula of
 * Appendix A: with W_p = U_p^T A_p (cdims[p] x r),
 *   M_n = U_n * MTTKRP(G, {W_p}_{p != n}, n),
 * which equals the MTTKRP of the expanded tensor because the unfolding of
 * (U_0 (x) ... (x) U_{N-1}) G is U_n G_[n] (Kronecker of the other U_p)^T and
 * (Kronecker of U_p)^T (Khatri-Rao of A_p) = Khatri-Rao of U_p^T A_p.  Only
 * products of the sizes of U_p, A_p and G appear. */
int oracle_tucker_mttkrp(int order, const int64_t* dims, const int64_t* cdims, const double* G,
                         const double* const* U, const double* const* A, int r, int n, double* M) {
    if (check_shape(order, dims, r) || check_shape(order, cdims, r) || n < 0 || n >= order) return -1;
    double* W[MAXORD] = {0};
    double* Y = (double*)malloc(sizeof(double) * (size_t)cdims[n] * (size_t)r);
    int rc = Y ? 0 : -2;
    for (int p = 0; p < order && rc == 0; ++p) {
        if (p == n) continue;
        W[p] = (double*)malloc(sizeof(double) * (size_t)cdims[p] * (size_t)r);
        if (!W[p]) { rc = -2; break; }
        for (int64_t q = 0; q < cdims[p]; ++q)
            for (int j = 0; j < r; ++j) {
                double s = 0.0;
                for (int64_t i = 0; i < dims[p]; ++i) s += U[p][i * cdims[p] + q] * A[p][i * r + j];
                W[p][q * r + j] = s;
            }
    }
    if (rc == 0) rc = oracle_mttkrp(order, cdims, G, (const double* const*)W, r, n, Y);
    if (rc == 0)
        for (int64_t i = 0; i < dims[n]; ++i)
            for (int j = 0; j < r; ++j) {
                double s = 0.0;
                for (int64_t q = 0; q < cdims[n]; ++q) s += U[n][i * cdims[n] + q] * Y[q * r + j];
                M[i * r + j] = s;
            }
    for (int p = 0; p < order; ++p) free(W[p]);
    free(Y);
    return rc;
}

/* ||(U_0 (x) ... (x) U_{N-1}) G||_F^2 without expanding:  <G, G x_0 Q_0 ... x_{N-1} Q_{N-1}>
 * with Q_p = U_p^T U_p (cdims[p] x cdims[p]); Z x_p Q replaces every mode-p
 * fibre z of Z by Q z. */
double oracle_tucker_norm_sq(int order, const int64_t* dims, const int64_t* cdims, const double* G,
                             const double* const* U) {
    if (check_shape(order, dims, 1) || check_shape(order, cdims, 1)) return NAN;
    const int64_t ctotal = numel_of(order, cdims);
    double* Z = (double*)malloc(sizeof(double) * (size_t)ctotal);
    double* Z2 = (double*)malloc(sizeof(double) * (size_t)ctotal);
    if (!Z || !Z2) { free(Z); free(Z2); return NAN; }
    memcpy(Z, G, sizeof(double) * (size_t)ctotal);
    for (int p = 0; p < order; ++p) {
        const int64_t rp = cdims[p];
        double* Q = (double*)malloc(sizeof(double) * (size_t)rp * (size_t)rp);
        if (!Q) { free(Z); free(Z2); return NAN; }
        for (int64_t a = 0; a < rp; ++a)
            for (int64_t b = 0; b < rp; ++b) {
                double s = 0.0;
                for (int64_t i = 0; i < dims[p]; ++i) s += U[p][i * rp + a] * U[p][i * rp + b];
                Q[a * rp + b] = s;
            }
        int64_t stride = 1;                       /* C order: stride of mode p */
        for (int l = p + 1; l < order; ++l) stride *= cdims[l];
        int64_t idx[MAXORD] = {0};
        for (int64_t lin = 0; lin < ctotal; ++lin) {
            const int64_t base = lin - idx[p] * stride;
            double s = 0.0;
            for (int64_t b = 0; b < rp; ++b) s += Q[idx[p] * rp + b] * Z[base + b * stride];
            Z2[lin] = s;
            odometer_next(order, cdims, idx);
        }
        memcpy(Z, Z2, sizeof(double) * (size_t)ctotal);
        free(Q);
    }
    double s = 0.0;
    for (int64_t c = 0; c < ctotal; ++c) s += G[c] * Z[c];
    free(Z);
    free(Z2);
    return s;
}

/* ------------------------------------------------------------------------ */
/* Solver: Alg. 1 (her = 0) and Alg. 2 (her = 1)                            */
/* ------------------------------------------------------------------------ */

/* The data term: a dense tensor T, or (Appendix A) a Tucker-format tensor
 * given by its core G (dims cdims) and factors U_p, never expanded. */
typedef struct {
    const double* T;            /* dense tensor, or the core G */
    const int64_t* cdims;       /* NULL for dense data */
    const double* const* U;     /* NULL for dense data */
} data_term;

static int data_mttkrp(const data_term* D, int order, const int64_t* dims, const double* const* A,
                       int r, int n, double* M) {
    if (!D->U) return oracle_mttkrp(order, dims, D->T, A, r, n, M);
    return oracle_tucker_mttkrp(order, dims, D->cdims, D->T, D->U, A, r, n, M);
}

/* ||T - [[A]]||^2: explicit for dense data; for Tucker data by the identity of
 * the restart mechanism with a fresh MTTKRP of the last mode (exact up to
 * rounding, pinned against explicit expansion on tiny inputs). */
static double data_objective(const data_term* D, int order, const int64_t* dims, double tnorm,
                             const double* const* A, int r) {
    if (!D->U) return oracle_objective_explicit(order, dims, D->T, A, r);
    const int last = order - 1;
    double* M = (double*)malloc(sizeof(double) * (size_t)dims[last] * (size_t)r);
    double* V = (double*)malloc(sizeof(double) * (size_t)r * (size_t)r);
    double* G[MAXORD] = {0};
    double f = NAN;
    int ok = M && V;
    for (int l = 0; l < order && ok; ++l) {
        G[l] = (double*)malloc(sizeof(double) * (size_t)r * (size_t)r);
        ok = G[l] != NULL;
        if (ok) oracle_gram(A[l], dims[l], r, G[l]);
    }
    if (ok) {
        oracle_hadamard_grams((const double* const*)G, order, last, r, V);
        if (data_mttkrp(D, order, dims, A, r, last, M) == 0)
            f = oracle_objective_identity(tnorm, M, A[last], dims[last], r, V);
    }
    for (int l = 0; l < order; ++l) free(G[l]);
    free(M);
    free(V);
    return f;
}

/* method: 0 = HALS, 1 = projected gradient, 2 = AO-Nesterov.
 * Outputs (each may be NULL), one entry per outer iteration k = 1..max_iters:
 *   out_fhat[k-1]     F-hat_k = ||T - [[A_hat^1..A_hat^{N-1}, A^N]]||^2 by the
 *                     identity from the last block's MTTKRP (Alg. 2, restart test);
 *   out_beta[k-1], out_beta_bar[k-1], out_restart[k-1]  after the decision;
 *   out_ftrue[k-1]    ||T - [[A_k]]||^2 (eq. err_true_def, times 2);
 *   out_fblock[(k-1)N + i]  ||T - X||^2 right after block i's update
 *                     (pins the monotone decrease of Alg. 1, Sec. 2.1);
 *   out_fhat0         F-hat_0 = ||T - [[A_0]]||^2;
 *   out_factors       per iteration 3 S values, S = sum_l dims[l] r: the
 *                     factors A^l_k right after the block updates, the
 *                     extrapolated A_hat^l_k before the decision, and A^l_k
 *                     after the decision, each mode after mode.
 * force (may be NULL): per iteration -1, or 0 / 1 to take the accept / restart
 * branch of Alg. 2 whatever the comparison of F-hat says (used by the tests to
 * follow a run that decided a tie the other way; the branch itself, its beta
 * updates and F-hat_{k-1} <- F-hat_k are Alg. 2's).
 * A holds the initial factors on entry and the final A_k on exit. */
static int solve_impl(const data_term* D, int order, const int64_t* dims, double* const* A, int r,
                      int her, int method, int inner_max, double inner_tol, int max_iters,
                      double beta0, double gamma, double gamma_bar, double eta,
                      double* out_fhat, double* out_beta, double* out_beta_bar, int* out_restart,
                      double* out_ftrue, double* out_fblock, double* out_fhat0, double* out_factors,
                      const int* force) {
    if (check_shape(order, dims, r) || inner_max < 1 || max_iters < 0) return -1;
    const double tnorm = D->U ? oracle_tucker_norm_sq(order, dims, D->cdims, D->T, D->U)
                              : oracle_norm_sq(D->T, numel_of(order, dims));
    double* Ahat[MAXORD];
    double* G[MAXORD];
    double* M[MAXORD];
    double* Aprev = NULL;
    double* V = (double*)malloc(sizeof(double) * (size_t)r * (size_t)r);
    int64_t maxrows = 0, S = 0;
    for (int l = 0; l < order; ++l) {
        if (dims[l] > maxrows) maxrows = dims[l];
        S += dims[l] * r;
        Ahat[l] = (double*)malloc(sizeof(double) * (size_t)dims[l] * (size_t)r);
        M[l] = (double*)malloc(sizeof(double) * (size_t)dims[l] * (size_t)r);
        G[l] = (double*)malloc(sizeof(double) * (size_t)r * (size_t)r);
        memcpy(Ahat[l], A[l], sizeof(double) * (size_t)dims[l] * (size_t)r); /* A_hat_0 = A_0 */
    }
    Aprev = (double*)malloc(sizeof(double) * (size_t)maxrows * (size_t)r);

    double state[3];
    state[0] = beta0;   /* beta_0 */
    state[1] = 1.0;     /* beta_bar_0 = 1 */
    state[2] = data_objective(D, order, dims, tnorm, (const double* const*)A, r);
    if (out_fhat0) *out_fhat0 = state[2];

    for (int k = 1; k <= max_iters; ++k) {
        const double beta = state[0];
        for (int i = 0; i < order; ++i) {
            const int64_t n = dims[i] * r;
            /* the other blocks enter at their pairing values A_hat (eq.
             * NNLS_her_exact); without HER, A_hat == A and this is Alg. 1 */
            for (int l = 0; l < order; ++l)
                if (l != i) oracle_gram(Ahat[l], dims[l], r, G[l]);
            oracle_hadamard_grams((const double* const*)G, order, i, r, V);
            data_mttkrp(D, order, dims, (const double* const*)Ahat, r, i, M[i]);
            memcpy(Aprev, A[i], sizeof(double) * (size_t)n);          /* A_{k-1}^i */
            if (method == 0) oracle_hals(A[i], dims[i], r, M[i], V, inner_max, inner_tol);
            else if (method == 1) oracle_pgd(A[i], dims[i], r, M[i], V, inner_max, inner_tol);
            else oracle_nesterov(A[i], dims[i], r, M[i], V, inner_max, inner_tol);
            if (her) oracle_extrapolate(A[i], Aprev, beta, n, Ahat[i]);
            else memcpy(Ahat[i], A[i], sizeof(double) * (size_t)n);
            if (out_fblock)
                out_fblock[(int64_t)(k - 1) * order + i] =
                    data_objective(D, order, dims, tnorm, (const double* const*)A, r);
        }
        if (out_factors) {
            double* o = out_factors + (int64_t)(k - 1) * 3 * S;
            for (int l = 0; l < order; ++l) {
                memcpy(o, A[l], sizeof(double) * (size_t)dims[l] * (size_t)r);
                memcpy(o + S, Ahat[l], sizeof(double) * (size_t)dims[l] * (size_t)r);
                o += dims[l] * r;
            }
        }
        /* F-hat_k = F(A_hat^1..A_hat^{N-1}, A^N): M and V of the last block
         * were formed against exactly those A_hat (Alg. 2, restart test). */
        const int last = order - 1;
        const double fhat = oracle_objective_identity(tnorm, M[last], A[last], dims[last], r, V);
        int restart = 0;
        if (her) {
            const int f = force ? force[k - 1] : -1;
            /* a forced branch compares an infinite F-hat, then records the real one */
            restart = oracle_her_decide(state, f < 0 ? fhat : (f ? INFINITY : -INFINITY), gamma, gamma_bar, eta);
            state[2] = fhat;
            for (int l = 0; l < order; ++l) {
                const size_t bytes = sizeof(double) * (size_t)dims[l] * (size_t)r;
                if (restart) memcpy(Ahat[l], A[l], bytes);   /* abandon A_hat */
                else memcpy(A[l], Ahat[l], bytes);           /* keep A_hat */
            }
        } else {
            state[2] = fhat;
        }
        if (out_factors) {
            double* o = out_factors + (int64_t)(k - 1) * 3 * S + 2 * S;
            for (int l = 0; l < order; ++l) {
                memcpy(o, A[l], sizeof(double) * (size_t)dims[l] * (size_t)r);
                o += dims[l] * r;
            }
        }
        if (out_fhat) out_fhat[k - 1] = fhat;
        if (out_beta) out_beta[k - 1] = state[0];
        if (out_beta_bar) out_beta_bar[k - 1] = state[1];
        if (out_restart) out_restart[k - 1] = restart;
        if (out_ftrue)
            out_ftrue[k - 1] = data_objective(D, order, dims, tnorm, (const double* const*)A, r);
    }
    for (int l = 0; l < order; ++l) { free(Ahat[l]); free(M[l]); free(G[l]); }
    free(Aprev);
    free(V);
    return 0;
}

/* Alg. 1 / Alg. 2 on a dense tensor T (see solve_impl for the outputs). */
int oracle_solve(int order, const int64_t* dims, const double* T, double* const* A, int r,
                 int her, int method, int inner_max, double inner_tol, int max_iters,
                 double beta0, double gamma, double gamma_bar, double eta,
                 double* out_fhat, double* out_beta, double* out_beta_bar, int* out_restart,
                 double* out_ftrue, double* out_fblock, double* out_fhat0, double* out_factors,
                 const int* force) {
    const data_term D = {T, NULL, NULL};
    return solve_impl(&D, order, dims, A, r, her, method, inner_max, inner_tol, max_iters, beta0, gamma,
                      gamma_bar, eta, out_fhat, out_beta, out_beta_bar, out_restart, out_ftrue, out_fblock,
                      out_fhat0, out_factors, force);
}

/* Alg. 1 / Alg. 2 on the Tucker-format objective F_t of Appendix A (eq.
 * objFunTucker): the data tensor is (U_0 (x) ... (x) U_{N-1}) G, entering only
 * through oracle_tucker_mttkrp and oracle_tucker_norm_sq. */
int oracle_solve_tucker(int order, const int64_t* dims, const int64_t* cdims, const double* G,
                        const double* const* U, double* const* A, int r,
                        int her, int method, int inner_max, double inner_tol, int max_iters,
                        double beta0, double gamma, double gamma_bar, double eta,
                        double* out_fhat, double* out_beta, double* out_beta_bar, int* out_restart,
                        double* out_ftrue, double* out_fblock, double* out_fhat0, double* out_factors,
                        const int* force) {
    if (!cdims || !U || check_shape(order, cdims, 1)) return -1;
    const data_term D = {G, cdims, U};
    return solve_impl(&D, order, dims, A, r, her, method, inner_max, inner_tol, max_iters, beta0, gamma,
                      gamma_bar, eta, out_fhat, out_beta, out_beta_bar, out_restart, out_ftrue, out_fblock,
                      out_fhat0, out_factors, force);
}

/* ------------------------------------------------------------------------ */
/* BF16 storage                                                              */
/* ------------------------------------------------------------------------ */

/* FP32 -> bfloat16 with round-to-nearest, ties to even (IEEE 754 rounding of
 * the 24-bit significand to 8 bits); NaN stays NaN. */
void oracle_round_bf16(const float* in, uint16_t* out, int64_t n) {
    for (int64_t i = 0; i < n; ++i) {
        uint32_t u;
        memcpy(&u, &in[i], 4);
        if ((u & 0x7f800000u) == 0x7f800000u && (u & 0x007fffffu)) {
            out[i] = (uint16_t)((u >> 16) | 0x0040u);
            continue;
        }
        const uint32_t lsb = (u >> 16) & 1u;
        u += 0x7fffu + lsb;
        out[i] = (uint16_t)(u >> 16);
    }
}
