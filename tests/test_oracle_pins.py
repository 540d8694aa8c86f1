"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test names the passage of arXiv 2001.04321 it pins and the independent
source of truth: a library routine (numpy einsum / eigvalsh, scipy nnls, torch's
bfloat16 cast), a closed form, a brute-force enumeration, a finite-difference
gradient, an invariant of the algorithm, or a hand-worked table in
``tests/golden/``.  All run on the CPU in a few seconds.
"""
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rand_problem(dims, r, seed):
    rng = np.random.default_rng(seed)
    T = rng.random(dims)
    F = [rng.random((d, r)) for d in dims]
    return T, F


def einsum_mttkrp(T, F, n):
    """Library route: numpy.einsum over the full contraction (independent of the oracle)."""
    N = T.ndim
    letters = "abcdefgh"[:N]
    spec = letters + "," + ",".join(letters[l] + "z" for l in range(N) if l != n) + "->" + letters[n] + "z"
    return np.einsum(spec, T, *[F[l] for l in range(N) if l != n])


def einsum_full(F):
    N = len(F)
    letters = "abcdefgh"[:N]
    spec = ",".join(letters[l] + "z" for l in range(N)) + "->" + letters
    return np.einsum(spec, *F)


# --- MTTKRP (Sec. 2, def:B, def:grad, unfold/lrunfold) -----------------------

@pytest.mark.parametrize("dims,r", [((5, 4, 3), 3), ((3, 4, 2, 3), 2), ((6, 5), 4), ((2, 3, 2, 2, 3), 2)])
def test_mttkrp_three_routes_agree(dims, r):
    T, F = rand_problem(dims, r, 1)
    for n in range(len(dims)):
        M_def = oracle.mttkrp(T, F, n)
        M_kr = oracle.mttkrp_kr(T, F, n)
        M_lib = einsum_mttkrp(T, F, n)
        np.testing.assert_allclose(M_def, M_lib, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(M_kr, M_lib, rtol=1e-12, atol=1e-12)


def test_mttkrp_rank1_closed_form():
    # T = a (x) b (x) c and rank-1 factors (x, y, z): M_0 = a (b.y)(c.z), etc.
    rng = np.random.default_rng(3)
    a, b, c = rng.random(4), rng.random(5), rng.random(6)
    x, y, z = rng.random(4), rng.random(5), rng.random(6)
    T = a[:, None, None] * b[None, :, None] * c[None, None, :]
    F = [x[:, None], y[:, None], z[:, None]]
    np.testing.assert_allclose(oracle.mttkrp(T, F, 0)[:, 0], a * (b @ y) * (c @ z), rtol=1e-13)
    np.testing.assert_allclose(oracle.mttkrp(T, F, 1)[:, 0], b * (a @ x) * (c @ z), rtol=1e-13)
    np.testing.assert_allclose(oracle.mttkrp(T, F, 2)[:, 0], c * (a @ x) * (b @ y), rtol=1e-13)


def test_mttkrp_kr_order_matters():
    # A transposed Khatri-Rao order would still pass on cubes; non-cubic dims and
    # distinct factors expose it: the KR route must match the library exactly.
    T, F = rand_problem((2, 5, 3), 2, 9)
    np.testing.assert_allclose(oracle.mttkrp_kr(T, F, 1), einsum_mttkrp(T, F, 1), rtol=1e-13)


# --- Grams and the Hadamard-of-Grams identity (Appendix A) --------------------

def test_gram_and_hadamard_equal_explicit_kr_gram():
    dims, r = (4, 3, 5), 3
    _, F = rand_problem(dims, r, 4)
    G = [oracle.gram(A) for A in F]
    for A, g in zip(F, G):
        np.testing.assert_allclose(g, A.T @ A, rtol=1e-13)
    for n in range(3):
        others = [F[l] for l in range(3) if l != n]
        B = np.einsum("iz,jz->ijz", *others).reshape(-1, r)   # any row order: B^T B is order-free
        np.testing.assert_allclose(oracle.hadamard_grams(G, n), B.T @ B, rtol=1e-12)


# --- Objective (eq. objFun; restart-test expansion, Sec. 3.1) -----------------

@pytest.mark.parametrize("dims,r", [((5, 4, 3), 3), ((3, 4, 2, 3), 2), ((7, 6), 3)])
def test_objective_explicit_and_identity(dims, r):
    T, F = rand_problem(dims, r, 5)
    X = einsum_full(F)
    ref = float(np.sum((T - X) ** 2))
    assert oracle.objective_explicit(T, F) == pytest.approx(ref, rel=1e-12)
    N = len(dims)
    G = [oracle.gram(A) for A in F]
    tn = oracle.norm_sq(T)
    assert tn == pytest.approx(float(np.sum(T * T)), rel=1e-13)
    for n in range(N):
        M = oracle.mttkrp(T, F, n)
        V = oracle.hadamard_grams(G, n)
        assert oracle.objective_identity(tn, M, F[n], V) == pytest.approx(ref, rel=1e-10, abs=1e-10)


def test_gradient_identity_finite_difference():
    # grad_{A_n} (1/2)||T - X||^2 = A_n V_n - M_n (eq. def:grad with Appendix A's V);
    # checked against central differences of the explicit objective.
    T, F = rand_problem((4, 3, 5), 2, 6)
    G = [oracle.gram(A) for A in F]
    h = 1e-6
    for n in range(3):
        grad = F[n] @ oracle.hadamard_grams(G, n) - oracle.mttkrp(T, F, n)
        fd = np.zeros_like(F[n])
        for i in range(F[n].shape[0]):
            for p in range(F[n].shape[1]):
                Fp = [A.copy() for A in F]
                Fm = [A.copy() for A in F]
                Fp[n][i, p] += h
                Fm[n][i, p] -= h
                fd[i, p] = (0.5 * oracle.objective_explicit(T, Fp) - 0.5 * oracle.objective_explicit(T, Fm)) / (2 * h)
        np.testing.assert_allclose(grad, fd, rtol=1e-6, atol=1e-7)


def test_cp_gradient_matches_finite_differences_and_vanishes_at_exact_fit():
    # oracle.cp_gradient forms X - T explicitly and applies the MTTKRP; central
    # differences of the explicit objective pin it, and at an exact
    # factorization (T = [[F]]) the gradient is zero.
    T, F = rand_problem((3, 4, 2, 3), 2, 8)
    h = 1e-6
    for n in range(4):
        g = oracle.cp_gradient(T, F, n)
        fd = np.zeros_like(F[n])
        for i in range(F[n].shape[0]):
            for p in range(F[n].shape[1]):
                Fp = [A.copy() for A in F]
                Fm = [A.copy() for A in F]
                Fp[n][i, p] += h
                Fm[n][i, p] -= h
                fd[i, p] = (0.5 * oracle.objective_explicit(T, Fp) - 0.5 * oracle.objective_explicit(T, Fm)) / (2 * h)
        np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-7)
    X = np.einsum("iz,jz,kz,lz->ijkl", *F)
    for n in range(4):
        assert np.abs(oracle.cp_gradient(X, F, n)).max() <= 1e-12


# --- HALS (Sec. 2.1.4) --------------------------------------------------------

def _block_problem(seed, I=6, r=3, dims_other=(5, 4)):
    rng = np.random.default_rng(seed)
    others = [rng.random((d, r)) for d in dims_other]
    B = np.einsum("iz,jz->ijz", *others).reshape(-1, r)
    Tn = rng.random((I, B.shape[0]))
    return Tn @ B, B.T @ B, B, Tn


def test_hals_converges_to_scipy_nnls():
    scipy_opt = pytest.importorskip("scipy.optimize")
    M, V, B, Tn = _block_problem(7)
    A0 = np.random.default_rng(8).random((M.shape[0], V.shape[0]))
    A, sweeps = oracle.hals(A0, M, V, inner_max=5000, inner_tol=0.0)
    for i in range(M.shape[0]):
        x, _ = scipy_opt.nnls(B, Tn[i])
        np.testing.assert_allclose(A[i], x, rtol=1e-7, atol=1e-9)


def test_hals_last_column_is_exact_1d_minimiser():
    # after a sweep the last column solves its 1-D NNLS exactly: KKT conditions
    M, V, _, _ = _block_problem(9)
    A0 = np.random.default_rng(10).random((M.shape[0], V.shape[0]))
    A, _ = oracle.hals(A0, M, V, inner_max=1)
    j = V.shape[0] - 1
    g = (A @ V - M)[:, j]
    pos = A[:, j] > 0
    np.testing.assert_allclose(g[pos], 0.0, atol=1e-10)
    assert np.all(g[~pos] >= -1e-12)


def test_hals_one_sweep_decreases_block_objective():
    M, V, B, Tn = _block_problem(11)
    A0 = np.random.default_rng(12).random((M.shape[0], V.shape[0]))
    A, _ = oracle.hals(A0, M, V, inner_max=1)
    f = lambda A: np.sum((A @ B.T - Tn) ** 2)
    assert f(A) <= f(A0) + 1e-12
    assert np.all(A >= 0)


def test_hals_zero_diagonal_column_left_unchanged():
    M, V, _, _ = _block_problem(13)
    V = V.copy()
    V[1, :] = 0.0
    V[:, 1] = 0.0
    A0 = np.random.default_rng(14).random((M.shape[0], V.shape[0]))
    A, _ = oracle.hals(A0, M, V, inner_max=1)
    np.testing.assert_array_equal(A[:, 1], A0[:, 1])


def test_hals_stop_rule_counts_sweeps():
    M, V, _, _ = _block_problem(15)
    A0 = np.random.default_rng(16).random((M.shape[0], V.shape[0]))
    _, s1 = oracle.hals(A0, M, V, inner_max=1)
    _, s50 = oracle.hals(A0, M, V, inner_max=50, inner_tol=1e-2)
    _, s_all = oracle.hals(A0, M, V, inner_max=7, inner_tol=0.0)
    assert s1 == 1 and 1 < s50 <= 50 and s_all == 7


# --- PGD (Sec. 2.2, eq. projgrad) ---------------------------------------------

def test_lambda_max_matches_eigvalsh():
    rng = np.random.default_rng(17)
    for r in (1, 2, 5, 20, 33):
        X = rng.random((40, r))
        V = X.T @ X
        assert oracle.lambda_max(V) == pytest.approx(float(np.linalg.eigvalsh(V)[-1]), rel=1e-12)


def test_pgd_converges_to_scipy_nnls_and_descends():
    scipy_opt = pytest.importorskip("scipy.optimize")
    M, V, B, Tn = _block_problem(18)
    A0 = np.random.default_rng(19).random((M.shape[0], V.shape[0]))
    f = lambda A: np.sum((A @ B.T - Tn) ** 2)
    A1, _ = oracle.pgd(A0, M, V, inner_max=1)
    assert f(A1) <= f(A0) + 1e-12
    A, _ = oracle.pgd(A0, M, V, inner_max=200000, inner_tol=0.0)
    for i in range(M.shape[0]):
        x, _ = scipy_opt.nnls(B, Tn[i])
        np.testing.assert_allclose(A[i], x, rtol=1e-5, atol=1e-7)


# --- HER extrapolation and decision (Alg. 2) ----------------------------------

def test_extrapolate_worked_values():
    A = np.array([1.0, 2.0, 0.0, 3.0])
    P = np.array([2.0, 1.0, 1.0, 3.0])
    # 1 + .5(1-2) = .5 ; 2 + .5(2-1) = 2.5 ; 0 + .5(0-1) = -.5 -> 0 ; 3 + 0 = 3
    np.testing.assert_array_equal(oracle.extrapolate(A, P, 0.5), [0.5, 2.5, 0.0, 3.0])
    np.testing.assert_array_equal(oracle.extrapolate(A, P, 0.0), A)


def _read_table(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_her_decide_golden_table():
    state = [0.5, 1.0, 10.0]
    f = 10.0
    for step, d, beta, beta_bar in _read_table("her_beta_table.txt"):
        f = f - 1.0 if d == "a" else f + 1.0
        restart = oracle.her_decide(state, f)
        assert restart == (d == "r")
        assert state[0] == pytest.approx(float(beta), rel=1e-14)
        assert state[1] == pytest.approx(float(beta_bar), rel=1e-14)
        assert state[2] == f


def test_her_tie_accepts():
    state = [0.5, 1.0, 3.0]
    assert oracle.her_decide(state, 3.0) == 0


# --- Whole solver (Alg. 1 / Alg. 2) -------------------------------------------

def test_plain_hals_monotone_per_block_update():
    # Alg. 1: the objective does not increase after any block update (Sec. 2.1)
    T, _ = synth.make_tensor((8, 7, 6), 3, 1e-2, seed=21, dtype=np.float64)
    init = synth.make_init((8, 7, 6), 3, seed=1)
    _, tr = oracle.solve(T, init, 15, her=False, track_blocks=True)
    f = np.concatenate([[tr.fhat0[0]], tr.fblock])
    assert np.all(np.diff(f) <= 1e-12 * oracle.norm_sq(T))


def test_plain_fhat_equals_true_objective():
    # without extrapolation A_hat == A, so F-hat (identity) must equal explicit F
    T, _ = synth.make_tensor((6, 5, 7), 2, 1e-2, seed=22, dtype=np.float64)
    init = synth.make_init((6, 5, 7), 2, seed=2)
    _, tr = oracle.solve(T, init, 8, her=False, track_true=True)
    np.testing.assert_allclose(tr.fhat, tr.ftrue, rtol=1e-9)


def test_her_invariants_and_restart_rule():
    T, _ = synth.make_tensor((10, 9, 8), 3, 1e-2, seed=23, dtype=np.float64)
    init = synth.make_init((10, 9, 8), 3, seed=3)
    F, tr = oracle.solve(T, init, 40, her=True, track_true=True)
    assert np.all(tr.beta > 0) and np.all(tr.beta <= tr.beta_bar + 1e-15) and np.all(tr.beta_bar <= 1.0)
    prev = np.concatenate([[tr.fhat0[0]], tr.fhat[:-1]])
    np.testing.assert_array_equal(tr.restart, (tr.fhat > prev).astype(np.int32))
    for A in F:
        assert np.all(A >= 0)
    assert tr.restart.sum() >= 1   # this seed restarts at least once (exercise both branches)


def test_noiseless_exact_recovery():
    # noiseless low-rank tensors can be fitted exactly (Sec. 4.1: f_min = 0)
    dims, r = (12, 11, 10), 3
    ok = 0
    for run in range(3):
        T, _ = synth.make_tensor(dims, r, 0.0, seed=31 + run, dtype=np.float64)
        init = synth.make_init(dims, r, seed=run)
        _, tr = oracle.solve(T, init, 400, her=True, track_true=True)
        rel = np.sqrt(tr.ftrue[-1] / oracle.norm_sq(T))
        ok += rel < 1e-6
    assert ok >= 2


def test_her_beats_plain_on_illconditioned():
    # the paper's central empirical claim (Sec. 4): same iteration count, lower error
    dims, r = (20, 20, 20), 4
    T, _ = synth.make_tensor(dims, r, 1e-3, seed=41, recipe="illcond", dtype=np.float64)
    init = synth.make_init(dims, r, seed=4)
    _, plain = oracle.solve(T, init, 150, her=False, track_true=True)
    _, her = oracle.solve(T, init, 150, her=True, track_true=True)
    assert her.ftrue[-1] < plain.ftrue[-1]


def test_pgd_solver_runs_and_descends_first_step():
    T, _ = synth.make_tensor((6, 6, 6), 2, 1e-2, seed=42, dtype=np.float64)
    init = synth.make_init((6, 6, 6), 2, seed=5)
    _, tr = oracle.solve(T, init, 5, her=False, method="pgd", inner_max=3, track_blocks=True)
    f = np.concatenate([[tr.fhat0[0]], tr.fblock])
    assert np.all(np.diff(f) <= 1e-12 * oracle.norm_sq(T))


# --- BF16 storage rounding ----------------------------------------------------

def test_round_bf16_matches_torch_rne():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(50)
    x = np.concatenate([rng.standard_normal(10000).astype(np.float32) * 100,
                        np.array([1.0, 1.00390625, 1.01171875, 0.0, -0.0, 3.4e38, 1e-40], dtype=np.float32)])
    ours = oracle.round_bf16(x)
    ref = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    np.testing.assert_array_equal(ours, ref)
    # a tie rounds to even: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7
    assert oracle.bf16_to_f64(oracle.round_bf16(np.float32(1.00390625))) == 1.0


def test_golden_defaults_file():
    vals = {k: float(v) for k, v in _read_table("her_defaults.txt")}
    assert vals["beta0"] == 0.5 and vals["gamma"] == 1.05 and vals["gamma_bar"] == 1.01 and vals["eta"] == 1.5
    # the relation 0 < beta <= beta_bar <= 1 < gamma_bar <= gamma <= eta (Sec. 3.1, eq. HER:relation)
    assert 0 < vals["beta0"] <= vals["beta_bar0"] <= 1 < vals["gamma_bar"] <= vals["gamma"] <= vals["eta"]
