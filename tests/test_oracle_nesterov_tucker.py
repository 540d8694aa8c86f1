"""Pins of the oracle's AO-Nesterov block update (Sec. 2.1 AO-Nesterov with
the momentum sequence of Appendix B) and of its Tucker-format data term
(Appendix A), against facts that do not come from the oracle itself."""
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _block_problem(seed, I=6, r=3, dims_other=(5, 4)):
    rng = np.random.default_rng(seed)
    others = [rng.random((d, r)) for d in dims_other]
    B = np.einsum("iz,jz->ijz", *others).reshape(-1, r)
    Tn = rng.random((I, B.shape[0]))
    return Tn @ B, B.T @ B, B, Tn


# --- AO-Nesterov --------------------------------------------------------------

def test_nesterov_converges_to_scipy_nnls():
    scipy_opt = pytest.importorskip("scipy.optimize")
    M, V, B, Tn = _block_problem(61)
    A0 = np.random.default_rng(62).random((M.shape[0], V.shape[0]))
    A, steps = oracle.nesterov(A0, M, V, inner_max=20000, inner_tol=0.0)
    assert steps == 20000
    for i in range(M.shape[0]):
        x, _ = scipy_opt.nnls(B, Tn[i])
        np.testing.assert_allclose(A[i], x, rtol=1e-7, atol=1e-9)


def test_nesterov_first_step_is_projected_gradient_step():
    # t_0 = 1 gives zero momentum before the first step: one step of AO-Nesterov
    # is one projected gradient step of eq. projgrad (pinned against scipy nnls)
    M, V, _, _ = _block_problem(63)
    A0 = np.random.default_rng(64).random((M.shape[0], V.shape[0]))
    A1, s1 = oracle.nesterov(A0, M, V, inner_max=1)
    P1, _ = oracle.pgd(A0, M, V, inner_max=1)
    assert s1 == 1
    np.testing.assert_array_equal(A1, P1)


def test_nesterov_momentum_golden_table():
    rows = []
    with open(os.path.join(GOLDEN, "nesterov_momentum_table.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    V = np.diag([1.0, 0.25])
    M = np.array([[1.0, 1.0], [1.0, -1.0]])
    A0 = np.zeros((2, 2))
    for s, _t, _w, x in rows:
        A, steps = oracle.nesterov(A0, M, V, inner_max=int(s), inner_tol=0.0)
        assert steps == int(s)
        assert A[0, 0] == pytest.approx(1.0, rel=1e-15)
        assert A[0, 1] == pytest.approx(x, rel=1e-12)
        assert A[1, 0] == pytest.approx(1.0, rel=1e-15) and A[1, 1] == 0.0


def test_nesterov_descends_faster_than_pgd_on_illconditioned_block():
    # the point of the momentum: on an ill-conditioned block it reaches a lower block
    # objective than plain projected gradient in the same number of steps
    rng = np.random.default_rng(65)
    base = rng.random((40, 1))
    B = base + 0.05 * rng.random((40, 4))
    Tn = rng.random((5, 40))
    M, V = Tn @ B, B.T @ B
    A0 = rng.random((5, 4))
    f = lambda A: np.sum((A @ B.T - Tn) ** 2)
    An, _ = oracle.nesterov(A0, M, V, inner_max=50, inner_tol=0.0)
    Ap, _ = oracle.pgd(A0, M, V, inner_max=50, inner_tol=0.0)
    assert f(An) < f(Ap)


def test_nesterov_stop_rule_and_solver_descent():
    M, V, _, _ = _block_problem(66)
    A0 = np.random.default_rng(67).random((M.shape[0], V.shape[0]))
    _, s50 = oracle.nesterov(A0, M, V, inner_max=50, inner_tol=1e-2)
    assert 1 < s50 <= 50
    # Alg. 1 with AO-Nesterov50 blocks: the first outer iteration lowers the objective
    T, _ = synth.make_tensor((7, 6, 5), 2, 1e-2, seed=68, dtype=np.float64)
    init = synth.make_init((7, 6, 5), 2, seed=6)
    _, tr = oracle.solve(T, init, 3, her=False, method="nesterov", inner_max=50, track_true=True)
    assert tr.ftrue[0] < tr.fhat0[0]


# --- Tucker-format data (Appendix A) ------------------------------------------

def _tucker(dims, cdims, seed):
    rng = np.random.default_rng(seed)
    G = rng.random(cdims)
    U = [rng.random((d, c)) for d, c in zip(dims, cdims)]
    return G, U


def einsum_expand(G, U):
    N = G.ndim
    core = "abcdefgh"[:N]
    full = "ijklmnop"[:N]
    spec = core + "," + ",".join(full[p] + core[p] for p in range(N)) + "->" + full
    return np.einsum(spec, G, *U)


@pytest.mark.parametrize("dims,cdims,r", [((7, 6, 5), (3, 4, 2), 3), ((5, 4, 6, 3), (2, 3, 2, 2), 2)])
def test_tucker_expand_mttkrp_and_norm(dims, cdims, r):
    G, U = _tucker(dims, cdims, 70)
    T = einsum_expand(G, U)
    np.testing.assert_allclose(oracle.tucker_expand(G, U), T, rtol=1e-13)
    assert oracle.tucker_norm_sq(G, U) == pytest.approx(float(np.sum(T * T)), rel=1e-12)
    F = [np.random.default_rng(71 + l).random((d, r)) for l, d in enumerate(dims)]
    for n in range(len(dims)):
        np.testing.assert_allclose(oracle.tucker_mttkrp(G, U, F, n), oracle.mttkrp(T, F, n), rtol=1e-12)


def test_tucker_identity_bases_reduce_to_dense_solver():
    # U_p = I: the Tucker-format tensor is the core itself, so the two solvers agree
    dims, r = (6, 5, 4), 2
    T, _ = synth.make_tensor(dims, r, 1e-2, seed=72, dtype=np.float64)
    init = synth.make_init(dims, r, seed=7)
    U = [np.eye(d) for d in dims]
    Fd, trd = oracle.solve(T, init, 12, her=True, track_true=True)
    Ft, trt = oracle.solve_tucker(T, U, init, 12, her=True, track_true=True)
    np.testing.assert_allclose(trt.fhat, trd.fhat, rtol=1e-10)
    np.testing.assert_array_equal(trt.restart, trd.restart)
    for a, b in zip(Ft, Fd):
        np.testing.assert_allclose(a, b, rtol=1e-9, atol=1e-12)


def test_tucker_solver_matches_dense_solver_on_expanded_tensor():
    # F_t of eq. objFunTucker is F of the expanded tensor: same trajectory
    dims, cdims, r = (8, 7, 6), (3, 3, 2), 2
    G, U = _tucker(dims, cdims, 73)
    T = einsum_expand(G, U)
    init = synth.make_init(dims, r, seed=8)
    _, trd = oracle.solve(T, init, 15, her=True, track_true=True)
    _, trt = oracle.solve_tucker(G, U, init, 15, her=True, track_true=True)
    assert trt.fhat0[0] == pytest.approx(trd.fhat0[0], rel=1e-10)
    np.testing.assert_array_equal(trt.restart, trd.restart)
    np.testing.assert_allclose(trt.fhat, trd.fhat, rtol=1e-8, atol=1e-10 * trd.fhat0[0])
    np.testing.assert_allclose(trt.ftrue, trd.ftrue, rtol=1e-8, atol=1e-10 * trd.fhat0[0])
