"""Pins of how the oracle strings Alg. 2 together, not only of its pieces.

Each piece of the HER iteration is pinned in ``test_oracle_pins.py``.  These
tests pin the composition, using the factors the oracle records at every
iteration (right after the block updates, the extrapolated ones before the
decision, and the ones after it):

* with beta_0 = 0 the weight stays 0 (both branches of eqs. HER_eq:beta_update
  and HER_eq:beta_bar_update keep it there), so Alg. 2 must reproduce Alg. 1;
* F-hat_k is F at (A_hat^1_k, .., A_hat^{N-1}_k, A^N_k) (Alg. 2, restart test),
  checked by an explicit reconstruction with numpy, and differs from F at the
  all-extrapolated point;
* the extrapolation uses beta_{k-1} and the factors kept by the previous
  decision (eq. extproj_her);
* the decision copies one sequence onto the other for every block and
  restarts exactly when F-hat rises (Alg. 2);
* block i is updated against the extrapolated blocks A_hat^l_k (l < i) and
  A_hat^l_{k-1} (l > i) (eq. NNLS_her_exact): with the inner solve run to
  convergence, every updated row is scipy's NNLS solution for the Khatri-Rao
  matrix of those blocks.
"""
import numpy as np
import pytest

import oracle
import synth


def explicit_objective(T, F):
    letters = "abcdefgh"[:T.ndim]
    spec = ",".join(c + "z" for c in letters) + "->" + letters
    X = np.einsum(spec, *F)
    return float(np.sum((T - X) ** 2))


def _problem(dims=(9, 8, 7), r=3, seed=23, noise=1e-2):
    T, _ = synth.make_tensor(dims, r, noise, seed=seed, dtype=np.float64)
    init = [A.astype(np.float64) for A in synth.make_init(dims, r, seed=seed % 7)]
    return T, init


@pytest.mark.parametrize("method", ["hals", "pgd", "nesterov"])
def test_beta0_zero_reproduces_alg1(method):
    T, init = _problem()
    F1, plain = oracle.solve(T, init, 25, her=False, method=method, inner_max=3)
    F2, her0 = oracle.solve(T, init, 25, her=True, beta0=0.0, method=method, inner_max=3, track_true=True)
    np.testing.assert_array_equal(her0.fhat, plain.fhat)
    np.testing.assert_array_equal(her0.beta, 0.0)
    for a, b in zip(F1, F2):
        np.testing.assert_array_equal(a, b)
    # without extrapolation F-hat is the objective at A_k itself
    np.testing.assert_allclose(her0.fhat, her0.ftrue, rtol=1e-9)


def test_fhat_is_objective_at_extrapolated_pairing():
    T, init = _problem()
    K = 30
    _, tr = oracle.solve(T, init, K, her=True, track_factors=True)
    N = T.ndim
    gap = 0.0
    for k in range(1, K + 1):
        Ah, Au = tr.A_hat(k), tr.A_updated(k)
        point = Ah[:N - 1] + [Au[N - 1]]
        assert tr.fhat[k - 1] == pytest.approx(explicit_objective(T, point), rel=1e-10)
        gap = max(gap, abs(explicit_objective(T, Ah) - tr.fhat[k - 1]) / tr.fhat[k - 1])
    assert gap > 1e-3    # F at A_hat^N would be a different sequence


def test_extrapolation_uses_previous_beta_and_kept_factors():
    T, init = _problem()
    K, beta0 = 30, 0.5
    _, tr = oracle.solve(T, init, K, her=True, beta0=beta0, track_factors=True)
    assert 0 < tr.restart.sum() < K           # both branches occur
    prev = init
    wrong_beta = 0      # iterations where beta_k in place of beta_{k-1} would give another A_hat
    for k in range(1, K + 1):
        beta = beta0 if k == 1 else tr.beta[k - 2]
        for l, (a, p, ah) in enumerate(zip(tr.A_updated(k), prev, tr.A_hat(k))):
            np.testing.assert_allclose(ah, np.maximum(0.0, a + beta * (a - p)), rtol=1e-13, atol=1e-15)
            alt = np.maximum(0.0, a + tr.beta[k - 1] * (a - p))
            wrong_beta += int(np.abs(alt - ah).max() > 1e-9 * np.abs(ah).max())
        prev = tr.A_after(k)
    assert wrong_beta >= K // 2


def test_decision_copies_whole_sequence_and_restarts_when_fhat_rises():
    T, init = _problem()
    K = 30
    _, tr = oracle.solve(T, init, K, her=True, track_factors=True)
    fprev = tr.fhat0[0]
    for k in range(1, K + 1):
        assert tr.restart[k - 1] == int(tr.fhat[k - 1] > fprev)
        src = tr.A_updated(k) if tr.restart[k - 1] else tr.A_hat(k)
        for a, b in zip(tr.A_after(k), src):
            np.testing.assert_array_equal(a, b)
        fprev = tr.fhat[k - 1]


def _kr_and_unfolding(T, F, i):
    """Library route: the unfolding of mode i and the matching Khatri-Rao rows
    (C order over the other modes), via numpy reshapes and einsum."""
    others = [l for l in range(T.ndim) if l != i]
    Ti = np.moveaxis(T, i, 0).reshape(T.shape[i], -1)
    letters = "abcdefgh"[:len(others)]
    spec = ",".join(c + "z" for c in letters) + "->" + letters + "z"
    B = np.einsum(spec, *[F[l] for l in others]).reshape(-1, F[others[0]].shape[1])
    return Ti, B


def test_block_update_pairs_with_extrapolated_blocks():
    scipy_opt = pytest.importorskip("scipy.optimize")
    dims, r = (6, 5, 4), 2
    T, init = _problem(dims, r, seed=51, noise=5e-2)
    K = 5
    _, tr = oracle.solve(T, init, K, her=True, inner_max=6000, inner_tol=0.0, track_factors=True)
    prev_hat = init                    # A_hat_0 = A_0
    moved = 0.0
    for k in range(1, K + 1):
        Au, Ah = tr.A_updated(k), tr.A_hat(k)
        for i in range(len(dims)):
            pairing = [Ah[l] if l < i else prev_hat[l] for l in range(len(dims))]
            Ti, B = _kr_and_unfolding(T, pairing, i)
            for row in range(dims[i]):
                x, _ = scipy_opt.nnls(B, Ti[row])
                np.testing.assert_allclose(Au[i][row], x, rtol=1e-6, atol=1e-8)
            moved = max(moved, max(float(np.abs(Ah[l] - Au[l]).max()) for l in range(i)) if i else 0.0)
        # after the decision A_hat_k and A_k coincide (Alg. 2 sets one to the other)
        prev_hat = tr.A_after(k)
    assert moved > 1e-3     # extrapolated and updated blocks differ: pairing on A would fail


def test_forced_decisions_follow_alg2_branches():
    # the tests' tie-following hook: forcing the decision the comparison would take changes
    # nothing; forcing the other one takes that branch of Alg. 2 with its beta updates
    # (eqs. HER_eq:beta_update, HER_eq:beta_bar_update) and keeps F-hat_{k-1} <- F-hat_k
    T, init = _problem()
    K = 20
    _, a = oracle.solve(T, init, K, her=True, track_factors=True)
    _, same = oracle.solve(T, init, K, her=True, force=a.restart.astype(np.int32))
    np.testing.assert_array_equal(same.fhat, a.fhat)
    k = 4
    force = np.full(K, -1, dtype=np.int32)
    force[k] = 1 - a.restart[k]
    _, b = oracle.solve(T, init, K, her=True, force=force, track_factors=True)
    np.testing.assert_array_equal(b.fhat[:k + 1], a.fhat[:k + 1])
    assert b.restart[k] == 1 - a.restart[k]
    beta_prev, bar_prev = a.beta[k - 1], a.beta_bar[k - 1]
    if b.restart[k]:
        assert b.beta[k] == pytest.approx(beta_prev / 1.5) and b.beta_bar[k] == pytest.approx(beta_prev)
        src = b.A_updated(k + 1)
    else:
        assert b.beta[k] == pytest.approx(min(bar_prev, 1.05 * beta_prev))
        assert b.beta_bar[k] == pytest.approx(min(1.0, 1.01 * bar_prev))
        src = b.A_hat(k + 1)
    for x, y in zip(b.A_after(k + 1), src):
        np.testing.assert_array_equal(x, y)
    # the next decision compares against this iteration's real F-hat
    assert b.restart[k + 1] == int(b.fhat[k + 1] > b.fhat[k])
