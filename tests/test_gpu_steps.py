"""Parity of steps a2-a8 (Grams, Hadamard of Grams, HALS/PGD block update,
HER extrapolation and decision, objective by reuse, explicit residual,
||T||^2, bf16 cast) through the C ABI against the FP64 oracle."""
import os

import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import device_tensor, rel_fro

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def cuda(x, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


@pytest.mark.parametrize("rows,r", [(500, 20), (1000, 64), (3, 1), (129, 7), (4000, 16)])
def test_gram(rows, r):
    import paper_2001_04321_gb300 as ntf
    A = np.random.default_rng(rows + r).random((rows, r)).astype(np.float32)
    G = ntf.gram(cuda(A)).cpu().numpy()
    assert rel_fro(G, oracle.gram(A)) <= 1e-6
    assert np.array_equal(G, G.T)


def test_hadamard_grams():
    import paper_2001_04321_gb300 as ntf
    rng = np.random.default_rng(1)
    Gs = [rng.random((6, 6)) for _ in range(4)]
    for skip in (-1, 0, 2, 3):
        V = ntf.hadamard_grams([cuda(g) for g in Gs], skip).cpu().numpy()
        ref = oracle.hadamard_grams(Gs, skip)
        np.testing.assert_allclose(V, ref, rtol=1e-15)


def _block(seed, I, r, dims_other=(30, 20)):
    rng = np.random.default_rng(seed)
    others = [rng.random((d, r)) for d in dims_other]
    B = np.einsum("iz,jz->ijz", *others).reshape(-1, r)
    Tn = rng.random((I, B.shape[0]))
    M = (Tn @ B).astype(np.float32)
    V = B.T @ B
    A0 = rng.random((I, r)).astype(np.float32)
    return A0, M, V


@pytest.mark.parametrize("method", ["hals", "pgd"])
@pytest.mark.parametrize("rows,r,inner", [(300, 10, 1), (300, 10, 20), (1500, 12, 1), (1500, 12, 8), (64, 33, 3),
                                          (7, 1, 4)])
def test_block_update(method, rows, r, inner):
    import paper_2001_04321_gb300 as ntf
    A0, M, V = _block(rows * 7 + r, rows, r)
    A = cuda(A0)
    ntf.bcd_update(A, cuda(M), cuda(V), method=method, inner_max=inner, inner_tol=0.0)
    if method == "hals":
        ref, _ = oracle.hals(A0, M, V, inner_max=inner, inner_tol=0.0)
    else:
        ref, _ = oracle.pgd(A0, M, V, inner_max=inner, inner_tol=0.0)
    got = A.cpu().numpy()
    assert rel_fro(got, ref) <= (1e-5 if inner == 1 else 1e-4)
    assert np.all(got >= 0)


@pytest.mark.parametrize("rows", [400, 2000])
def test_block_update_stop_rule(rows):
    # the inner stopping rule of Sec. 4.1 stops early: result equals the oracle's
    import paper_2001_04321_gb300 as ntf
    A0, M, V = _block(77 + rows, rows, 8)
    A = cuda(A0)
    ntf.bcd_update(A, cuda(M), cuda(V), method="hals", inner_max=50, inner_tol=1e-2)
    ref, sweeps = oracle.hals(A0, M, V, inner_max=50, inner_tol=1e-2)
    assert 1 < sweeps < 50
    assert rel_fro(A.cpu().numpy(), ref) <= 1e-4


def test_hals_zero_diagonal_column_unchanged():
    import paper_2001_04321_gb300 as ntf
    A0, M, V = _block(5, 100, 4)
    V = V.copy()
    V[2, :] = 0
    V[:, 2] = 0
    A = cuda(A0)
    ntf.bcd_update(A, cuda(M), cuda(V), method="hals")
    assert np.array_equal(A.cpu().numpy()[:, 2], A0[:, 2])


def test_extrapolate():
    import torch
    import paper_2001_04321_gb300 as ntf
    rng = np.random.default_rng(3)
    A = rng.random(1000).astype(np.float32)
    P = rng.random(1000).astype(np.float32)
    beta = torch.tensor([0.7], dtype=torch.float64, device="cuda")
    out = ntf.her_extrapolate(cuda(A), cuda(P), beta).cpu().numpy()
    ref = oracle.extrapolate(A, P, 0.7)
    np.testing.assert_allclose(out, ref, rtol=1e-6, atol=1e-7)
    assert np.all(out >= 0) and np.any(out == 0)


def test_objective_identity_and_residual_and_norm():
    import torch
    import paper_2001_04321_gb300 as ntf
    dims, r = (30, 25, 20), 4
    T, _ = synth.make_tensor(dims, r, 1e-2, seed=8)
    F = synth.make_init(dims, r, seed=8)
    buf, d, ld = device_tensor(T)
    tn = ntf.tensor_norm_sq(buf, dims=d, ld=ld)
    assert abs(tn.item() - oracle.norm_sq(T)) <= 1e-7 * oracle.norm_sq(T)
    Fd = [cuda(A) for A in F]
    G = [oracle.gram(A) for A in F]
    V = oracle.hadamard_grams(G, 2)
    M = oracle.mttkrp(T, F, 2).astype(np.float32)
    got = ntf.objective(tn, cuda(M), Fd[2], cuda(V)).item()
    ref = oracle.objective_identity(oracle.norm_sq(T), M, F[2], V)
    assert abs(got - ref) <= 1e-6 * oracle.norm_sq(T)
    res = ntf.residual_sq(buf, Fd, dims=d, ld=ld).item()
    ref2 = oracle.objective_explicit(T, F)
    assert abs(res - ref2) <= 1e-5 * ref2


def test_residual_small_relative_to_norm():
    # a near-exact fit: the explicit residual must not cancel (it forms T - X first)
    import paper_2001_04321_gb300 as ntf
    dims, r = (40, 30, 20), 3
    T, A_true = synth.make_tensor(dims, r, 1e-4, seed=9)
    F = [A.astype(np.float32) for A in A_true]
    buf, d, ld = device_tensor(T)
    res = ntf.residual_sq(buf, [cuda(A) for A in F], dims=d, ld=ld).item()
    ref = oracle.objective_explicit(T, F)
    assert ref < 1e-6 * oracle.norm_sq(T)
    assert abs(res - ref) <= 2e-2 * ref


def test_bf16_cast_bit_exact():
    import torch
    rng = np.random.default_rng(11)
    x = np.concatenate([rng.standard_normal(4093).astype(np.float32) * 30,
                        np.array([1.00390625, 1.01171875, -2.00781250, 0.0], dtype=np.float32)])
    T = x.reshape(1, 1, -1)
    buf, d, ld = device_tensor(T, "bf16")
    got = buf.view(torch.int16).cpu().numpy().view(np.uint16)[: x.size]
    assert np.array_equal(got, oracle.round_bf16(x))
    assert ld % 8 == 0 and np.all(buf.view(torch.int16).cpu().numpy()[x.size:ld] == 0)


def _golden_table():
    rows = []
    with open(os.path.join(GOLDEN, "her_beta_table.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_her_step_golden_table_and_copies():
    import torch
    import paper_2001_04321_gb300 as ntf
    state = torch.zeros(ntf.HER_STATE_BYTES, dtype=torch.uint8, device="cuda")
    f = torch.tensor([10.0], dtype=torch.float64, device="cuda")
    ntf.her_state_init(state, f)
    A = [torch.full((5, 3), 1.0, device="cuda"), torch.full((4, 3), 2.0, device="cuda")]
    Ah = [torch.full((5, 3), 3.0, device="cuda"), torch.full((4, 3), 4.0, device="cuda")]
    fv = 10.0
    for step, dec, beta, beta_bar in _golden_table():
        fv = fv - 1.0 if dec == "a" else fv + 1.0
        f.fill_(fv)
        before_A = [a.clone() for a in A]
        before_Ah = [a.clone() for a in Ah]
        ntf.her_step(state, A, Ah, f)
        s = ntf.her_state_read(state)
        assert s["last_restart"] == (dec == "r")
        assert s["beta"] == pytest.approx(float(beta), rel=1e-14)
        assert s["beta_bar"] == pytest.approx(float(beta_bar), rel=1e-14)
        assert s["f_hat_prev"] == fv
        for l in range(2):
            if dec == "r":
                assert torch.equal(Ah[l], before_A[l]) and torch.equal(A[l], before_A[l])
            else:
                assert torch.equal(A[l], before_Ah[l]) and torch.equal(Ah[l], before_Ah[l])
        # make the pair differ again for the next step
        A[0].add_(0.5)
        Ah[1].add_(0.25)
    s = ntf.her_state_read(state)
    assert s["iters"] == 6 and s["restarts"] == 3


def test_bounded_wait_gives_up_and_reports_timeout():
    # a kernel waits on an mbarrier that nothing arrives on: it gives up after 10 ms,
    # the host reads NTF_ETIMEOUT, the error word is cleared and the context stays usable
    import torch
    import paper_2001_04321_gb300 as ntf
    st = ntf.check_wait_timeout(10_000_000)
    assert st == 5   # NTF_ETIMEOUT
    ntf.device_status()   # cleared: no error now
    A = torch.rand(100, 8, device="cuda")
    G = ntf.gram(A).cpu().numpy()
    assert np.allclose(G, (A.double().T @ A.double()).cpu().numpy(), rtol=1e-6)
