"""CP loss as a torch.autograd.Function (step a9): forward (1/2)||T - X||^2 and
the hand-written backward A_n V_n - M_n (Sec. 2, eq. def:grad) through the C
ABI, against central differences of the FP64 oracle objective and against the
oracle's explicit-residual gradient."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import device_tensor, rel_fro

pytestmark = pytest.mark.gpu


def _leaf(A):
    import torch
    return torch.from_numpy(np.ascontiguousarray(A, dtype=np.float32)).cuda().requires_grad_(True)


def test_cploss_central_differences_30cube_r4():
    # 30^3, r = 4: every factor entry against a central difference (step 1e-3) of
    # the FP64 explicit objective.  The loss is quadratic in each single entry,
    # so the central difference is exact up to rounding.
    import paper_2001_04321_gb300 as ntf
    dims, r = (30, 30, 30), 4
    T, _ = synth.make_tensor(dims, r, 0.05, seed=77)
    F = [A.astype(np.float32) for A in synth.make_init(dims, r, seed=77)]
    Td, d, ld = device_tensor(T)
    leaves = [_leaf(A) for A in F]
    loss = ntf.cp_loss(Td, leaves, dims=d, ld=ld)
    loss.backward()
    T64 = T.astype(np.float64)
    F64 = [A.astype(np.float64) for A in F]
    ref_loss = 0.5 * oracle.objective_explicit(T64, F64)
    assert loss.item() == pytest.approx(ref_loss, rel=1e-5)
    h = 1e-3
    for n in range(3):
        fd = np.zeros_like(F64[n])
        for i in range(dims[n]):
            for p in range(r):
                Fp = [A.copy() for A in F64]
                Fm = [A.copy() for A in F64]
                Fp[n][i, p] += h
                Fm[n][i, p] -= h
                fd[i, p] = 0.5 * (oracle.objective_explicit(T64, Fp) - oracle.objective_explicit(T64, Fm)) / (2 * h)
        assert rel_fro(leaves[n].grad.cpu().numpy(), fd) <= 1e-4, n


@pytest.mark.parametrize("dims,r,dtype", [((13, 7, 9, 6), 5, "f32"), ((17, 11, 40), 8, "bf16"),
                                          ((129, 3, 70), 33, "f32")])
def test_cploss_matches_oracle_gradient(dims, r, dtype):
    # every factor's gradient against the MTTKRP of the explicit residual, with
    # an upstream gradient of 3 (loss scaled before backward)
    import paper_2001_04321_gb300 as ntf
    T, _ = synth.make_tensor(dims, r, 0.05, seed=5)
    F = [A.astype(np.float32) for A in synth.make_init(dims, r, seed=5)]
    Td, d, ld = device_tensor(T, dtype)
    Tref = T.astype(np.float64)
    if dtype == "bf16":
        Tref = oracle.bf16_to_f64(oracle.round_bf16(np.ascontiguousarray(T, dtype=np.float32)))
    leaves = [_leaf(A) for A in F]
    loss = ntf.cp_loss(Td, leaves, dims=d, ld=ld)
    (3.0 * loss).backward()
    F64 = [A.astype(np.float64) for A in F]
    assert loss.item() == pytest.approx(0.5 * oracle.objective_explicit(Tref, F64), rel=1e-5)
    for n in range(len(dims)):
        ref = 3.0 * oracle.cp_gradient(Tref, F64, n)
        assert rel_fro(leaves[n].grad.cpu().numpy(), ref) <= 1e-5, n


def test_cploss_partial_requires_grad_and_graph_composition():
    # only factor 1 asks for a gradient; the loss composes with torch ops
    import torch
    import paper_2001_04321_gb300 as ntf
    dims, r = (12, 10, 8), 3
    T, _ = synth.make_tensor(dims, r, 0.0, seed=9)
    F = [A.astype(np.float32) for A in synth.make_init(dims, r, seed=9)]
    Td, d, ld = device_tensor(T)
    A0 = torch.from_numpy(F[0]).cuda()
    A1 = _leaf(F[1])
    A2 = torch.from_numpy(F[2]).cuda()
    loss = ntf.cp_loss(Td, [A0, A1, A2], dims=d, ld=ld)
    (loss * loss).backward()
    F64 = [A.astype(np.float64) for A in F]
    ref = 2.0 * loss.item() * oracle.cp_gradient(T.astype(np.float64), F64, 1)
    assert rel_fro(A1.grad.cpu().numpy(), ref) <= 1e-5


def test_cploss_gradient_descent_decreases_loss():
    # a few projected gradient steps driven by torch.optim with the hand-written backward
    import torch
    import paper_2001_04321_gb300 as ntf
    dims, r = (40, 30, 20), 6
    T, _ = synth.make_tensor(dims, r, 0.01, seed=3)
    F = [A.astype(np.float32) for A in synth.make_init(dims, r, seed=3)]
    Td, d, ld = device_tensor(T)
    leaves = [_leaf(A) for A in F]
    opt = torch.optim.SGD(leaves, lr=1e-4)
    losses = []
    for _ in range(20):
        opt.zero_grad()
        loss = ntf.cp_loss(Td, leaves, dims=d, ld=ld)
        loss.backward()
        opt.step()
        with torch.no_grad():
            for A in leaves:
                A.clamp_(min=0)
        losses.append(loss.item())
    assert losses[-1] < losses[0]
    assert all(np.isfinite(losses))


def test_cploss_fullsize_300cube_r32_sampled_rows():
    # 300^3, r = 32: sampled gradient rows against the oracle's row-by-row
    # MTTKRP of the tensor slab and its Grams
    import torch
    import paper_2001_04321_gb300 as ntf
    w = synth.WORKLOADS["cube300_r32"]
    dims, r = w["dims"], w["rank"]
    T, _ = synth.make_tensor(dims, r, w["noise_rel"], seed=w["seed"], recipe=w["recipe"])
    F = [A.astype(np.float32) for A in synth.make_init(dims, r, seed=0)]
    Td = torch.from_numpy(T).cuda()
    leaves = [_leaf(A) for A in F]
    loss = ntf.cp_loss(Td, leaves)
    loss.backward()
    F64 = [A.astype(np.float64) for A in F]
    G = [oracle.gram(A) for A in F64]
    rng = np.random.default_rng(1)
    for n in range(3):
        g = leaves[n].grad.cpu().numpy()
        V = oracle.hadamard_grams(G, n)
        for j in sorted(set([0, dims[n] - 1] + list(rng.integers(0, dims[n], 3)))):
            sl = [slice(None)] * 3
            sl[n] = slice(j, j + 1)
            Fs = list(F64)
            Fs[n] = F64[n][j:j + 1]
            M = oracle.mttkrp(np.ascontiguousarray(T[tuple(sl)]), Fs, n)[0]
            AV = F64[n][j] @ V
            ref = AV - M
            err = np.linalg.norm(g[j] - ref)
            assert err <= 1e-5 * (np.linalg.norm(AV) + np.linalg.norm(M)), (n, j)
    ntf.device_status()


def test_block_gradient_entry_point():
    import torch
    import paper_2001_04321_gb300 as ntf
    rng = np.random.default_rng(4)
    for rows, r in [(1, 1), (333, 20), (5000, 64)]:
        A = rng.random((rows, r)).astype(np.float32)
        M = rng.random((rows, r)).astype(np.float32)
        B = rng.random((r, r))
        V = B @ B.T
        s = torch.tensor(2.5, dtype=torch.float64, device="cuda")
        out = ntf.block_gradient(torch.from_numpy(A).cuda(), torch.from_numpy(M).cuda(),
                                 torch.from_numpy(V).cuda(), -0.5, scale_dev=s).cpu().numpy()
        ref = -1.25 * (A.astype(np.float64) @ V - M)
        assert rel_fro(out, ref) <= 1e-6
    with pytest.raises(ntf.NTFError):
        ntf.block_gradient(torch.zeros(4, 65, device="cuda"), torch.zeros(4, 65, device="cuda"),
                           torch.zeros(65, 65, dtype=torch.float64, device="cuda"))


def test_cploss_with_precomputed_norm_and_cuda_graph():
    # ||T||^2 passed in gives the same loss and gradients; the forward + backward can be
    # captured as one CUDA graph and replayed, matching the eager result bit for bit
    import torch
    import paper_2001_04321_gb300 as ntf
    dims, r = (40, 30, 20), 6
    T, _ = synth.make_tensor(dims, r, 0.05, seed=21)
    F = [A.astype(np.float32) for A in synth.make_init(dims, r, seed=21)]
    Td, d, ld = device_tensor(T)
    leaves = [_leaf(A) for A in F]
    loss = ntf.cp_loss(Td, leaves, dims=d, ld=ld)
    loss.backward()
    ref = [A.grad.clone() for A in leaves]
    tn = ntf.tensor_norm_sq(Td, dims=d, ld=ld)
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    leaves2 = [_leaf(A) for A in F]

    def step():
        for A in leaves2:
            A.grad = None
        out = ntf.cp_loss(Td, leaves2, dims=d, ld=ld, tnorm_sq=tn)
        out.backward()
        return out

    with torch.cuda.stream(st):
        for _ in range(2):
            l2 = step()
    torch.cuda.synchronize()
    assert l2.item() == loss.item()
    assert all(torch.equal(a.grad, b) for a, b in zip(leaves2, ref))
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st, capture_error_mode="thread_local"):
        l3 = step()
    for A in leaves2:
        A.grad = None
    g.replay()
    torch.cuda.synchronize()
    assert l3.item() == loss.item()
    F64 = [A.astype(np.float64) for A in F]
    for n in range(3):
        assert rel_fro(ref[n].cpu().numpy(), oracle.cp_gradient(T.astype(np.float64), F64, n)) <= 1e-5
