"""Tucker-format data (Appendix A) through the C ABI against the FP64 oracle:
the MTTKRP through the core, the norm, and the HER solver on F_t."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import check_trajectory, rel_fro

pytestmark = pytest.mark.gpu


def _tucker(dims, cdims, seed, **kw):
    import torch
    import paper_2001_04321_gb300 as ntf
    G, U = synth.make_tucker(dims, cdims, seed, **kw)
    X = ntf.Tucker(torch.from_numpy(G).cuda(), [torch.from_numpy(u).cuda() for u in U])
    return G, U, X


@pytest.mark.parametrize("dims,cdims,r", [
    ((40, 50, 60), (5, 6, 7), 4),          # ragged core rows (7 -> pitch 8)
    ((153, 238, 1400), (30, 30, 30), 20),  # the video shape, frames cut to 1400
    ((33, 17, 25, 12), (4, 3, 5, 2), 3),   # 4-way
    ((300, 200, 100), (64, 64, 64), 64),   # largest Tucker rank and rank
    ((70, 80), (9, 12), 5),                # matrix
    ((20, 30, 40), (1, 1, 1), 1),          # rank-one core
])
def test_tucker_mttkrp_matches_oracle(dims, cdims, r):
    import torch
    import paper_2001_04321_gb300 as ntf
    G, U, X = _tucker(dims, cdims, 11 + r)
    F = synth.make_init(dims, r, seed=r)
    Fd = [torch.from_numpy(A).cuda() for A in F]
    for n in range(len(dims)):
        got = ntf.tucker_mttkrp(X, Fd, n).cpu().numpy()
        ref = oracle.tucker_mttkrp(G, U, F, n)
        assert rel_fro(got, ref) <= 1e-5, (n, rel_fro(got, ref))


def test_tucker_norm_matches_oracle_and_expansion():
    import paper_2001_04321_gb300 as ntf
    dims, cdims = (20, 15, 10), (4, 5, 3)
    G, U, X = _tucker(dims, cdims, 3)
    got = ntf.tucker_norm_sq(X).item()
    assert got == pytest.approx(oracle.tucker_norm_sq(G, U), rel=1e-6)
    T = oracle.tucker_expand(G, U)
    assert got == pytest.approx(float(np.sum(T * T)), rel=1e-6)
    _, _, X2 = _tucker((153, 238, 14000), (30, 30, 30), 4)
    G2, U2 = synth.make_tucker((153, 238, 14000), (30, 30, 30), 4)
    assert ntf.tucker_norm_sq(X2).item() == pytest.approx(oracle.tucker_norm_sq(G2, U2), rel=1e-6)


def test_tucker_mttkrp_full_video_shape_sampled():
    # 153 x 238 x 14000 (the surveillance video's shape) with a 30^3 core, rank 20: the
    # compressed oracle runs at full size, so every row is compared
    import torch
    import paper_2001_04321_gb300 as ntf
    dims, cdims, r = (153, 238, 14000), (30, 30, 30), 20
    G, U, X = _tucker(dims, cdims, 5)
    F = synth.make_init(dims, r, seed=5)
    Fd = [torch.from_numpy(A).cuda() for A in F]
    for n in range(3):
        got = ntf.tucker_mttkrp(X, Fd, n).cpu().numpy()
        ref = oracle.tucker_mttkrp(G, U, F, n)
        assert rel_fro(got, ref) <= 1e-5


def test_tucker_mttkrp_equals_dense_mttkrp_of_expanded_tensor():
    import torch
    import paper_2001_04321_gb300 as ntf
    dims, cdims, r = (24, 20, 16), (5, 4, 6), 6
    G, U, X = _tucker(dims, cdims, 6)
    T = oracle.tucker_expand(G, U).astype(np.float32)
    F = synth.make_init(dims, r, seed=6)
    Fd = [torch.from_numpy(A).cuda() for A in F]
    Td = torch.from_numpy(T).cuda()
    for n in range(3):
        a = ntf.tucker_mttkrp(X, Fd, n).cpu().numpy()
        b = ntf.mttkrp(Td, Fd, n).cpu().numpy()
        assert rel_fro(a, b) <= 1e-5


@pytest.mark.parametrize("her,par", [(True, {}), (False, {}),
                                     (True, dict(beta0=0.95, gamma=1.5, gamma_bar=1.2, eta=2.0))])
def test_tucker_solver_trajectory(her, par):
    import torch
    import paper_2001_04321_gb300 as ntf
    # the Tucker form of a noisy rank-6 CP tensor (core: superdiagonal + 5% U[0,1]); the
    # aggressive HER parameters of the third case make iteration 5 restart
    dims, cdims, r, iters = (60, 70, 300), (8, 8, 8), 6, 25
    G, U, X = _tucker(dims, cdims, 7, rank=6, noise=0.05)
    init = synth.make_init(dims, r, seed=7)
    s = ntf.Solver.tucker(X, [torch.from_numpy(A).cuda() for A in init],
                          ntf.Opts(her=her, max_iters=iters, **par))
    fh, rs, prev = [], [], 0
    for _ in range(iters):
        s.run(1)
        rep = s.report()
        fh.append(rep.f_hat_last)
        rs.append(rep.restarts - prev)
        prev = rep.restarts
    s.close()
    Fo, tr = oracle.solve_tucker(G, U, init, iters, her=her, track_true=True, **par)
    if par:
        assert tr.restart.sum() >= 1
    tn = oracle.tucker_norm_sq(G, U)
    check_trajectory(fh, rs, tr, tn, 8, f_true=rep.f_true_last, f_true_ref=tr.ftrue[-1])
    assert rep.tnorm_sq == pytest.approx(tn, rel=1e-6)


def test_solve_tucker_matches_dense_solve_on_expanded_tensor():
    import torch
    import paper_2001_04321_gb300 as ntf
    dims, cdims, r = (30, 25, 20), (4, 4, 4), 4
    G, U, X = _tucker(dims, cdims, 8)
    T = oracle.tucker_expand(G, U).astype(np.float32)
    init = synth.make_init(dims, r, seed=8)
    Ft = [torch.from_numpy(A).cuda() for A in init]
    rt = ntf.solve_tucker(X, Ft, ntf.Opts(max_iters=30))
    Td = torch.from_numpy(T).cuda()
    Fd = [torch.from_numpy(A).cuda() for A in init]
    rd = ntf.solve(Td, Fd, ntf.Opts(max_iters=30))
    assert rt.f_true_last == pytest.approx(rd.f_true_last, rel=1e-3)
    assert rt.iters == rd.iters == 30
