"""Whole-solver parity (Alg. 1 / Alg. 2) against the FP64 oracle from the same
initial factors.  The paper's method is a heuristic iteration, so the check
is trajectory-wise: F-hat per iteration up to the first differing restart
decision, and always the final objective within 1e-3 relative.  The fused
path's factors are also compared element by element for the first
iterations."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import check_trajectory, device_tensor, follow_trajectory, rel_fro

pytestmark = pytest.mark.gpu


def _setup(dims, r, noise, seed, recipe="uniform"):
    import torch
    T, A_true = synth.make_tensor(dims, r, noise, seed=seed, recipe=recipe)
    init = synth.make_init(dims, r, seed=seed)
    buf, d, ld = device_tensor(T)
    Fd = [torch.from_numpy(A).cuda() for A in init]
    return T, init, buf, d, ld, Fd


def _trajectory(buf, d, ld, Fd, iters, opts):
    import paper_2001_04321_gb300 as ntf
    s = ntf.Solver(buf, Fd, opts, dims=d, ld=ld)
    fh, rs = [], []
    prev_restarts = 0
    for _ in range(iters):
        s.run(1)
        rep = s.report()
        fh.append(rep.f_hat_last)
        rs.append(rep.restarts - prev_restarts)
        prev_restarts = rep.restarts
    rep = s.report()
    s.close()
    return np.array(fh), np.array(rs), rep


_check_trajectory = check_trajectory


@pytest.mark.parametrize("her", [True, False])
def test_solver_trajectory_20cube(her):
    import paper_2001_04321_gb300 as ntf
    dims, r, iters = (20, 20, 20), 5, 50
    T, init, buf, d, ld, Fd = _setup(dims, r, 1e-2, 1234)
    fh, rs, rep = _trajectory(buf, d, ld, Fd, iters, ntf.Opts(her=her, max_iters=iters))
    _, tr = oracle.solve(T, init, iters, her=her, track_true=True)
    # identical decisions up to the first divergence; F-hat agrees there.  FP32
    # factors carry rounding of ~6e-8 relative per update, so F-hat (a difference
    # of terms of size ||T||^2) agrees to an absolute 1e-6 ||T||^2, not relatively.
    _check_trajectory(fh, rs, tr, oracle.norm_sq(T), 10, f_true=rep.f_true_last, f_true_ref=tr.ftrue[-1])
    if not her:
        assert rs.sum() == 0
        # Alg. 1 never increases F (up to FP32 rounding of the objective)
        assert np.all(np.diff(fh) <= 1e-6 * oracle.norm_sq(T))


def test_solver_4way_and_pgd():
    import paper_2001_04321_gb300 as ntf
    dims, r, iters = (10, 9, 8, 7), 4, 30
    T, init, buf, d, ld, Fd = _setup(dims, r, 1e-2, 77, recipe="sparse30")
    tn = oracle.norm_sq(T)
    fh, rs, rep = _trajectory(buf, d, ld, [A.clone() for A in Fd], iters, ntf.Opts(max_iters=iters))
    _, tr = oracle.solve(T, init, iters, her=True, track_true=True)
    _check_trajectory(fh, rs, tr, tn, 5, f_true=rep.f_true_last, f_true_ref=tr.ftrue[-1])
    opts = ntf.Opts(max_iters=10, method="pgd", inner_max=5, her=True)
    fh, rs, rep = _trajectory(buf, d, ld, [A.clone() for A in Fd], 10, opts)
    _, tr = oracle.solve(T, init, 10, her=True, method="pgd", inner_max=5, track_true=True)
    _check_trajectory(fh, rs, tr, tn, 5, f_true=rep.f_true_last, f_true_ref=tr.ftrue[-1])


def test_solver_ahals_inner_loop():
    import paper_2001_04321_gb300 as ntf
    dims, r, iters = (30, 25, 20), 4, 20
    T, init, buf, d, ld, Fd = _setup(dims, r, 1e-2, 91)
    opts = ntf.Opts(max_iters=iters, inner_max=50, inner_tol=1e-2)
    fh, rs, rep = _trajectory(buf, d, ld, [A.clone() for A in Fd], iters, opts)
    # this trajectory has a near-tie at iteration 14 (F_14 - F_13 = -8e-8 ||T||^2) that rounding
    # decides either way: the oracle follows the solver's branch there, and then every F-hat
    # and the final objective agree
    run = lambda force: oracle.solve(T, init, iters, her=True, inner_max=50, inner_tol=1e-2, track_true=True,
                                     force=force)
    _, tr, ties = follow_trajectory(fh, rs, run, oracle.norm_sq(T))
    assert ties <= 2
    assert abs(rep.f_true_last - tr.ftrue[-1]) <= 1e-3 * tr.ftrue[-1]


def test_solver_outputs_feasible_and_match_report():
    import paper_2001_04321_gb300 as ntf
    dims, r = (33, 21, 17), 6
    T, init, buf, d, ld, Fd = _setup(dims, r, 1e-2, 5)
    F = [A.clone() for A in Fd]
    rep = ntf.solve(buf, F, ntf.Opts(max_iters=25), dims=d, ld=ld)
    Fh = [A.cpu().numpy() for A in F]
    assert all(np.all(A >= 0) for A in Fh)
    assert rep.f_true_last == pytest.approx(oracle.objective_explicit(T, Fh), rel=1e-4)
    assert rep.rel_error == pytest.approx(np.sqrt(rep.f_true_last / oracle.norm_sq(T)), rel=1e-9)
    assert 0 < rep.beta_last <= rep.beta_bar_last <= 1.0


def test_solve_host_equals_device_solve():
    import torch
    import paper_2001_04321_gb300 as ntf
    dims, r = (24, 20, 16), 5
    T, init, buf, d, ld, Fd = _setup(dims, r, 1e-2, 6)
    F = [A.clone() for A in Fd]
    rep_d = ntf.solve(buf, F, ntf.Opts(max_iters=15), dims=d, ld=ld)
    Th = torch.from_numpy(T).pin_memory()
    Fh = [torch.from_numpy(A.copy()).pin_memory() for A in init]
    rep_h = ntf.solve_host(Th, Fh, ntf.Opts(max_iters=15))
    assert rep_h.f_true_last == rep_d.f_true_last
    for a, b in zip(F, Fh):
        assert torch.equal(a.cpu(), b)


def test_bf16_form_matches_fp32_error():
    import paper_2001_04321_gb300 as ntf
    dims, r, iters = (60, 50, 40), 6, 60
    T, init, buf, d, ld, Fd = _setup(dims, r, 1e-2, 12)
    F32 = [A.clone() for A in Fd]
    rep32 = ntf.solve(buf, F32, ntf.Opts(max_iters=iters), dims=d, ld=ld)
    F16 = [A.clone() for A in Fd]
    rep16 = ntf.solve(buf, F16, ntf.Opts(max_iters=iters, compute_dtype="bf16"), dims=d, ld=ld)
    # both reports are against the FP32 tensor; bf16 storage adds ~1e-3 relative quantisation noise
    assert abs(rep16.rel_error - rep32.rel_error) <= 1e-3


def test_noiseless_recovery_fp32():
    import paper_2001_04321_gb300 as ntf
    dims, r = (30, 30, 30), 3
    ok = 0
    for run in range(3):
        T, init, buf, d, ld, Fd = _setup(dims, r, 0.0, 300 + run)
        rep = ntf.solve(buf, Fd, ntf.Opts(max_iters=600), dims=d, ld=ld)
        ok += rep.rel_error < 1e-4
    assert ok >= 2


def test_graph_replay_matches_eager():
    import torch
    import paper_2001_04321_gb300 as ntf
    dims, r = (40, 30, 20), 5
    T, init, buf, d, ld, Fd = _setup(dims, r, 1e-2, 13)
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(st):
        # 70 iterations: two replays of the 32-iteration graph and 6 eager ones
        F1 = [A.clone() for A in Fd]
        r1 = ntf.solve(buf, F1, ntf.Opts(max_iters=70), dims=d, ld=ld)
        F2 = [A.clone() for A in Fd]
        r2 = ntf.solve(buf, F2, ntf.Opts(max_iters=70, use_graph=True), dims=d, ld=ld)
    assert r1.f_true_last == r2.f_true_last
    assert all(torch.equal(a, b) for a, b in zip(F1, F2))


def test_prepared_graph_with_timing_matches_eager():
    import torch
    import paper_2001_04321_gb300 as ntf
    dims, r = (40, 30, 20), 5
    T, init, buf, d, ld, Fd = _setup(dims, r, 1e-2, 14)
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(st):
        F1 = [A.clone() for A in Fd]
        s1 = ntf.Solver(buf, F1, ntf.Opts(), dims=d, ld=ld)
        s1.run(8)
        s1.get_factors(F1)
        F2 = [A.clone() for A in Fd]
        s2 = ntf.Solver(buf, F2, ntf.Opts(use_graph=True), dims=d, ld=ld)
        s2.run(3)
        s2.set_timing(True)
        s2.prepare_graph(5)
        before = ntf.launch_count()
        s2.run(5)
        ms, n, nbytes = s2.mttkrp_time()
        # 3-way tensor-core path: a stream and an epilogue per mode, 6 launches per iteration
        assert ntf.launch_count() - before >= 5 * 3 * 2
        s2.get_factors(F2)
        st.synchronize()
    assert n == 15 and ms > 0 and nbytes == T.size * 4
    assert all(torch.equal(a, b) for a, b in zip(F1, F2))
    s1.close()
    s2.close()


def test_solver_trajectory_unbalanced_shape():
    # the paper's unbalanced synthetic shape 150 x 1000 x 50 (Sec. 4.1), rank 12
    import paper_2001_04321_gb300 as ntf
    dims, r, iters = (150, 1000, 50), 12, 6
    T, init, buf, d, ld, Fd = _setup(dims, r, 1e-2, 1240)
    fh, rs, rep = _trajectory(buf, d, ld, Fd, iters, ntf.Opts(max_iters=iters))
    _, tr = oracle.solve(T, init, iters, her=True, track_true=True)
    _check_trajectory(fh, rs, tr, oracle.norm_sq(T), 3, f_true=rep.f_true_last, f_true_ref=tr.ftrue[-1])


def test_solver_illconditioned_100cube_her_beats_plain():
    # 100^3, rank 10, shared-base columns (ill-conditioned Grams), 0.1% noise:
    # trajectory parity for the first iterations, then HER ahead of plain HALS
    # after the same number of iterations (the paper's central claim, Sec. 4.2)
    import paper_2001_04321_gb300 as ntf
    w = synth.WORKLOADS["cube100_r10_illcond"]
    dims, r = w["dims"], w["rank"]
    T, init, buf, d, ld, Fd = _setup(dims, r, w["noise_rel"], w["seed"], recipe=w["recipe"])
    fh, rs, rep15 = _trajectory(buf, d, ld, [A.clone() for A in Fd], 15, ntf.Opts(max_iters=15))
    _, tr = oracle.solve(T, init, 15, her=True, track_true=True)
    _check_trajectory(fh, rs, tr, oracle.norm_sq(T), 5, f_true=rep15.f_true_last, f_true_ref=tr.ftrue[-1])
    F_her = [A.clone() for A in Fd]
    rep_her = ntf.solve(buf, F_her, ntf.Opts(max_iters=300), dims=d, ld=ld)
    F_plain = [A.clone() for A in Fd]
    rep_plain = ntf.solve(buf, F_plain, ntf.Opts(her=False, max_iters=300), dims=d, ld=ld)
    assert rep_her.f_true_last < rep_plain.f_true_last
    assert rep_her.restarts > 0


def test_solver_pgd_her_300cube_r32():
    # 300^3, rank 32, PGD + HER: one iteration against the oracle at full size,
    # then 200 iterations whose result is feasible, consistent and lower
    import torch
    import paper_2001_04321_gb300 as ntf
    w = synth.WORKLOADS["cube300_r32"]
    dims, r = w["dims"], w["rank"]
    T, _ = synth.make_tensor(dims, r, w["noise_rel"], seed=w["seed"], recipe=w["recipe"])
    init = synth.make_init(dims, r, seed=0)
    Td = torch.from_numpy(T).cuda()
    opts = ntf.Opts(method="pgd", inner_max=1, her=True, max_iters=1)
    F = [torch.from_numpy(A).cuda() for A in init]
    rep1 = ntf.solve(Td, F, opts)
    Fo, tr = oracle.solve(T, init, 1, her=True, method="pgd", inner_max=1)
    assert rep1.f_hat_last == pytest.approx(tr.fhat[0], rel=1e-5)
    for a, b in zip(F, Fo):
        assert rel_fro(a.cpu().numpy(), b) <= 1e-4
    F = [torch.from_numpy(A).cuda() for A in init]
    rep = ntf.solve(Td, F, ntf.Opts(method="pgd", inner_max=1, her=True, max_iters=200))
    assert np.isfinite(rep.f_true_last) and rep.f_true_last < rep1.f_true_last
    assert all(bool((A >= 0).all()) for A in F)
    assert rep.f_true_last == pytest.approx(ntf.residual_sq(Td, F).item(), rel=1e-6)


@pytest.mark.parametrize("her", [True, False])
def test_solver_trajectory_bf16_tensor_core_path(her):
    # the bf16 (tensor-core, 3-way) fused path against the oracle run on the same
    # bf16-rounded tensor; the MTTKRP's hi/lo factor split rounds at ~2^-17, so F-hat
    # agrees to 1e-5 ||T||^2
    import paper_2001_04321_gb300 as ntf
    dims, r, iters = (60, 50, 40), 6, 30
    T, init, buf, d, ld, Fd = _setup(dims, r, 1e-2, 4321)
    Tq = oracle.bf16_to_f64(oracle.round_bf16(T))
    fh, rs, rep = _trajectory(buf, d, ld, Fd, iters, ntf.Opts(her=her, max_iters=iters, compute_dtype="bf16"))
    Fo, tr = oracle.solve(Tq, init, iters, her=her)
    # the report evaluates the final factors against the FP32 tensor
    _check_trajectory(fh, rs, tr, oracle.norm_sq(Tq), 10, atol_rel=1e-5, f_true=rep.f_true_last,
                      f_true_ref=oracle.objective_explicit(T, Fo))
    if not her:
        assert rs.sum() == 0


def _factors_after(buf, d, ld, Fd, iters, opts):
    import torch
    import paper_2001_04321_gb300 as ntf
    s = ntf.Solver(buf, [A.clone() for A in Fd], opts, dims=d, ld=ld)
    out, rs = [], []
    prev = 0
    for _ in range(iters):
        s.run(1)
        F = [torch.empty_like(A) for A in Fd]
        s.get_factors(F)
        out.append([A.cpu().numpy() for A in F])
        rep = s.report()
        rs.append(rep.restarts - prev)
        prev = rep.restarts
    s.close()
    return out, np.array(rs)


@pytest.mark.parametrize("form", ["f32", "bf16"])
def test_fused_path_factors_elementwise(form):
    # the fused 6-launch path (HALS, extrapolation, Grams and decision inside the epilogues)
    # against the oracle's factors after each of the first 3 iterations, element by element
    import paper_2001_04321_gb300 as ntf
    dims, r, iters = (130, 300, 70), 20, 3
    T, init, buf, d, ld, Fd = _setup(dims, r, 1e-2, 4100)
    Tref = oracle.bf16_to_f64(oracle.round_bf16(T)) if form == "bf16" else T
    got, rs = _factors_after(buf, d, ld, Fd, iters, ntf.Opts(max_iters=iters, compute_dtype=form))
    _, tr = oracle.solve(Tref, init, iters, her=True, track_factors=True)
    np.testing.assert_array_equal(rs, tr.restart)
    # FP32: 3xTF32 products, FP32 sums; bf16: exact tensor, factor split into bf16 hi + lo
    # (2^-17 relative per entry), which HALS carries into small entries
    atol = 2e-5 if form == "f32" else 1e-4
    for k in range(1, iters + 1):
        for l, (a, ref) in enumerate(zip(got[k - 1], tr.A_after(k))):
            assert rel_fro(a, ref) <= 1e-4, (k, l, rel_fro(a, ref))
            np.testing.assert_allclose(a, ref, rtol=2e-3, atol=atol * np.abs(ref).max())


def test_fused_path_two_iterations_at_500cube():
    # the benchmark workload (500^3, rank 20, bf16 storage) for two iterations against the
    # oracle run on the same bf16-rounded tensor: F-hat, decisions and factors
    import torch
    import paper_2001_04321_gb300 as ntf
    w = synth.WORKLOADS["cube500_r20"]
    dims, r = w["dims"], w["rank"]
    T, _ = synth.make_tensor(dims, r, w["noise_rel"], seed=w["seed"], recipe=w["recipe"])
    init = synth.make_init(dims, r, seed=0)
    Td = torch.from_numpy(T).cuda()
    Fd = [torch.from_numpy(A).cuda() for A in init]
    got, rs = _factors_after(Td, list(dims), 0, Fd, 2, ntf.Opts(max_iters=2, compute_dtype="bf16"))
    del Td
    Tq = oracle.bf16_to_f64(oracle.round_bf16(T))
    del T
    _, tr = oracle.solve(Tq, init, 2, her=True, track_factors=True)
    np.testing.assert_array_equal(rs, tr.restart)
    for k in (1, 2):
        for a, ref in zip(got[k - 1], tr.A_after(k)):
            assert rel_fro(a, ref) <= 1e-4


@pytest.mark.parametrize("her", [False, True])
def test_illconditioned_100cube_500_iterations_final_objective(her):
    # the 100^3 ill-conditioned workload: 500 iterations of HALS and of HER-HALS against the
    # oracle from the same initial factors.  This workload fits down to its 0.1% noise: f ends
    # near 1e-6 ||T||^2, ten times the resolution of F-hat (~1e-7 ||T||^2 from FP32 MTTKRPs),
    # so late restart decisions become ties that rounding decides; the check verifies that
    # the first differing decision is such a tie, and bounds the end point by 1e-3 f plus the
    # resolution 1e-6 ||T||^2
    import paper_2001_04321_gb300 as ntf
    w = synth.WORKLOADS["cube100_r10_illcond"]
    dims, r, iters = w["dims"], w["rank"], 500
    T, init, buf, d, ld, Fd = _setup(dims, r, w["noise_rel"], w["seed"], recipe=w["recipe"])
    fh, rs, rep = _trajectory(buf, d, ld, [A.clone() for A in Fd], iters, ntf.Opts(her=her, max_iters=iters))
    _, tr = oracle.solve(T, init, iters, her=her, track_true=True)
    tn = oracle.norm_sq(T)
    k = _check_trajectory(fh, rs, tr, tn, 20, f_true=rep.f_true_last, f_true_ref=tr.ftrue[-1])
    if not her:
        assert k == iters and abs(rep.f_true_last - tr.ftrue[-1]) <= 1e-3 * tr.ftrue[-1]
    assert np.sqrt(rep.f_true_last / tn) <= 1.2e-3


@pytest.mark.parametrize("her", [False, True])
def test_nesterov_solver_trajectory(her):
    # AO-Nesterov blocks with 50 inner steps (the paper's HER-Nesterov50) on a small
    # unbalanced shape, against the oracle
    import paper_2001_04321_gb300 as ntf
    dims, r, iters = (30, 200, 10), 10, 12
    T, init, buf, d, ld, Fd = _setup(dims, r, 1e-2, 4200)
    opts = ntf.Opts(her=her, method="nesterov", inner_max=50, inner_tol=1e-2, max_iters=iters)
    fh, rs, rep = _trajectory(buf, d, ld, Fd, iters, opts)
    _, tr = oracle.solve(T, init, iters, her=her, method="nesterov", inner_max=50, inner_tol=1e-2, track_true=True)
    _check_trajectory(fh, rs, tr, oracle.norm_sq(T), 4, atol_rel=2e-6, f_true=rep.f_true_last,
                      f_true_ref=tr.ftrue[-1])


def test_nesterov_many_rows_path():
    # rows above one CTA run the step-per-launch kernel with the extrapolated point in the
    # workspace: one HER-Nesterov iteration on 2000 x 60 x 40 against the oracle's factors
    import torch
    import paper_2001_04321_gb300 as ntf
    dims, r = (2000, 60, 40), 8
    T, init, buf, d, ld, Fd = _setup(dims, r, 1e-2, 4300)
    F = [A.clone() for A in Fd]
    ntf.solve(buf, F, ntf.Opts(method="nesterov", inner_max=20, inner_tol=0.0, max_iters=1), dims=d, ld=ld)
    Fo, _ = oracle.solve(T, init, 1, method="nesterov", inner_max=20, inner_tol=0.0)
    for a, ref in zip(F, Fo):
        assert rel_fro(a.cpu().numpy(), ref) <= 1e-4


def test_stop_rules_rel_tol_and_max_seconds():
    import paper_2001_04321_gb300 as ntf
    dims, r = (60, 50, 40), 5
    T, init, buf, d, ld, Fd = _setup(dims, r, 1e-2, 4400)
    # the target relative error: stop at the first check (every 5 iterations) that meets it
    full = ntf.solve(buf, [A.clone() for A in Fd], ntf.Opts(max_iters=200), dims=d, ld=ld)
    target = 1.05 * full.rel_error
    rep = ntf.solve(buf, [A.clone() for A in Fd], ntf.Opts(max_iters=200, rel_tol=target, check_every=5),
                    dims=d, ld=ld)
    assert rep.iters < 200 and rep.iters % 5 == 0
    assert np.sqrt(rep.f_hat_last / rep.tnorm_sq) <= target
    # the trajectory up to there is the same as the full run's: one iteration less misses the target
    short = ntf.solve(buf, [A.clone() for A in Fd], ntf.Opts(max_iters=rep.iters - 5), dims=d, ld=ld)
    assert np.sqrt(short.f_hat_last / short.tnorm_sq) > target
    # a wall-time budget already spent stops at the first check
    rep = ntf.solve(buf, [A.clone() for A in Fd], ntf.Opts(max_iters=1000, max_seconds=1e-9, check_every=7),
                    dims=d, ld=ld, )
    assert rep.iters == 7
    with pytest.raises(ntf.NTFError):
        ntf.solve(buf, [A.clone() for A in Fd], ntf.Opts(max_seconds=-1.0), dims=d, ld=ld)


def test_her_parameters_outside_the_papers_ranges_are_rejected():
    # Alg. 2 takes beta0 in (0, 1); eq. HER:relation needs 1 < gamma_bar <= gamma <= eta
    import paper_2001_04321_gb300 as ntf
    dims, r = (12, 10, 8), 3
    T, init, buf, d, ld, Fd = _setup(dims, r, 1e-2, 4500)
    for bad in (dict(beta0=1.0), dict(beta0=0.0), dict(gamma_bar=1.0, gamma=1.0), dict(gamma=2.0, eta=1.5)):
        with pytest.raises(ntf.NTFError):
            ntf.solve(buf, [A.clone() for A in Fd], ntf.Opts(max_iters=1, **bad), dims=d, ld=ld)


@pytest.mark.parametrize("form", ["f32", "bf16"])
def test_reversed_layout_matches_last_mode_kernel(form, monkeypatch):
    # the 3-way tensor-core path streams the last mode's MTTKRP from a second copy of the
    # tensor with its modes reversed (row-stream kernel, running ahead of the epilogue before
    # it); NTF_PERM_LAST=0 keeps the last-mode kernel.  Both agree with the oracle's factors,
    # and with each other.
    import paper_2001_04321_gb300 as ntf
    dims, r, iters = (97, 130, 211), 12, 3
    T, init, buf, d, ld, Fd = _setup(dims, r, 1e-2, 4800)
    Tref = oracle.bf16_to_f64(oracle.round_bf16(T)) if form == "bf16" else T
    _, tr = oracle.solve(Tref, init, iters, her=True, track_factors=True)
    runs = {}
    for flag in ("1", "0"):
        monkeypatch.setenv("NTF_PERM_LAST", flag)
        got, rs = _factors_after(buf, d, ld, Fd, iters, ntf.Opts(max_iters=iters, compute_dtype=form))
        np.testing.assert_array_equal(rs, tr.restart)
        for a, ref in zip(got[-1], tr.A_after(iters)):
            assert rel_fro(a, ref) <= 1e-4
        runs[flag] = got[-1]
    for a, b in zip(runs["1"], runs["0"]):
        assert rel_fro(a, b) <= 1e-4


@pytest.mark.parametrize("form", ["f32", "bf16"])
def test_four_way_merged_pair_path(form, monkeypatch):
    # 4-way tensors with unpadded rows run the tensor-core path on merged-pair views (modes 0, 1
    # against the Khatri-Rao rows of (A_2, A_3); modes 2, 3 on a (I_2, I_3, I_0 I_1) copy against
    # those of (A_hat_0, A_hat_1)).  Factors after 3 iterations against the oracle, a 20-iteration
    # trajectory, and agreement with the generic 4-way path (NTF_DIRECT4=0).
    import paper_2001_04321_gb300 as ntf
    dims, r = (12, 16, 20, 24), 6
    T, init, buf, d, ld, Fd = _setup(dims, r, 1e-2, 4900, recipe="sparse30")
    assert ld == dims[-1]
    Tref = oracle.bf16_to_f64(oracle.round_bf16(T)) if form == "bf16" else T
    _, tr3 = oracle.solve(Tref, init, 3, her=True, track_factors=True)
    runs = {}
    for flag in ("1", "0"):
        monkeypatch.setenv("NTF_DIRECT4", flag)
        got, rs = _factors_after(buf, d, ld, Fd, 3, ntf.Opts(max_iters=3, compute_dtype=form))
        np.testing.assert_array_equal(rs, tr3.restart)
        for a, ref in zip(got[-1], tr3.A_after(3)):
            assert rel_fro(a, ref) <= 1e-4, (flag, rel_fro(a, ref))
        runs[flag] = got[-1]
    for a, b in zip(runs["1"], runs["0"]):
        assert rel_fro(a, b) <= 1e-4
    # the trajectory on uniform factors: with 30% zeroed factor entries both 4-way paths show
    # transient F-hat deviations of 1e-6 to 1e-5 ||T||^2 around iteration 9-12 (measured), the same
    # for this path and the generic one
    monkeypatch.setenv("NTF_DIRECT4", "1")
    iters = 20
    T, init, buf, d, ld, Fd = _setup(dims, r, 1e-2, 4900)
    Tref = oracle.bf16_to_f64(oracle.round_bf16(T)) if form == "bf16" else T
    fh, rs, rep = _trajectory(buf, d, ld, [A.clone() for A in Fd], iters,
                              ntf.Opts(max_iters=iters, compute_dtype=form))
    Fo, tr = oracle.solve(Tref, init, iters, her=True)
    _check_trajectory(fh, rs, tr, oracle.norm_sq(Tref), 8, atol_rel=1e-6 if form == "f32" else 1e-5,
                      f_true=rep.f_true_last, f_true_ref=oracle.objective_explicit(T, Fo))
