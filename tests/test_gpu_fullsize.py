"""Parity at the benchmark's full sizes, in the launch configuration the
benchmark times (the solver's own MTTKRP plans): sampled output rows that the
oracle computes one by one from the tensor slab of that row."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import rel_fro

pytestmark = pytest.mark.gpu

WORKLOADS = ["cube500_r20", "hyper80_r16_sparse30", "cube300_r32"]


def _slab_row(T, F, n, j):
    """MTTKRP row j of mode n by the oracle on the slab T[..., j, ...]."""
    sl = [slice(None)] * T.ndim
    sl[n] = slice(j, j + 1)
    Ts = np.ascontiguousarray(T[tuple(sl)])
    Fs = list(F)
    Fs[n] = F[n][j:j + 1]
    return oracle.mttkrp(Ts, Fs, n)[0]


@pytest.mark.parametrize("name", WORKLOADS)
def test_fullsize_sampled_rows(name):
    import torch
    import paper_2001_04321_gb300 as ntf
    w = synth.WORKLOADS[name]
    dims, r = w["dims"], w["rank"]
    T, _ = synth.make_tensor(dims, r, w["noise_rel"], seed=w["seed"], recipe=w["recipe"])
    F = synth.make_init(dims, r, seed=0)
    Td = torch.from_numpy(T).cuda()
    Fd = [torch.from_numpy(A).cuda() for A in F]
    bf, d, ldb = ntf.to_bf16(Td)
    Tq = None
    rng = np.random.default_rng(0)
    for n in range(len(dims)):
        M32 = ntf.mttkrp(Td, Fd, n).cpu().numpy()
        M16 = ntf.mttkrp(bf, Fd, n, dims=d, ld=ldb).cpu().numpy()
        rows = sorted(set([0, dims[n] - 1] + list(rng.integers(0, dims[n], 4))))
        for j in rows:
            ref = _slab_row(T, F, n, j)
            assert rel_fro(M32[j], ref) <= 1e-5, (name, n, j)
            assert rel_fro(M16[j], ref) <= 2e-2, (name, n, j)
        # rows of the bf16 form against the oracle on the same bf16-rounded slab
        j = rows[len(rows) // 2]
        sl = [slice(None)] * T.ndim
        sl[n] = slice(j, j + 1)
        slab_q = oracle.bf16_to_f64(oracle.round_bf16(np.ascontiguousarray(T[tuple(sl)])))
        Fs = list(F)
        Fs[n] = F[n][j:j + 1]
        assert rel_fro(M16[j], oracle.mttkrp(slab_q, Fs, n)[0]) <= 1e-5
        # every output is finite and nonnegative (nonnegative data and factors)
        assert np.all(np.isfinite(M32)) and np.all(M32 >= 0)
    ntf.device_status()


def test_fullsize_one_iteration_objective_matches_explicit():
    # after one HER iteration on 500^3 the F-hat reuse identity and the explicit
    # residual are consistent with each other and with the oracle on a sample
    import torch
    import paper_2001_04321_gb300 as ntf
    w = synth.WORKLOADS["cube500_r20"]
    T, _ = synth.make_tensor(w["dims"], w["rank"], w["noise_rel"], seed=w["seed"])
    F = synth.make_init(w["dims"], w["rank"], seed=0)
    Td = torch.from_numpy(T).cuda()
    Fd = [torch.from_numpy(A).cuda() for A in F]
    s = ntf.Solver(Td, Fd, ntf.Opts(her=False))
    s.run(1)
    rep = s.report()
    s.get_factors(Fd)
    # without extrapolation F-hat is F at the current factors
    assert rep.f_hat_last == pytest.approx(rep.f_true_last, rel=1e-3)
    Fh = [A.cpu().numpy() for A in Fd]
    # explicit residual of slab 0 by the oracle vs the library residual of that slab
    slab = np.ascontiguousarray(T[:1])
    ref = oracle.objective_explicit(slab, [Fh[0][:1], Fh[1], Fh[2]])
    got = ntf.residual_sq(torch.from_numpy(slab).cuda(), [torch.from_numpy(Fh[0][:1]).cuda(), Fd[1], Fd[2]]).item()
    assert got == pytest.approx(ref, rel=1e-4)
    s.close()
