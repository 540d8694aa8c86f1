"""A tensor kept in host memory and streamed to the device by slabs of mode 0
(the paper's remark in Sec. 4 on data sets too large for its implementation's
memory): MTTKRP, norm and the HER solver against the in-HBM path and the oracle."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import check_trajectory, device_tensor, rel_fro

pytestmark = pytest.mark.gpu


def _host(T):
    import torch
    return torch.from_numpy(np.ascontiguousarray(T, dtype=np.float32)).pin_memory()


@pytest.mark.parametrize("dims,r,slab", [
    ((37, 20, 16), 5, 4),          # ragged last slab (37 = 9 x 4 + 1)
    ((37, 20, 16), 5, 1),          # one mode-0 index per slab
    ((37, 20, 16), 5, 100),        # one slab
    ((12, 9, 10, 8), 4, 5),        # 4-way
    ((50, 24), 6, 7),              # matrix
    ((64, 96, 128), 20, 16),       # tensor-core rank
])
def test_streamed_mttkrp_matches_in_hbm_and_oracle(dims, r, slab):
    import torch
    import paper_2001_04321_gb300 as ntf
    T, _ = synth.make_tensor(dims, r, 1e-2, seed=sum(dims) + slab)
    F = synth.make_init(dims, r, seed=slab)
    Fd = [torch.from_numpy(A).cuda() for A in F]
    Th = _host(T)
    Td = torch.from_numpy(T).cuda()
    for n in range(len(dims)):
        got = ntf.mttkrp_streamed(Th, Fd, n, slab_rows=slab).cpu().numpy()
        ref = oracle.mttkrp(T, F, n)
        assert rel_fro(got, ref) <= 1e-5, (n, rel_fro(got, ref))
        assert rel_fro(got, ntf.mttkrp(Td, Fd, n).cpu().numpy()) <= 1e-5
    # bitwise reproducible (fixed slab order)
    a = ntf.mttkrp_streamed(Th, Fd, len(dims) - 1, slab_rows=slab)
    b = ntf.mttkrp_streamed(Th, Fd, len(dims) - 1, slab_rows=slab)
    assert torch.equal(a, b)


def test_streamed_rejects_device_memory():
    import torch
    import paper_2001_04321_gb300 as ntf
    Td = torch.zeros((8, 8, 8), device="cuda")
    import ctypes as C
    d = ntf._tensor_desc(Td)
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    ptrs = ntf._ptr_array([None, Td, Td])
    st = ntf.load().ntf_mttkrp_streamed(C.byref(d), ptrs, 2, 0, ntf._ptr(Td), ntf._ptr(ws), ws.numel(), 2,
                                        ntf._stream(None))
    assert st == 1 and b"host memory" in ntf.load().ntf_last_error()


@pytest.mark.parametrize("her", [True, False])
def test_streamed_solver_trajectory(her):
    import torch
    import paper_2001_04321_gb300 as ntf
    dims, r, iters = (45, 30, 20), 5, 25
    T, _ = synth.make_tensor(dims, r, 1e-2, seed=4600)
    init = synth.make_init(dims, r, seed=4600)
    s = ntf.Solver.streamed(_host(T), [torch.from_numpy(A).cuda() for A in init], ntf.Opts(her=her, max_iters=iters),
                            slab_rows=8)
    fh, rs, prev = [], [], 0
    for _ in range(iters):
        s.run(1)
        rep = s.report()
        fh.append(rep.f_hat_last)
        rs.append(rep.restarts - prev)
        prev = rep.restarts
    s.close()
    _, tr = oracle.solve(T, init, iters, her=her, track_true=True)
    tn = oracle.norm_sq(T)
    check_trajectory(fh, rs, tr, tn, 8, f_true=rep.f_true_last, f_true_ref=tr.ftrue[-1])
    assert rep.tnorm_sq == pytest.approx(tn, rel=1e-6)


def test_solve_streamed_matches_in_hbm_solve():
    import torch
    import paper_2001_04321_gb300 as ntf
    dims, r = (80, 60, 40), 8
    T, _ = synth.make_tensor(dims, r, 1e-2, seed=4700)
    init = synth.make_init(dims, r, seed=4700)
    Fs = [torch.from_numpy(A).cuda() for A in init]
    rs = ntf.solve_streamed(_host(T), Fs, ntf.Opts(max_iters=20), slab_rows=11)
    buf, d, ld = device_tensor(T)
    Fd = [torch.from_numpy(A).cuda() for A in init]
    rd = ntf.solve(buf, Fd, ntf.Opts(max_iters=20), dims=d, ld=ld)
    assert rs.f_true_last == pytest.approx(rd.f_true_last, rel=1e-3)
    assert rs.rel_error == pytest.approx(rd.rel_error, rel=1e-3)
