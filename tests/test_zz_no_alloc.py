"""ntf_mttkrp_noalloc: the allocation-free MTTKRP entry point (for callers that
cannot allocate device memory) must give the workspace entry point's result.

Kept in a file that pytest collects last, so a run that stops at the first
failure has already run every other test.  Calls go through the C ABI
directly (ctypes), two rounds of calls in a row on different problems
(including the FP32 last mode, whose tensor-core kernel uses other scratch
offsets), compared with ntf_mttkrp and with the FP64 oracle within the MTTKRP
tolerance of the other tests (rel. Frobenius <= 1e-5)."""
import ctypes as C

import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import device_tensor, rel_fro

pytestmark = pytest.mark.gpu


def _noalloc(buf, dims, ld, factors, mode):
    import torch
    import paper_2001_04321_gb300 as ntf
    L = ntf.load()
    d = ntf._tensor_desc(buf, dims, ld)
    rank = int(factors[0 if mode != 0 else 1].shape[1])
    out = torch.full((dims[mode], rank), float("nan"), dtype=torch.float32, device="cuda")
    ptrs = ntf._ptr_array([None if l == mode else A for l, A in enumerate(factors)])
    st = L.ntf_mttkrp_noalloc(C.byref(d), ptrs, rank, mode, ntf._ptr(out), ntf._stream(None))
    return st, out


def test_noalloc_matches_workspace_entry_on_two_calls_in_a_row():
    import torch
    import paper_2001_04321_gb300 as ntf
    probs = []
    for dims, r, dtype, seed in [((130, 300, 70), 20, "f32", 1), ((60, 50, 40, 9), 7, "bf16", 2),
                                 ((96, 120, 200), 16, "f32", 3)]:
        T, _ = synth.make_tensor(dims, r, 1e-2, seed=seed)
        init = synth.make_init(dims, r, seed=seed)
        F = [torch.from_numpy(A).cuda() for A in init]
        buf, d, ld = device_tensor(T, dtype)
        Tref = oracle.bf16_to_f64(oracle.round_bf16(T)) if dtype == "bf16" else T
        probs.append((buf, d, ld, F, Tref, init))
    # the shared scratch keeps the last call's contents; the third problem's mode is the
    # FP32 tensor's last mode in both rounds
    for modes in ((0, 3, 2), (1, 2, 2)):
        outs = []
        for (buf, d, ld, F, Tref, init), mode in zip(probs, modes):
            st, out = _noalloc(buf, d, ld, F, mode)
            assert st == 0, ntf.load().ntf_last_error()
            outs.append((out, buf, d, ld, F, mode, Tref, init))
        torch.cuda.synchronize()
        for out, buf, d, ld, F, mode, Tref, init in outs:
            got = out.cpu().numpy()
            ref = ntf.mttkrp(buf, F, mode, dims=d, ld=ld)
            assert rel_fro(got, ref.cpu().numpy()) <= 1e-5
            assert rel_fro(got, oracle.mttkrp(Tref, init, mode)) <= 1e-5
    ntf.device_status()


def test_noalloc_rejects_requests_beyond_its_scratch():
    import torch
    import paper_2001_04321_gb300 as ntf
    dims, r, mode = (8, 8192, 4), 64, 1
    T = torch.rand(*dims, device="cuda")
    F = [torch.rand(n, r, device="cuda") for n in dims]
    assert ntf.mttkrp_workspace_bytes(T, r, mode) > (16 << 20)
    st, out = _noalloc(T, list(dims), 0, F, mode)
    assert st == 1
    assert b"fixed scratch" in ntf.load().ntf_last_error()
    assert torch.isnan(out).all()             # nothing was launched
    ntf.device_status()
