"""MTTKRP (step a1) parity: CUDA path vs the FP64 oracle, element by element.

Tolerances: FP32 storage, rel. Frobenius <= 1e-5 against the oracle on the
same FP32 tensor.  BF16 storage: <= 1e-5 against the oracle on the same
bf16-rounded tensor (the kernel reads exact bf16 values and accumulates in
FP32) and <= 2e-2 against the FP32 tensor.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import device_tensor, rel_fro

pytestmark = pytest.mark.gpu

SHAPES = [
    ((37, 23, 19), 5),        # ragged in every mode
    ((20, 20, 20), 5),        # the 20^3 workload shape
    ((64, 128, 64), 16),      # exact tiles
    ((130, 300, 70), 20),     # several tiles per mode + ragged tails
    ((5, 7, 200), 1),         # rank 1, long last mode
    ((3, 4, 5, 6), 7),        # 4-way: two outer modes
    ((6, 5, 4, 3, 33), 12),   # 5-way
    ((40, 50), 9),            # 2-way (NMF)
    ((33, 17, 65), 40),       # rank > 32: two column blocks
    ((9, 300, 33), 64),       # maximum rank
    ((1, 1, 1), 3),           # degenerate
    ((2, 1, 130), 2),
    ((150, 1000, 50), 12),    # the paper's unbalanced synthetic shape (Sec. 4.1)
    ((150, 1000, 50), 25),
    ((50, 50, 50), 10),       # the paper's cube
    ((1, 200, 1), 4),
    ((8, 16, 2048), 16),      # few row tiles, long rows: column segments per row tile
    ((4, 3, 4096), 20),       # ... with ragged rows and the tensor-core rank limit below
    ((6, 40, 1536), 32),
]


def _problem(dims, r, seed):
    T, _ = synth.make_tensor(dims, r, 1e-2, seed=seed)
    F = synth.make_init(dims, r, seed=seed)
    return T, F


@pytest.mark.parametrize("dims,r", SHAPES)
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_mttkrp_matches_oracle(dims, r, dtype):
    import torch
    import paper_2001_04321_gb300 as ntf
    T, F = _problem(dims, r, seed=len(dims) * 100 + r)
    buf, d, ld = device_tensor(T, dtype)
    Fd = [torch.from_numpy(A).cuda() for A in F]
    if dtype == "bf16":
        Tq = oracle.bf16_to_f64(oracle.round_bf16(T))
    for n in range(len(dims)):
        M = ntf.mttkrp(buf, Fd, n, dims=d, ld=ld).cpu().numpy()
        if dtype == "f32":
            assert rel_fro(M, oracle.mttkrp(T, F, n)) <= 1e-5, (dims, r, n)
        else:
            assert rel_fro(M, oracle.mttkrp(Tq, F, n)) <= 1e-5, (dims, r, n)
            assert rel_fro(M, oracle.mttkrp(T, F, n)) <= 2e-2, (dims, r, n)


def test_mttkrp_is_bitwise_reproducible_and_ignores_row_padding():
    import torch
    import paper_2001_04321_gb300 as ntf
    dims, r = (50, 70, 45), 12
    T, F = _problem(dims, r, 5)
    Fd = [torch.from_numpy(A).cuda() for A in F]
    buf, d, ld = device_tensor(T, "f32")
    nan_buf, _, _ = device_tensor(T, "f32", pad_value=float("nan"))   # padding holds NaN
    for n in range(3):
        a = ntf.mttkrp(buf, Fd, n, dims=d, ld=ld).cpu().numpy()
        b = ntf.mttkrp(buf, Fd, n, dims=d, ld=ld).cpu().numpy()
        c = ntf.mttkrp(nan_buf, Fd, n, dims=d, ld=ld).cpu().numpy()
        assert np.array_equal(a, b) and np.array_equal(a, c)


def test_mttkrp_rejects_bad_arguments():
    import torch
    import paper_2001_04321_gb300 as ntf
    T = torch.rand(4, 5, 8, device="cuda")
    F = [torch.rand(4, 3, device="cuda"), torch.rand(5, 3, device="cuda"), torch.rand(8, 3, device="cuda")]
    with pytest.raises(ntf.NTFError) as e:
        ntf.mttkrp(T, F, 3)
    assert e.value.status == 1
    host_F = [F[0], F[1].cpu().contiguous(), F[2]]
    with pytest.raises(ntf.NTFError):
        ntf.mttkrp(T, host_F, 0)                     # host pointer as a factor
    odd = torch.rand(4, 5, 7, device="cuda")         # 28-byte rows: not 16-byte aligned
    with pytest.raises(ntf.NTFError) as e:
        ntf.mttkrp(odd, F[:2] + [torch.rand(7, 3, device="cuda")], 0)
    assert "16 bytes" in str(e.value)
    ws = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(ntf.NTFError) as e:
        ntf.mttkrp(T, F, 0, workspace=ws)
    assert "workspace" in str(e.value)
    ntf.device_status()


def test_fp32_tensor_core_mttkrp_is_unbiased():
    # The tensor core's FP32 accumulation drops about half a unit toward zero when it adds
    # into a large running sum.  The 3xTF32 kernels take each chunk's T_lo steps first, while
    # the sum is small, and keep the mean relative deviation from the oracle near -1e-7 and
    # below 1.5e-7 (T_hi's steps first gave -2.3e-7 in every mode; FFMA about 1e-9).
    import torch
    import paper_2001_04321_gb300 as ntf
    dims, r = (64, 128, 64), 16
    T, F = _problem(dims, r, 2)
    buf, d, ld = device_tensor(T, "f32")
    Fd = [torch.from_numpy(A).cuda() for A in F]
    for n in range(3):
        M = ntf.mttkrp(buf, Fd, n, dims=d, ld=ld).cpu().numpy().astype(np.float64)
        R = oracle.mttkrp(T, F, n)
        assert abs(np.sum(M - R) / np.sum(R)) <= 1.5e-7, n


_CHILD = r"""
import sys, numpy as np, torch
sys.path[:0] = [{root!r}, {tests!r}]
import oracle, synth
import paper_2001_04321_gb300 as ntf
from gpu_helpers import device_tensor, rel_fro
for dims, r in [((37, 23, 19), 5), ((130, 300, 70), 20), ((3, 4, 5, 6), 7)]:
    T, _ = synth.make_tensor(dims, r, 1e-2, seed=r)
    F = synth.make_init(dims, r, seed=r)
    buf, d, ld = device_tensor(T, "f32")
    Fd = [torch.from_numpy(A).cuda() for A in F]
    for n in range(len(dims)):
        M = ntf.mttkrp(buf, Fd, n, dims=d, ld=ld).cpu().numpy()
        e = rel_fro(M, oracle.mttkrp(T, F, n))
        assert e <= 1e-5, (dims, r, n, e)
print("ok")
"""


@pytest.mark.parametrize("mode", ["0", "2"])
def test_fp32_kernel_selection(mode):
    # NTF_TF32=0 (FFMA kernels for every mode) and 2 (tensor cores before the last mode)
    # are read once per process, so each runs in a child process
    import os, subprocess, sys
    here = os.path.dirname(os.path.abspath(__file__))
    code = _CHILD.format(root=os.path.dirname(here), tests=here)
    env = dict(os.environ, NTF_TF32=mode)
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0 and "ok" in out.stdout, out.stderr[-2000:]


@pytest.mark.parametrize("dims,r", [((300, 300, 300), 32), ((200, 330, 250), 20)])
def test_fp32_tensor_core_streams_repeat_exactly(dims, r):
    # The 3xTF32 row streams hand chunks to four MMA warps and take tiles from a run-time
    # counter; every tile writes its own slot, so repeated launches must agree bit for bit,
    # and each must match the oracle.  Ten chunks per row tile in mode 0 (300 columns).
    import torch
    import paper_2001_04321_gb300 as ntf
    T, F = _problem(dims, r, 11)
    buf, d, ld = device_tensor(T, "f32")
    Fd = [torch.from_numpy(A).cuda() for A in F]
    for n in range(len(dims)):
        R = oracle.mttkrp(T, F, n)
        first = ntf.mttkrp(buf, Fd, n, dims=d, ld=ld).cpu().numpy()
        assert rel_fro(first, R) <= 1e-5, (n, rel_fro(first, R))
        for _ in range(8):
            again = ntf.mttkrp(buf, Fd, n, dims=d, ld=ld).cpu().numpy()
            assert np.array_equal(first, again), (n, float(np.max(np.abs(first - again))))
