"""Helpers shared by the GPU tests (no method arithmetic here)."""
import numpy as np


def rel_fro(x, ref):
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(x - ref) / (den if den > 0 else 1.0))


def device_tensor(T, dtype="f32", pad_value=0.0):
    """Place a C-order numpy tensor on cuda:0 with 16-byte last-mode rows.

    Returns (buffer, dims, ld).  For "bf16" the library's own cast is used
    (step a8); the oracle side rounds independently with oracle.round_bf16.
    """
    import torch
    import paper_2001_04321_gb300 as ntf
    dims = list(T.shape)
    C = dims[-1]
    ld = -(-C // 4) * 4
    rows = int(np.prod(dims[:-1]))
    host = np.full((rows, ld), pad_value, dtype=np.float32)
    host[:, :C] = np.asarray(T, dtype=np.float32).reshape(rows, C)
    buf = torch.from_numpy(host).cuda()
    if dtype == "f32":
        return buf, dims, ld
    import ctypes as Cc
    d = ntf._tensor_desc(buf, dims, ld)
    ldb = int(ntf.load().ntf_bf16_ld(Cc.byref(d)))
    out = torch.empty(rows * ldb, dtype=torch.bfloat16, device="cuda")
    ntf._check(ntf.load().ntf_tensor_to_bf16(Cc.byref(d), ntf._ptr(out), ldb, ntf._stream(None)))
    return out, dims, ldb
