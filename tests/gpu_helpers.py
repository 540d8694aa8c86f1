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


def check_trajectory(fh, rs, tr, tnorm_sq, min_k, atol_rel=1e-6, f_true=None, f_true_ref=None):
    """Trajectory parity of a solver run against the oracle's trace ``tr`` from the same
    initial factors.

    F-hat agrees with the oracle's while every restart decision has matched, to an absolute
    ``atol_rel ||T||^2``: F-hat is a difference of terms of size ||T||^2 formed from FP32
    factors and MTTKRPs, so that is its resolution.  A first differing decision is allowed only
    where the oracle's own margin F_k - F_{k-1} is below what the two sequences resolve
    (2 atol): a tie that rounding decides.  The final objective always agrees within 1e-3
    relative of the oracle's, plus the same resolution ``atol_rel ||T||^2``."""
    atol = atol_rel * tnorm_sq
    same = np.cumprod(np.asarray(rs) == tr.restart).astype(bool)
    k = int(same.sum())
    assert k >= min_k, f"decisions differ from iteration {k + 1}"
    np.testing.assert_allclose(np.asarray(fh)[:k], tr.fhat[:k], rtol=0, atol=atol)
    if k < len(rs):
        prev = tr.fhat[k - 1] if k > 0 else tr.fhat0[0]
        assert abs(tr.fhat[k] - prev) <= 2 * atol, "a restart decision differs away from a tie"
    if f_true is not None:
        assert abs(f_true - f_true_ref) <= 1e-3 * f_true_ref + atol, (f_true, f_true_ref, atol)
    return k


def follow_trajectory(fh, rs, run_oracle, tnorm_sq, atol_rel=1e-6, max_ties=8):
    """Trajectory parity that follows a tie.  ``run_oracle(force)`` runs the oracle with the
    per-iteration forced decisions ``force`` (-1 = Alg. 2's own comparison) and returns
    ``(factors, trace)``.  Wherever the solver decided differently from the oracle, the oracle's own
    margin must be a tie below F-hat's resolution (2 atol, ``atol = atol_rel ||T||^2``); the oracle
    is then rerun taking the solver's branch there, until every decision matches.  Then F-hat
    agrees at every iteration.  Returns ``(factors, trace, ties)`` of the matching oracle run."""
    atol = atol_rel * tnorm_sq
    rs = np.asarray(rs)
    fh = np.asarray(fh)
    force = np.full(len(rs), -1, dtype=np.int32)
    for _ in range(max_ties + 1):
        F, tr = run_oracle(force)
        diff = np.nonzero(rs != tr.restart)[0]
        if diff.size == 0:
            np.testing.assert_allclose(fh, tr.fhat, rtol=0, atol=atol)
            return F, tr, int((force >= 0).sum())
        k = int(diff[0])
        np.testing.assert_allclose(fh[:k], tr.fhat[:k], rtol=0, atol=atol)
        prev = tr.fhat[k - 1] if k > 0 else tr.fhat0[0]
        assert abs(tr.fhat[k] - prev) <= 2 * atol, f"decision {k + 1} differs away from a tie"
        force[k] = rs[k]
    raise AssertionError(f"more than {max_ties} ties")
