"""The sharded form of the path, simulated on one GPU: the tensor is split into
P slabs along mode 0 and every slab runs through the C ABI on its own, as a
rank would.  Mode-0 MTTKRP rows are local to their slab; for every other mode
the slabs' MTTKRPs are partial sums whose plain sum (the all-reduce of
I_n x r floats) must equal the unsharded MTTKRP; ||T||^2 and the Gram of the
sharded factor are likewise sums over slabs.  This is the exchange a
multi-GPU run would make; the benchmark itself runs replicas."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import rel_fro

pytestmark = pytest.mark.gpu


def _bounds(I0, P):
    return [(I0 * s) // P for s in range(P + 1)]


@pytest.mark.parametrize("dims,r,P", [((24, 20, 16), 5, 2), ((37, 12, 8, 16), 7, 3), ((150, 100, 48), 20, 4)])
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_slab_partials_sum_to_unsharded(dims, r, P, dtype):
    import torch
    import paper_2001_04321_gb300 as ntf
    T, _ = synth.make_tensor(dims, r, 1e-2, seed=sum(dims) + P)
    F = synth.make_init(dims, r, seed=P)
    Td = torch.from_numpy(T).cuda()
    Fd = [torch.from_numpy(A).cuda() for A in F]
    if dtype == "bf16":
        full, d, ld = ntf.to_bf16(Td)
        Tref = oracle.bf16_to_f64(oracle.round_bf16(T))
    else:
        full, d, ld = Td.reshape(-1), list(dims), dims[-1]
        Tref = T.astype(np.float64)
    slab_elems = int(np.prod(dims[1:-1])) * ld        # storage elements per mode-0 index
    b = _bounds(dims[0], P)
    for n in range(len(dims)):
        ref = ntf.mttkrp(full, Fd, n, dims=d, ld=ld).cpu().numpy()
        parts = []
        for s in range(P):
            view = full[b[s] * slab_elems:b[s + 1] * slab_elems]
            sd = [b[s + 1] - b[s]] + list(dims[1:])
            Fs = [Fd[0][b[s]:b[s + 1]].contiguous()] + Fd[1:]
            parts.append(ntf.mttkrp(view, Fs, n, dims=sd, ld=ld).cpu().numpy())
        if n == 0:
            got = np.concatenate(parts, axis=0)
            assert np.array_equal(got.shape, ref.shape)
        else:
            got = np.sum(parts, axis=0)
        assert rel_fro(got, ref) <= 1e-5, (n, dtype)
        assert rel_fro(got, oracle.mttkrp(Tref, F, n)) <= 1e-5, (n, dtype)
    # ||T||^2 and the Gram of the sharded factor as sums over slabs
    tn = sum(ntf.tensor_norm_sq(full[b[s] * slab_elems:b[s + 1] * slab_elems],
                                dims=[b[s + 1] - b[s]] + list(dims[1:]), ld=ld).item() for s in range(P))
    assert tn == pytest.approx(oracle.norm_sq(Tref), rel=1e-6)
    G0 = sum(ntf.gram(Fd[0][b[s]:b[s + 1]].contiguous()).cpu().numpy() for s in range(P))
    assert rel_fro(G0, oracle.gram(F[0])) <= 1e-6
