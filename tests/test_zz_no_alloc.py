"""The allocation-free entry point gap_gp_energy_noalloc, for callers that
cannot allocate device memory while they run (an MD engine that owns every
device buffer, a loop that must not synchronise on cudaMalloc/cudaFree).

Called twice in a row through the C-ABI, its local energies must equal the
local energies gap_predict returns on the FP64 path, within the FP64 parity
tolerance of the other tests (1e-6 eV per atom); its descriptor gradients are
checked against the definition evaluated on the host from the same sparse
points.  Two cells are used: 64 atoms (one 64-row tile of the contraction)
and 216 atoms (several row tiles and a ragged last one).  The device's free
memory is read before and after the calls (after a warm-up call) and must
not change.  This file is collected last so that a failure here stops a `-x`
run only after every other test has run; it also passes on its own."""
import ctypes

import numpy as np
import pytest

from paper_2310_03921_gb300 import synth as S
from _models import oracle_model

pytestmark = pytest.mark.gpu


def test_gp_energy_noalloc_matches_predict_twice():
    import torch

    from paper_2310_03921_gb300 import build, gap
    build.build()
    torch.cuda.set_device(0)
    _, _, sparse, alpha = oracle_model(0, 100)
    w = S.workload(0)
    soap = gap.Soap.from_spec(w.soap)
    model = gap.Model(soap, sparse, alpha, w.delta, w.zeta)
    X, a = np.asarray(sparse[0]), np.asarray(alpha[0])
    L = gap.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    cases = []
    for s in (S.structures(0)[0], S.displaced_diamond(0, 7, (3, 3, 3), 0.1)):
        batch = gap.Batch.from_synth(S.make_batch([s]), device="cuda")
        ref = model.predict(batch, precision="fp64")["local_e"].cpu().numpy()
        phat = soap.descriptor(batch, precision="fp64").contiguous()
        n, D = phat.shape
        q = phat.cpu().numpy() @ X.T
        grad_ref = (w.zeta * w.delta ** 2 * a * q ** (w.zeta - 1)) @ X
        eps = torch.empty((n,), dtype=torch.float64, device="cuda")
        grad = torch.empty((n, D), dtype=torch.float64, device="cuda")
        cases.append((n, D, phat, ref, grad_ref, eps, grad))
    assert [c[0] for c in cases] == [64, 216]

    def call(n, phat, eps, grad):
        return L.gap_gp_energy_noalloc(model.h, 0, n, ctypes.c_void_p(phat.data_ptr()),
                                       ctypes.c_void_p(eps.data_ptr()), ctypes.c_void_p(grad.data_ptr()), stream)

    # warm-up (the first call on a device looks up the scratch address, and
    # the first launch of each kernel loads its module)
    for n, D, phat, _, _, eps, grad in cases:
        eps.fill_(float("nan"))
        grad.fill_(float("nan"))
        assert call(n, phat, eps, grad) == 0, L.gap_last_error()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for rep in range(2):
        for n, D, phat, ref, grad_ref, eps, grad in cases:
            eps.fill_(float("nan"))
            grad.fill_(float("nan"))
            st = call(n, phat, eps, grad)
            assert st == 0, L.gap_last_error()
            torch.cuda.synchronize()
            assert np.abs(eps.cpu().numpy() - ref).max() <= 1e-6, (rep, n)
            assert np.abs(grad.cpu().numpy() - grad_ref).max() <= 1e-9 * max(1.0, np.abs(grad_ref).max()), (rep, n)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0

    # a request beyond the static scratch is rejected, not run
    big = 1 << 20
    n, D, phat, _, _, eps, grad = cases[0]
    st = call(big, phat, eps, grad)
    assert st == -1 and b"static limit" in L.gap_last_error()
