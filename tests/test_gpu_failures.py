"""Failure statuses and hand-written FP64 arithmetic, through the C-ABI.

- GAP_ETIMEOUT: the tcgen05 GEMM's bounded waits are made to run out (a
  producer that issues nothing, a wait limit of microseconds); the call must
  report the expiry and leave the device usable for the next GEMM.
- GAP_ENOMEM: the library's workspace allocations are made to fail on the
  host side; every entry point must return GAP_ENOMEM with a message, and
  the same call must succeed (and give the same result) once allocation is
  restored.
- The FP64 reciprocal and reciprocal square root of the factorisation's
  block kernel (Newton steps from an FP32 estimate, no FP64 division or
  square root) against correctly rounded references over a sweep of
  exponents and mantissas, and beside CUDA's own 1.0 / x and rsqrt(x).
"""
import numpy as np
import pytest

from paper_2310_03921_gb300 import synth as S
from _models import oracle_model

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_2310_03921_gb300 import build, gap
    build.build()
    return gap


def test_tensor_core_wait_expiry_reports_timeout(G):
    st, code = G.test_tc_timeout(20000)  # 20 us per wait
    assert st == -4, G.lib().gap_last_error()
    # the MMA issuer and the epilogue both saw their waits run out
    assert code & 2 and code & 4, code
    assert b"wait expired" in G.lib().gap_last_error()
    # the context is intact: a normal GEMM right after is exact on integers
    rng = np.random.default_rng(5)
    A = rng.integers(-8, 9, size=(200, 64)).astype(np.float32)
    B = rng.integers(-8, 9, size=(300, 64)).astype(np.float32)
    C = G.test_bf16_gemm(A, B)
    assert np.array_equal(C, A @ B.T)


def test_allocation_failure_reports_enomem_and_recovers(G):
    import torch
    _, _, sparse, alpha = oracle_model(0, 100)
    w = S.workload(0)
    soap = G.Soap.from_spec(w.soap)
    model = G.Model(soap, sparse, alpha, w.delta, w.zeta)
    cells = [S.displaced_diamond(0, 31, (2, 2, 2), 0.1), S.displaced_diamond(0, 32, (3, 2, 2), 0.1)]
    batch = G.Batch.from_synth(S.make_batch(cells), device="cuda")
    try:
        for after in (0, 1, 3):
            G.test_fail_alloc(after)
            with pytest.raises(G.GapError) as ei:
                # a layout this model has not seen: its workspaces must grow
                model.predict(G.Batch.from_synth(S.make_batch(cells * (after + 2)), device="cuda"))
            assert ei.value.status == -2
            assert b"failed" in G.lib().gap_last_error()
    finally:
        G.test_fail_alloc(-1)
    torch.cuda.synchronize()
    ref = model.predict(batch, precision="fp64")
    again = model.predict(batch, precision="fp64")
    assert np.array_equal(ref["forces"].cpu().numpy(), again["forces"].cpu().numpy())
    # and the result is the oracle's
    import oracle as O
    soap_o, model_o, _, _ = oracle_model(0, 100)
    Eo, _, Fo, _ = O.predict(soap_o, model_o, cells[1])
    assert np.abs(ref["forces"].cpu().numpy()[cells[0].n:] - Fo).max() <= 1e-6


def _ulps(a, ref):
    """|a - ref| in units of the last place of ref (FP64)."""
    return np.abs(a - ref) / np.spacing(np.abs(ref))


def test_fp64_reciprocal_and_rsqrt_within_one_ulp(G):
    rng = np.random.default_rng(11)
    # every exponent whose reciprocal is a normal number, random mantissas,
    # and the mantissa extremes (1, 2 - ulp) at each exponent
    e = np.arange(-1020, 1021)
    m = rng.uniform(1.0, 2.0, size=e.size)
    x = np.concatenate([np.ldexp(m, e), np.ldexp(1.0, e), np.ldexp(np.nextafter(2.0, 1.0), e),
                        rng.uniform(0.5, 2.0, 4000),  # the equilibrated pivots' range
                        np.ldexp(rng.uniform(1.0, 2.0, 2000), rng.integers(-60, 60, 2000))])
    out = G.test_fp64_recip(x)
    ours_r, ours_s, cuda_r, cuda_s = out.T
    ref_r = 1.0 / x  # IEEE division: correctly rounded
    xl = x.astype(np.longdouble)
    ref_s = (np.longdouble(1) / np.sqrt(xl)).astype(np.float64)
    if np.finfo(np.longdouble).nmant < 60:
        pytest.skip("no extended precision on this host for the rsqrt reference")
    assert np.array_equal(cuda_r, ref_r)  # CUDA's 1.0 / x is IEEE-rounded
    assert _ulps(ours_r, ref_r).max() <= 1.0
    assert _ulps(ours_s, ref_s).max() <= 1.0
    assert _ulps(cuda_s, ref_s).max() <= 2.0
    # mostly correctly rounded
    assert np.mean(ours_r == ref_r) > 0.99
    assert np.mean(ours_s == ref_s) > 0.9
