"""GPU checks of single kernels through the C-ABI: the split-precision
tcgen05 GEMM against an FP64 product, and the radial-integral table against
the oracle's quadrature."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_2310_03921_gb300 import build, gap
    build.build()
    return gap


@pytest.mark.parametrize("rows,cols,K", [(128, 256, 64), (300, 520, 336), (1, 1, 16), (129, 257, 80),
                                         (256, 512, 4096)])
def test_bf16x3_gemm_matches_fp64_product(G, rows, cols, K):
    rng = np.random.default_rng(rows * 7 + cols)
    A = rng.normal(size=(rows, K)).astype(np.float32)
    B = rng.normal(size=(cols, K)).astype(np.float32)
    C = G.test_bf16x3_gemm(A, B)
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    scale = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64).T
    # hi+lo carries ~16 bits per operand; FP32 accumulation adds K * 2^-24
    bound = scale * (2.0 ** -15 + K * 2.0 ** -23) + 1e-6
    err = np.abs(C - ref)
    assert np.all(err <= bound), float((err / bound).max())


def test_radial_table_matches_oracle_integrals(G):
    for (n, l, rc, sig) in [(6, 4, 5.0, 0.5), (10, 8, 4.5, 0.5), (8, 8, 5.0, 0.5)]:
        soap = G.Soap(n, l, rc, sig)
        tab = soap.radial_table()
        osoap = O.Soap(n, l, rc, sig)
        G_ = tab.shape[0] - 1
        for k in [0, 1, 37, 600, 1333, 2047, G_]:
            r = k * rc / G_
            I, dI = O.radial_integrals(osoap, r)
            scale = max(1.0, np.abs(I).max())
            assert np.abs(tab[k, :, :, 0] - I).max() < 1e-11 * scale
            assert np.abs(tab[k, :, :, 1] - dI).max() < 1e-10 * max(1.0, np.abs(dI).max())
