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


@pytest.mark.parametrize("nsplit", [2, 3])
@pytest.mark.parametrize("rows,cols,K", [(128, 256, 64), (300, 520, 336), (1, 1, 16), (129, 257, 80),
                                         (256, 512, 4096)])
def test_bf16_split_gemm_matches_fp64_product(G, rows, cols, K, nsplit):
    rng = np.random.default_rng(rows * 7 + cols)
    A = rng.normal(size=(rows, K)).astype(np.float32)
    B = rng.normal(size=(cols, K)).astype(np.float32)
    C = G.test_bf16_gemm(A, B, nsplit)
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    scale = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64).T
    # two planes carry ~16 bits per operand, three ~24; FP32 accumulation adds K * 2^-24
    rep = 2.0 ** -15 if nsplit == 2 else 2.0 ** -21
    bound = scale * (rep + K * 2.0 ** -23) + 1e-6
    err = np.abs(C - ref)
    assert np.all(err <= bound), float((err / bound).max())


def test_three_planes_are_more_accurate_and_long_k_stays_accurate(G):
    """Three planes shrink the operand rounding; long K stays accurate because
    every 256-wide K chunk accumulates in a fresh TMEM buffer and the chunk
    results are summed in FP32 registers."""
    rng = np.random.default_rng(5)
    A = rng.normal(size=(256, 512)).astype(np.float32)
    B = rng.normal(size=(384, 512)).astype(np.float32)
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    e2 = np.abs(G.test_bf16_gemm(A, B, 2) - ref).max()
    e3 = np.abs(G.test_bf16_gemm(A, B, 3) - ref).max()
    assert e3 < e2
    A = rng.normal(size=(128, 16384)).astype(np.float32)
    B = rng.normal(size=(128, 16384)).astype(np.float32)
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    err = np.abs(G.test_bf16_gemm(A, B, 2) - ref) / np.sqrt(16384)
    assert err.max() < 2e-4


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


def test_integer_products_accumulate_exactly(G):
    """BF16 integers |v| <= 128 multiply exactly and their K-sums below 2^24
    accumulate exactly in the FP32 tensor-memory accumulator (the property
    the error-free modular GEMM of the least-squares solve relies on)."""
    rng = np.random.default_rng(8)
    for K, lim in ((256, 128), (1024, 64), (4096, 31)):
        A = rng.integers(-lim, lim + 1, size=(192, K)).astype(np.float32)
        B = rng.integers(-lim, lim + 1, size=(320, K)).astype(np.float32)
        A[0] = lim
        B[0] = lim                                  # one all-maximal dot product
        exact = A.astype(np.int64) @ B.astype(np.int64).T
        C = G.test_bf16_gemm(A, B, 2)
        assert np.array_equal(C.astype(np.int64), exact), K
