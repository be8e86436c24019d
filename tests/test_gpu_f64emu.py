"""The FP64-accurate integer-modular product on the tensor cores (the Gram
matrices and triangular products of the GAP_SOLVE_CHOLQR_TC solve).

Integer-valued inputs make the exact product computable on the host: the
device result must be that product rounded to FP64 (two roundings: the
128-bit integer to FP64 and nothing else).  Real-valued inputs with a wide
dynamic range are checked against exact rational dot products for sampled
entries, with the normwise FP64 bound K 2^-52 max|a_i| max|b_j|."""
import math
from fractions import Fraction

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_2310_03921_gb300 import build, gap
    build.build()
    return gap


def _exact_int_product(A, B):
    """A B^T exactly for integer matrices |entries| < 2^41: 21-bit halves
    multiplied in int64 (partial sums < 2^55), recombined as Python ints."""
    A, B = A.astype(np.int64), B.astype(np.int64)
    A1, A0 = A >> 20, A & (2 ** 20 - 1)
    B1, B0 = B >> 20, B & (2 ** 20 - 1)
    hh, mid, ll = A1 @ B1.T, A1 @ B0.T + A0 @ B1.T, A0 @ B0.T
    out = np.empty(hh.shape)
    for idx in np.ndindex(hh.shape):
        out[idx] = float((int(hh[idx]) << 40) + (int(mid[idx]) << 20) + int(ll[idx]))
    return out


def _ulps(got, exact):
    return np.abs(got - exact) / np.maximum(np.abs(exact), 1e-300) / 2.0 ** -52


@pytest.mark.parametrize("rows,cols,K", [(150, 270, 300), (1, 1, 1), (129, 257, 64), (300, 40, 4097)])
def test_integer_products_are_exact(G, rows, cols, K):
    rng = np.random.default_rng(rows + cols + K)
    A = rng.integers(-2 ** 40, 2 ** 40, size=(rows, K)).astype(np.float64)
    B = rng.integers(-2 ** 40, 2 ** 40, size=(cols, K)).astype(np.float64)
    C = G.test_f64_gemm(A, B)
    assert _ulps(C, _exact_int_product(A, B)).max() <= 2.0


def test_long_inner_dimension_gram_is_exact(G):
    """m = 70000 rows: 274 chunks of 256 accumulate in int32 registers
    (with the periodic reduction modulo p after 64 chunks)."""
    rng = np.random.default_rng(3)
    Y = rng.integers(-2 ** 20, 2 ** 20, size=(70000, 64)).astype(np.int64)
    Gm = G.test_f64_gram(Y.astype(np.float64))
    exact = Y.T @ Y                                   # |entries| < 2^57: exact in int64
    assert np.array_equal(Gm, Gm.T)
    assert _ulps(Gm, exact.astype(np.float64)).max() <= 2.0


def test_gram_with_extreme_residues_is_exact(G):
    """Odd multiples of 128 with a column maximum in [2^52, 2^53) enter the
    product unscaled and have residue +-128 modulo 256, the largest the
    narrow moduli produce: every product in a diagonal entry's K chunks is
    +2^14, the largest chunk sums the FP32 tensor memory has to hold exactly."""
    rng = np.random.default_rng(5)
    Y = 128 * (2 * rng.integers(-2 ** 36, 2 ** 36, size=(2000, 8)) + 1)
    Y[0, :] = 128 * (3 * 2 ** 44 + 1)  # column maxima 3 2^51 + 128
    Gm = G.test_f64_gram(Y.astype(np.float64))
    Yo = Y.astype(object)
    exact = np.array(Yo.T.dot(Yo), dtype=np.float64)
    assert np.array_equal(Gm, Gm.T)
    assert _ulps(Gm, exact).max() <= 2.0


def _exact_dot(a, b):
    return float(sum(Fraction(x) * Fraction(y) for x, y in zip(a, b)))


def test_wide_range_products_meet_the_fp64_bound(G):
    rng = np.random.default_rng(5)
    rows, cols, K = 96, 80, 1000
    A = rng.normal(size=(rows, K)) * 10.0 ** rng.uniform(-6, 6, size=(rows, K))
    B = rng.normal(size=(cols, K)) * 10.0 ** rng.uniform(-6, 6, size=(cols, K))
    C = G.test_f64_gemm(A, B)
    amax, bmax = np.abs(A).max(1), np.abs(B).max(1)
    for i, j in zip(rng.integers(0, rows, 40), rng.integers(0, cols, 40)):
        ex = _exact_dot(A[i], B[j])
        bound = K * 2.0 ** -52 * amax[i] * bmax[j] + 2.0 ** -51 * abs(ex)
        assert abs(C[i, j] - ex) <= bound, (i, j)


def test_triangular_operand_skips_only_zero_blocks(G):
    rng = np.random.default_rng(7)
    n = 700
    A = rng.normal(size=(333, n))
    B = np.tril(rng.normal(size=(n, n)))              # B[j][k] = 0 for k > j
    full = G.test_f64_gemm(A, B)
    tri = G.test_f64_gemm(A, B, b_lower=True)
    assert np.array_equal(full, tri)
    ref = A @ B.T
    scale = np.abs(A).max(1)[:, None] * np.abs(B).max(1)[None, :]
    assert np.all(np.abs(tri - ref) <= n * 2.0 ** -51 * scale + 1e-300)


def test_gram_matches_fp64_and_is_symmetric(G):
    rng = np.random.default_rng(9)
    Y = rng.normal(size=(5000, 300)) * 10.0 ** rng.uniform(-3, 3, size=300)
    Gm = G.test_f64_gram(Y)
    assert np.array_equal(Gm, Gm.T)
    ref = Y.T @ Y
    colmax = np.abs(Y).max(0)
    assert np.all(np.abs(Gm - ref) <= 5000 * 2.0 ** -51 * np.outer(colmax, colmax))


@pytest.mark.parametrize("n", [1, 40, 64, 65, 130, 700, 2000])
def test_recursive_cholesky_and_inverse(G, n):
    """Upper factor R of an SPD matrix and X = R^-1 by the recursive
    factorisation (tensor-core off-diagonal products, FP64 blocks of <= 64)."""
    rng = np.random.default_rng(n)
    A = rng.normal(size=(n + 50, n)) * 10.0 ** rng.uniform(-2, 2, size=n)
    Gm = A.T @ A
    R, X = G.test_chol_inv(Gm)
    assert np.array_equal(np.tril(R, -1), np.zeros((n, n))) and np.array_equal(np.tril(X, -1), np.zeros((n, n)))
    d = np.sqrt(np.diag(Gm))
    # Backward error of the factor, scaled by the diagonal.  The off-diagonal
    # blocks are formed through the inverses of the leading blocks
    # (R12 = R11^-T B), so the bound carries a factor of their conditioning
    # (a Householder/TRSM Cholesky would stay within (n + 1) u).
    assert (np.abs(R.T @ R - Gm) / np.outer(d, d)).max() <= 64 * n * 2.0 ** -53
    R_np = np.linalg.cholesky(Gm).T
    assert (np.abs(R - R_np) / np.abs(np.diag(R_np))[None, :]).max() <= 1e-9
    assert np.abs(R @ X - np.eye(n)).max() <= 1e-10


def test_cholesky_reports_non_positive_definite(G):
    Gm = np.eye(100)
    Gm[70, 70] = -1.0
    with pytest.raises(G.GapError) as e:
        G.test_chol_inv(Gm)
    assert e.value.status == -5


def _nearest_away(q):
    """The FP64 nearest to the exact rational q, ties away from zero (the
    device's rounding of its exact integers)."""
    q = Fraction(q)
    f = float(q)  # nearest, ties to even
    if f != 0.0 and 2 * abs(q - Fraction(f)) == Fraction(math.ulp(f)) and abs(Fraction(f)) < abs(q):
        f = math.copysign(abs(f) + math.ulp(f), f)
    return f


def _round_exact(x, scale=0):
    """_nearest_away of each entry of an object array of integers times 2^-scale."""
    return np.vectorize(lambda v: _nearest_away(Fraction(v, 2 ** scale)), otypes=[np.float64])(x)


@pytest.mark.parametrize("m,n", [(500, 200), (37, 130), (0, 70)])
def test_congruence_of_integer_data_is_exact(G, m, n):
    """W^T (Y^T Y + Kt) W and W^T Y^T b for integer Y, b, Kt, W: every
    fixed-point rounding is exact, so the device values must be the exact
    integers rounded once (compared with Python integer arithmetic)."""
    rng = np.random.default_rng(m + n)
    Y = rng.integers(-2 ** 10, 2 ** 10, size=(m, n)).astype(np.int64)
    b = rng.integers(-2 ** 10, 2 ** 10, size=m).astype(np.int64)
    L = rng.integers(-8, 9, size=(n + 5, n)).astype(np.int64)
    Kt = L.T @ L
    W = np.triu(rng.integers(-2 ** 10, 2 ** 10, size=(n, n))).astype(np.int64)
    np.fill_diagonal(W, rng.integers(1, 2 ** 10, size=n))
    Gd, cd, Wt = G.test_congruence(Y.astype(np.float64), b.astype(np.float64), Kt.astype(np.float64),
                                   W.astype(np.float64))
    assert np.array_equal(Wt, W.astype(np.float64))
    G1 = (Y.T @ Y + Kt).astype(object)
    Wo = W.astype(object)
    exact = Wo.T.dot(G1).dot(Wo)
    assert np.array_equal(Gd, _round_exact(exact))
    cex = Wo.T.dot((Y.T @ b).astype(object))
    assert np.array_equal(cd, _round_exact(cex))


def _to_int_scaled(A, s):
    """Exact integers A 2^s of an FP64 array (s large enough)."""
    out = np.empty(A.shape, dtype=object)
    for idx in np.ndindex(A.shape):
        num, den = Fraction(float(A[idx])).as_integer_ratio()
        v = Fraction(num, den) * (Fraction(2) ** s)
        assert v.denominator == 1
        out[idx] = v.numerator
    return out


def test_congruence_of_ill_conditioned_system_is_correctly_rounded(G):
    """The shapes of a fit: Y with column scales over 10^8, Kt positive
    definite, W the inverse Cholesky factor of the shifted Gram matrix (full
    53-bit entries, rounded by the device to the W~ it returns).  Y, b and
    Kt carry 30-bit significands, so that V's fixed-point grid holds them
    exactly; the reference is W~^T (Y^T Y + Kt) W~ in rational arithmetic."""
    rng = np.random.default_rng(11)
    m, n = 300, 48
    def short(x):
        e = np.floor(np.log2(np.abs(x) + 1e-300))
        return np.ldexp(np.round(np.ldexp(x, (29 - e).astype(int))), (e - 29).astype(int))
    Y = short(rng.normal(size=(m, n)) * 10.0 ** rng.uniform(-4, 4, size=n))
    b = short(rng.normal(size=m) * 1e3)
    A = rng.normal(size=(n, n)) * 1e-3
    Kt = short(A.T @ A + 1e-6 * np.eye(n))
    Kt = np.triu(Kt) + np.triu(Kt, 1).T
    Gm = Y.T @ Y + Kt
    Rc = np.linalg.cholesky(Gm + 1e-10 * np.trace(Gm) * np.eye(n)).T
    W = np.triu(np.linalg.inv(Rc))
    Gd, cd, Wt = G.test_congruence(Y, b, Kt, W)
    # W~ is W rounded in the metric of V's column scales d_k (53 bits below
    # the largest |W_ki| d_k of each column; d_k within a factor 2 of it)
    d = np.maximum(np.abs(Y).max(0), np.sqrt(np.diag(Kt)))[:, None]
    assert (np.abs(Wt - W) * d <= 2.0 ** -51 * (np.abs(W) * d).max(0)[None, :]).all()
    s = 1200
    Yi, bi, Ki = _to_int_scaled(Y, 64), _to_int_scaled(b, 64), _to_int_scaled(Kt, 128)
    Wi = _to_int_scaled(Wt, s)
    G1 = Yi.T.dot(Yi) + Ki                     # exact, scaled 2^128
    ex = Wi.T.dot(G1).dot(Wi)                 # scaled 2^(128 + 2 s)
    cex = Wi.T.dot(Yi.T.dot(bi))              # scaled 2^(128 + s)
    ref = _round_exact(ex, 128 + 2 * s)
    cref = _round_exact(cex, 128 + s)
    assert np.array_equal(Gd, ref)
    assert np.array_equal(cd, cref)
