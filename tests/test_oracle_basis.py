"""Pins of the oracle's building blocks against closed forms and library routines.

Cutoff (Eq. 18), radial basis (reading: Gram-Schmidt of (rc - r)^(k+2)),
modified spherical Bessel functions, real spherical harmonics and the radial
integral of one Gaussian (Eqs. 19-20).
"""
import math

import numpy as np
import pytest
import scipy.special as sp

import oracle as O


def test_fcut_eq18_piecewise():
    rc, d = 5.0, 1.0
    assert O.fcut(0.0, rc, d)[0] == 1.0
    assert O.fcut(3.999, rc, d)[0] == 1.0
    assert O.fcut(5.0, rc, d)[0] == 0.0
    assert O.fcut(7.0, rc, d)[0] == 0.0
    # midpoint of the transition: cos(pi/2) = 0 -> 1/2
    assert O.fcut(4.5, rc, d)[0] == pytest.approx(0.5, abs=1e-15)
    # continuity and derivative by central differences inside the transition
    for r in np.linspace(4.05, 4.95, 7):
        f, df = O.fcut(r, rc, d)
        h = 1e-6
        assert df == pytest.approx((O.fcut(r + h, rc, d)[0] - O.fcut(r - h, rc, d)[0]) / (2 * h), abs=1e-8)
        assert f == pytest.approx(0.5 * (math.cos(math.pi * (r - rc + d) / d) + 1.0), abs=1e-15)


@pytest.mark.parametrize("n_max,rc", [(6, 5.0), (8, 5.0), (10, 4.5)])
def test_radial_basis_orthonormal(n_max, rc):
    soap = O.Soap(n_max, 0, rc, 0.5)
    x, w = np.polynomial.legendre.leggauss(40)   # exact for the degree-26 products
    r = 0.5 * rc * (x + 1)
    w = 0.5 * rc * w
    G = np.array([O.radial_basis(soap, ri) for ri in r])
    S = (G * (w * r * r)[:, None]).T @ G
    assert np.abs(S - np.eye(n_max)).max() < 1e-11


@pytest.mark.parametrize("n_max,rc", [(6, 5.0), (10, 4.5)])
def test_radial_basis_is_gram_schmidt_of_polynomials(n_max, rc):
    """g_n lies in span{(rc-r)^(k+2), k<=n}, is orthogonal to the earlier
    members and has a positive component along (rc-r)^(n+2)."""
    soap = O.Soap(n_max, 0, rc, 0.5)
    x, w = np.polynomial.legendre.leggauss(40)
    r = 0.5 * rc * (x + 1)
    w = 0.5 * rc * w
    G = np.array([O.radial_basis(soap, ri) for ri in r])          # [q][n]
    u = 1.0 - r / rc
    Phi = np.stack([u ** (k + 2) for k in range(1, n_max + 1)], 1)  # scale-free family
    for n in range(n_max):
        overlaps = (Phi[:, :n + 1] * (w * r * r)[:, None]).T @ G[:, n]
        scale = np.sqrt(((G[:, n] ** 2) * w * r * r).sum() * ((Phi[:, :n + 1] ** 2) * (w * r * r)[:, None]).sum(0))
        assert np.all(np.abs(overlaps[:n]) < 1e-10 * scale[:n])
        assert overlaps[n] > 0
        # in the span: least-squares fit by the first n+1 members reproduces g_n on the nodes
        coef, *_ = np.linalg.lstsq(Phi[:, :n + 1], G[:, n], rcond=None)
        assert np.abs(Phi[:, :n + 1] @ coef - G[:, n]).max() < 1e-6 * np.abs(G[:, n]).max()


@pytest.mark.parametrize("x", [1e-3, 0.3, 2.0, 11.0, 60.0])
def test_bessel_closed_forms(x):
    i0 = math.sinh(x) / x
    i1 = (x * math.cosh(x) - math.sinh(x)) / x ** 2
    i2 = ((x * x + 3) * math.sinh(x) - 3 * x * math.cosh(x)) / x ** 3
    for l, ref in [(0, i0), (1, i1), (2, i2)]:
        v, _ = O.bessel_scaled(l, x)
        ref_scaled = ref * math.exp(-x)
        if x >= 0.3:    # the closed forms cancel badly below that
            assert v == pytest.approx(ref_scaled, rel=1e-12)


@pytest.mark.parametrize("x", [0.05, 1.5, 7.0, 40.0, 99.0])
def test_bessel_recurrence_and_derivative(x):
    L = 10
    v = np.array([O.bessel_scaled(l, x)[0] for l in range(L + 2)])
    dv = np.array([O.bessel_scaled(l, x)[1] for l in range(L + 1)])
    # i_{l-1} - i_{l+1} = (2l+1)/x i_l  and  i_l' = i_{l+1} + l/x i_l
    for l in range(1, L + 1):
        assert v[l - 1] - v[l + 1] == pytest.approx((2 * l + 1) / x * v[l], rel=1e-10, abs=1e-300)
        assert dv[l] == pytest.approx(v[l + 1] + l / x * v[l], rel=1e-12, abs=1e-300)
    assert dv[0] == pytest.approx(v[1], rel=1e-12)
    if x > 50:
        assert v[0] == pytest.approx(1.0 / (2 * x), rel=1e-12)   # e^-x sinh(x)/x -> 1/(2x)


def _scipy_real_ylm(L, u):
    """Real Y_lm in the oracle's sign convention from scipy's complex ones."""
    theta = math.acos(max(-1.0, min(1.0, u[2])))
    phi = math.atan2(u[1], u[0])
    out = np.zeros((L + 1) ** 2)
    for l in range(L + 1):
        for m in range(0, l + 1):
            y = complex(sp.sph_harm_y(l, m, theta, phi))
            if m == 0:
                out[l * l + l] = y.real
            else:
                s = math.sqrt(2.0) * (-1) ** m
                out[l * l + l + m] = s * y.real
                out[l * l + l - m] = s * y.imag
    return out


def test_ylm_matches_scipy():
    rng = np.random.default_rng(7)
    for _ in range(20):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        Y, _ = O.ylm(10, u)
        assert np.abs(Y - _scipy_real_ylm(10, u)).max() < 1e-12


def test_ylm_orthonormal_and_addition_theorem():
    L = 8
    ct, wt = np.polynomial.legendre.leggauss(L + 2)
    nphi = 2 * L + 2
    phis = 2 * np.pi * np.arange(nphi) / nphi
    Ys, ws = [], []
    for c, w in zip(ct, wt):
        st = math.sqrt(1 - c * c)
        for ph in phis:
            Ys.append(O.ylm(L, [st * math.cos(ph), st * math.sin(ph), c])[0])
            ws.append(w * 2 * np.pi / nphi)
    Ys, ws = np.array(Ys), np.array(ws)
    assert np.abs((Ys * ws[:, None]).T @ Ys - np.eye((L + 1) ** 2)).max() < 1e-12
    rng = np.random.default_rng(3)
    for _ in range(5):
        a, b = rng.normal(size=3), rng.normal(size=3)
        a /= np.linalg.norm(a)
        b /= np.linalg.norm(b)
        Ya, Yb = O.ylm(L, a)[0], O.ylm(L, b)[0]
        for l in range(L + 1):
            s = slice(l * l, (l + 1) ** 2)
            assert Ya[s] @ Yb[s] == pytest.approx((2 * l + 1) / (4 * np.pi) * sp.eval_legendre(l, a @ b), abs=1e-13)


def test_ylm_at_north_pole_and_gradient():
    L = 8
    Y, _ = O.ylm(L, [0.0, 0.0, 1.0])
    for l in range(L + 1):
        for m in range(-l, l + 1):
            ref = math.sqrt((2 * l + 1) / (4 * math.pi)) if m == 0 else 0.0
            assert Y[l * l + l + m] == pytest.approx(ref, abs=1e-14)
    # gradient of the polynomial extension by central differences
    u = np.array([0.3, -0.5, 0.7])
    _, dY = O.ylm(L, u)
    h = 1e-6
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        fd = (O.ylm(L, u + e)[0] - O.ylm(L, u - e)[0]) / (2 * h)
        assert np.abs(fd - dY[:, a]).max() < 1e-7


@pytest.mark.parametrize("rj", [0.0, 1.3, 2.35, 4.6])
def test_radial_integral_against_direct_quadrature(rj):
    """c_nl0 of one Gaussian on the +z axis (Eqs. 19-20) by direct 2-D
    quadrature in (r, cos t) must equal I_nl(rj) sqrt((2l+1)/4pi)."""
    rc, sig, N, L = 5.0, 0.5, 6, 6
    soap = O.Soap(N, L, rc, sig)
    I, _ = O.radial_integrals(soap, rj)
    xr, wr = np.polynomial.legendre.leggauss(160)
    r = 0.5 * rc * (xr + 1)
    wr = 0.5 * rc * wr
    ct, wc = np.polynomial.legendre.leggauss(120)
    G = np.array([O.radial_basis(soap, ri) for ri in r])
    dist2 = r[:, None] ** 2 + rj ** 2 - 2 * r[:, None] * rj * ct[None, :]
    dens = np.exp(-dist2 / (2 * sig ** 2))                      # [r][ct]
    for l in range(L + 1):
        yl = math.sqrt((2 * l + 1) / (4 * math.pi)) * sp.eval_legendre(l, ct)
        ang = 2 * math.pi * (dens * (wc * yl)[None, :]).sum(1)    # [r]
        c = ((wr * r * r * ang)[:, None] * G).sum(0)              # [n]
        ref = I[:, l] * math.sqrt((2 * l + 1) / (4 * math.pi))
        assert np.abs(c - ref).max() < 1e-10 * max(1.0, np.abs(ref).max())


def test_radial_integral_derivative_and_quadrature_convergence():
    soap = O.Soap(8, 8, 5.0, 0.5)
    soap_fine = O.Soap(8, 8, 5.0, 0.5, quad_n=320)
    for rj in [1.1, 2.4, 3.9, 4.8]:
        I, dI = O.radial_integrals(soap, rj)
        If, _ = O.radial_integrals(soap_fine, rj)
        assert np.abs(I - If).max() < 1e-13 * max(1.0, np.abs(If).max())
        h = 1e-5
        fd = (O.radial_integrals(soap, rj + h)[0] - O.radial_integrals(soap, rj - h)[0]) / (2 * h)
        assert np.abs(fd - dI).max() < 1e-7 * max(1.0, np.abs(dI).max())
