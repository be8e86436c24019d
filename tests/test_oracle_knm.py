"""Pins of the oracle's K_NM rows (text after Eq. 4) and of the regularised
least-squares solve (Eq. 4 against Eqs. 5-9)."""
import numpy as np
import pytest

import oracle as O
from paper_2310_03921_gb300 import synth as S
from _models import oracle_model


@pytest.fixture(scope="module")
def small():
    soap, model, sparse, alpha = oracle_model(0, 40)
    return soap, model, S.displaced_diamond(0, 77, (1, 1, 2), 0.12)


def test_knm_times_alpha_reproduces_predict(small):
    """K_E alpha = E and K_F alpha = F: the rows hold k and -dk/dr."""
    soap, model, s = small
    K = O.knm(soap, model, s)
    E, _, F, _ = O.predict(soap, model, s)
    assert K.shape == (1 + 3 * s.n, 40)
    assert K[0] @ model.alpha == pytest.approx(E, abs=1e-11)
    assert np.abs((K[1:] @ model.alpha).reshape(-1, 3) - F).max() < 1e-11


def test_knm_column_by_finite_differences(small):
    """Column m: E_m(r) = sum_i delta^2 (p_hat_i . x_m)^zeta from the descriptor
    alone; its energy row entry and -dE_m/dr_ja by central differences."""
    soap, model, s = small
    K = O.knm(soap, model, s)
    m = 7
    x = model.sparse[m]
    d2, z = model.c.delta ** 2, model.c.zeta

    def Em(st):
        return d2 * ((O.descriptor(soap, st)[0] @ x) ** z).sum()

    assert K[0, m] == pytest.approx(Em(s), abs=1e-12)
    h = 1e-4
    for a, c in [(0, 0), (5, 2), (15, 1)]:
        sp, sm = (S.Structure(s.pos.copy(), s.species, s.cell, s.pbc) for _ in range(2))
        sp.pos[a, c] += h
        sm.pos[a, c] -= h
        fd = -(Em(sp) - Em(sm)) / (2 * h)
        assert K[1 + 3 * a + c, m] == pytest.approx(fd, abs=1e-7)


def test_knm_multispecies_block_structure():
    soap, model, sparse, alpha = oracle_model(3, 6, n_max=3, l_max=2, n_cells=2)
    s = S.structures(3, 1)[0]
    K = O.knm(soap, model, s)
    E, _, F, _ = O.predict(soap, model, s)
    assert K[0] @ model.alpha == pytest.approx(E, abs=1e-10)
    assert np.abs((K[1:] @ model.alpha).reshape(-1, 3) - F).max() < 1e-10
    offs = model.offsets
    for sp in range(4):
        cols = slice(offs[sp], offs[sp + 1])
        if not np.any(s.species == sp):
            assert np.abs(K[:, cols]).max() == 0.0


def test_kmm_symmetric_psd(small):
    soap, model, _ = small
    Kmm = O.kmm(model, soap.dim)
    assert np.abs(Kmm - Kmm.T).max() < 1e-14
    assert np.allclose(np.diag(Kmm), model.c.delta ** 2)   # normalised descriptors: k(x, x) = delta^2
    assert np.linalg.eigvalsh(Kmm).min() > -1e-10


def test_qr_solution_equals_normal_equations():
    rng = np.random.default_rng(4)
    R, M = 80, 12
    K = rng.normal(size=(R, M))
    y = rng.normal(size=R)
    sig = rng.uniform(0.05, 0.5, size=R)
    B = rng.normal(size=(M, M))
    Kmm = B @ B.T + 0.5 * np.eye(M)
    c1 = O.solve_normal(K, y, sig, Kmm, 1e-8)
    c2 = O.solve_qr(K, y, sig, Kmm, 1e-8)
    assert np.abs(c1 - c2).max() < 1e-10 * np.abs(c1).max()
    # and both satisfy the stationarity condition of Eq. 4
    W = 1.0 / sig ** 2
    resid = (Kmm + 1e-8 * np.eye(M) + (K * W[:, None]).T @ K) @ c1 - (K * W[:, None]).T @ y
    assert np.abs(resid).max() < 1e-9


def test_teacher_student_fit():
    """Targets from a teacher alpha*: the fitted model reproduces teacher
    energies and forces on held-out cells to well within sigma."""
    soap, model, sparse, alpha = oracle_model(0, 30)
    teacher = model
    cells = [S.displaced_diamond(0, 500 + c, (1, 1, 2), 0.1) for c in range(3)]
    Ks, ys, sig = [], [], []
    for s in cells:
        K = O.knm(soap, teacher, s)
        E, _, F, _ = O.predict(soap, teacher, s)
        Ks.append(K)
        ys.append(np.concatenate([[E], F.reshape(-1)]))
        sig.append(np.concatenate([[1e-3 * np.sqrt(s.n)], np.full(3 * s.n, 1e-2)]))
    K, y, sg = np.concatenate(Ks), np.concatenate(ys), np.concatenate(sig)
    c = O.solve_qr(K, y, sg, O.kmm(teacher, soap.dim), 1e-8)
    student = O.Model(sparse, [c], teacher.c.delta, teacher.c.zeta)
    held = S.displaced_diamond(0, 600, (1, 1, 2), 0.1)
    Et, _, Ft, _ = O.predict(soap, teacher, held)
    Es, _, Fs, _ = O.predict(soap, student, held)
    assert abs(Es - Et) < 1e-2
    assert np.abs(Fs - Ft).max() < 1e-2


@pytest.mark.parametrize("zeta", [2, 3, 4])
def test_kernel_exponent_by_homogeneity(small, zeta):
    """The dot-product kernel delta^2 (p_hat . x)^zeta (Eqs. 2, 13) is
    homogeneous of degree zeta in the sparse point: scaling one sparse point
    by c scales its energy row entry, its force row entries, and the local
    energies and forces of a model whose only nonzero coefficient is that
    point's, by c^zeta, and row and column m of K_MM likewise.  An exponent
    slip anywhere (zeta - 1 or zeta + 1 in gp_eval, the K_NM rows or K_MM)
    changes the ratio from c^zeta."""
    soap, _, s = small
    _, _, sparse, alpha = oracle_model(0, 40)
    X = np.array(sparse[0])
    m, c = 5, 1.7
    a = np.zeros(X.shape[0])
    a[m] = 0.3
    X2 = X.copy()
    X2[m] *= c
    d = 1.3
    mod1, mod2 = O.Model([X], [a], d, zeta), O.Model([X2], [a], d, zeta)
    K1, K2 = O.knm(soap, mod1, s), O.knm(soap, mod2, s)
    cz = c ** zeta
    assert np.abs(K2[:, m] - cz * K1[:, m]).max() <= 1e-12 * np.abs(K1[:, m]).max() * cz
    others = np.arange(X.shape[0]) != m
    assert np.array_equal(K2[:, others], K1[:, others])
    E1, le1, F1, V1 = O.predict(soap, mod1, s)
    E2, le2, F2, V2 = O.predict(soap, mod2, s)
    assert E2 == pytest.approx(cz * E1, rel=1e-12)
    assert np.abs(le2 - cz * le1).max() <= 1e-12 * cz * np.abs(le1).max()
    assert np.abs(F2 - cz * F1).max() <= 1e-12 * cz * np.abs(F1).max()
    assert np.abs(V2 - cz * V1).max() <= 1e-12 * cz * np.abs(V1).max()
    # and the prefactor enters squared: delta -> 2 delta scales everything by 4
    E3 = O.predict(soap, O.Model([X], [a], 2 * d, zeta), s)[0]
    assert E3 == pytest.approx(4 * E1, rel=1e-13)
    # K_MM: row and column m scale by c^zeta, the diagonal entry by c^(2 zeta)
    D = X.shape[1]
    M1, M2 = O.kmm(mod1, D), O.kmm(mod2, D)
    scale = np.ones(X.shape[0])
    scale[m] = cz
    assert np.abs(M2 - scale[:, None] * scale[None, :] * M1).max() <= 1e-12 * cz * cz * np.abs(M1).max()
