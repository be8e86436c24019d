"""Pins of the oracle's energies, forces and virials (Eqs. 1-3, 13) by exact
identities, invariances and finite differences of the energy."""
import numpy as np
import pytest

import oracle as O
from paper_2310_03921_gb300 import synth as S
from _models import oracle_model


@pytest.fixture(scope="module")
def c1():
    soap, model, _, _ = oracle_model(0, 100)
    return soap, model, S.structures(0)[0]


def _energy(soap, model, s):
    return O.predict(soap, model, s)[0]


def test_energy_is_sum_of_local_and_forces_sum_to_zero(c1):
    soap, model, s = c1
    E, le, F, V = O.predict(soap, model, s)
    assert E == pytest.approx(le.sum(), abs=1e-12)
    assert np.abs(F.sum(0)).max() < 1e-12
    assert np.abs(V - V.T).max() < 1e-10 * np.abs(V).max()


def test_local_energy_matches_direct_kernel_sum(c1):
    """eps_i = delta^2 sum_m alpha_m (p_hat_i . x_m)^zeta evaluated from the descriptor."""
    soap, model, s = c1
    _, le, _, _ = O.predict(soap, model, s)
    ph, _ = O.descriptor(soap, s)
    ref = model.c.delta ** 2 * ((ph @ model.sparse.T) ** model.c.zeta) @ model.alpha
    assert np.abs(le - ref).max() < 1e-12


def test_forces_by_finite_differences(c1):
    soap, model, s = c1
    _, _, F, _ = O.predict(soap, model, s)
    h = 1e-4
    for a, x in [(0, 0), (13, 1), (41, 2), (63, 0)]:
        sp, sm = (S.Structure(s.pos.copy(), s.species, s.cell, s.pbc) for _ in range(2))
        sp.pos[a, x] += h
        sm.pos[a, x] -= h
        fd = -(_energy(soap, model, sp) - _energy(soap, model, sm)) / (2 * h)
        assert fd == pytest.approx(F[a, x], abs=1e-6)


def test_virial_by_finite_strain(c1):
    """V_ab = -dE/de_ab under r -> (I + e) r applied to positions and cell."""
    soap, model, s = c1
    _, _, _, V = O.predict(soap, model, s)
    h = 1e-5
    for a, b in [(0, 0), (1, 2), (2, 1), (0, 1)]:
        e = np.zeros((3, 3))
        e[a, b] = h
        def strained(sign):
            T = np.eye(3) + sign * e
            return S.Structure(s.pos @ T.T, s.species, s.cell @ T.T, s.pbc)
        fd = -(_energy(soap, model, strained(1)) - _energy(soap, model, strained(-1))) / (2 * h)
        assert fd == pytest.approx(V[a, b], abs=1e-6 * max(1.0, abs(V[a, b])))


def test_rotation_translation_invariance(c1):
    soap, model, s = c1
    E, _, F, V = O.predict(soap, model, s)
    q, _ = np.linalg.qr(np.random.default_rng(11).normal(size=(3, 3)))
    q *= np.sign(np.linalg.det(q))
    s2 = S.Structure(s.pos @ q.T + 3.3, s.species, s.cell @ q.T, s.pbc)
    E2, _, F2, V2 = O.predict(soap, model, s2)
    assert E2 == pytest.approx(E, abs=1e-10)
    assert np.abs(F2 - F @ q.T).max() < 1e-10
    assert np.abs(V2 - q @ V @ q.T).max() < 1e-9


def test_sampled_equals_full(c1):
    soap, model, s = c1
    _, le, F, _ = O.predict(soap, model, s)
    sel = [2, 30, 63]
    le_s, F_s = O.predict_sampled(soap, model, s, sel)
    assert np.abs(le_s - le[sel]).max() < 1e-12
    assert np.abs(F_s - F[sel]).max() < 1e-12


def test_two_body_dimer_closed_form():
    """Two atoms, SOAP switched off (no sparse points): E = delta2^2 sum_m
    alpha_m f_cut(r) exp(-(r - x_m)^2 / (2 theta^2)), one unordered pair."""
    w = S.workload(4)
    tb = w.two_body
    soap = O.Soap(4, 2, 4.5, 0.5)
    model = O.Model([np.zeros((0, soap.dim))], [np.zeros(0)], 1.0, 4, two_body=tb)
    for r in [1.6, 3.0, 3.9]:
        pos = np.array([[5.0, 5.0, 5.0], [5.0 + r, 5.0, 5.0]])
        s = S.Structure(pos, np.zeros(2, np.int32), np.eye(3) * 30.0, np.ones(3, np.int32))
        E, le, F, _ = O.predict(soap, model, s)
        f, df = O.fcut(r, tb.rc, tb.d)
        k = np.exp(-(r - tb.x) ** 2 / (2 * tb.theta ** 2))
        ref = tb.delta ** 2 * (tb.alpha * f * k).sum()
        dref = tb.delta ** 2 * (tb.alpha * (df - f * (r - tb.x) / tb.theta ** 2) * k).sum()
        assert E == pytest.approx(ref, rel=1e-13)
        assert le[0] == pytest.approx(0.5 * ref, rel=1e-13)
        assert F[1, 0] == pytest.approx(-dref, rel=1e-12, abs=1e-12)
        assert F[0, 0] == pytest.approx(dref, rel=1e-12, abs=1e-12)


def test_multispecies_mixed_forces_by_finite_differences():
    w = S.workload(3)
    soap, model, _, _ = oracle_model(3, 12, n_max=4, l_max=3, n_cells=3)
    s = S.structures(3, 3)[2]
    E, le, F, V = O.predict(soap, model, s)
    assert np.abs(F.sum(0)).max() < 1e-11
    h = 1e-4
    for a, x in [(0, 0), (7, 2), (s.n - 1, 1)]:
        sp, sm = (S.Structure(s.pos.copy(), s.species, s.cell, s.pbc) for _ in range(2))
        sp.pos[a, x] += h
        sm.pos[a, x] -= h
        fd = -(O.predict(soap, model, sp)[0] - O.predict(soap, model, sm)[0]) / (2 * h)
        assert fd == pytest.approx(F[a, x], abs=1e-6)
    assert w.soap.mix_K == 4


def test_two_body_plus_soap_forces_by_finite_differences():
    soap, model, _, _ = oracle_model(4, 30, n_max=5, l_max=3, n_cells=1)
    full = S.random_packing(4, 7, 60, 0.1, 1.4)
    E, le, F, V = O.predict(soap, model, full)
    assert E == pytest.approx(le.sum(), abs=1e-10)
    h = 1e-4
    for a, x in [(3, 1), (40, 0)]:
        sp, sm = (S.Structure(full.pos.copy(), full.species, full.cell, full.pbc) for _ in range(2))
        sp.pos[a, x] += h
        sm.pos[a, x] -= h
        fd = -(O.predict(soap, model, sp)[0] - O.predict(soap, model, sm)[0]) / (2 * h)
        assert fd == pytest.approx(F[a, x], abs=2e-6 * max(1.0, abs(F[a, x])))
