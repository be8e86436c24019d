"""The paper's printed parameter sets (tests/golden/paper_parameter_sets.json)
run through the oracle: dimensions follow from n_max, l_max (Sec. 3.3.2), the
kernel of an environment with itself is delta^2 (Eqs. 13, 24) and forces are
the negative energy gradient at the paper's hyperparameters."""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2310_03921_gb300 import synth as S

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_parameter_sets.json")))


@pytest.mark.parametrize("key", ["si_gap", "hea_soap"])
def test_paper_soap_parameter_sets(key):
    g = GOLD[key]
    n, l = g["n_max"], g["l_max"]
    soap = O.Soap(n, l, g["cutoff"], g["atom_gaussian_width"], d=g["cutoff_transition_width"])
    assert soap.dim == n * (n + 1) // 2 * (l + 1)
    s = S.displaced_diamond(0, 31, (1, 1, 2), 0.1)
    ph, _ = O.descriptor(soap, s)
    delta, zeta = g["energy_scale"], int(g["soap_exponent"])
    model = O.Model([ph[:4]], [np.array([0.3, -0.2, 0.1, 0.05])], delta, zeta)
    assert np.allclose(np.diag(O.kmm(model, soap.dim)), delta ** 2)
    E, le, F, V = O.predict(soap, model, s)
    h = 1e-4
    sp, sm = (S.Structure(s.pos.copy(), s.species, s.cell, s.pbc) for _ in range(2))
    sp.pos[3, 1] += h
    sm.pos[3, 1] -= h
    fd = -(O.predict(soap, model, sp)[0] - O.predict(soap, model, sm)[0]) / (2 * h)
    assert fd == pytest.approx(F[3, 1], abs=1e-6 * max(1.0, abs(F[3, 1])))


def test_paper_two_body_parameter_set():
    g = GOLD["hea_distance_2b"]
    tb = S.TwoBodySpec(rc=g["cutoff"], d=g["cutoff_transition_width"], theta=g["lengthscale_uniform"],
                       delta=g["energy_scale"], x=np.linspace(1.5, 4.5, g["n_sparse"]),
                       alpha=np.linspace(-0.1, 0.1, g["n_sparse"]))
    soap = O.Soap(2, 1, 5.0, 0.5)
    model = O.Model([np.zeros((0, soap.dim))], [np.zeros(0)], 1.0, 2, two_body=tb)
    pos = np.array([[5.0, 5.0, 5.0], [5.0, 7.5, 5.0]])
    s = S.Structure(pos, np.zeros(2, np.int32), np.eye(3) * 30.0, np.ones(3, np.int32))
    E, _, F, _ = O.predict(soap, model, s)
    k = np.exp(-(2.5 - tb.x) ** 2 / (2 * tb.theta ** 2))
    assert E == pytest.approx(tb.delta ** 2 * (tb.alpha * k).sum(), rel=1e-13)   # f_cut(2.5) = 1


def test_paper_full_descriptor_dimension():
    """The paper prints the dimension of its C/H/O SOAP descriptor (8 radial
    functions per element, l up to 8): 2700.  It fixes the storage of the
    fully coupled spectrum: channel pairs a <= b over all (species, n)
    channels, times l_max + 1 (24 * 25 / 2 * 9)."""
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_descriptor_dimension.json")))
    q = g["qm9_cho_soap"]
    soap = O.Soap(q["n_max"], q["l_max"], 5.0, 0.5, n_species=len(q["species"]))
    assert soap.dim == q["full_dimension"]
