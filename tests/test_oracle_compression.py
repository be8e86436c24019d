"""Pins of the oracle's compressed descriptors (Sec. 3.3.3 tensor
decomposition and tensor sketch, nu_R / nu_S correlation orders; Sec. 3.3.4
soap_turbo recipes).  Independent of the compression code itself: the
paper's sketch identity E[p~ . p~'] = K sigma^4 p . p', closed forms from the
expansion coefficients, agreement with the uncompressed descriptor where a
recipe is lossless, rotation invariance, and energies by finite differences
are exercised by the GPU tests against these functions."""
import numpy as np
import pytest

import oracle as O
from paper_2310_03921_gb300 import synth as S


def _soap():
    return O.Soap(4, 3, 5.0, 0.5, 1.0, n_species=2)


def _cell(seed, sig=0.15):
    s = S.displaced_diamond(0, seed, (1, 1, 1), sig)
    sp = S.SplitMix64(seed).integers(s.n, 0, 1).astype(np.int32)
    return S.Structure(s.pos, sp, s.cell, s.pbc)


def test_sketch_identity_in_expectation():
    """E[p~ . p~'] = K sigma^4 p . p' (Sec. 3.3.3) for independent w, u with
    E[w_i w_j] = sigma^2 delta_ij: with many channels the normalised sketches'
    dot products approach those of the full descriptor."""
    soap = _soap()
    s1, s2 = _cell(1), _cell(2)
    p1, p2 = O.descriptor(soap, s1)[0], O.descriptor(soap, s2)[0]
    Nc = 8
    K = 40000
    rng = np.random.default_rng(0)
    comp = dict(recipe="sketch", w=rng.normal(size=(K, Nc)), u=rng.normal(size=(K, Nc)))
    q1, q2 = O.compressed_descriptor(soap, s1, comp), O.compressed_descriptor(soap, s2, comp)
    ref = p1 @ p2.T
    got = q1 @ q2.T
    # relative error ~ K^-1/2 ~ 0.5 %
    assert np.abs(got - ref).max() <= 0.03


def test_decomposition_with_unit_weights_is_the_diagonal():
    """w^k = e_k (K = S n_max): p~^k_l = sum_m c_{k,lm}^2 = p_{kk l}."""
    soap = _soap()
    s = _cell(3)
    ph, pn = O.descriptor(soap, s)
    comp = dict(recipe="decomposition", w=np.eye(8))
    q = O.compressed_descriptor(soap, s, comp)
    # diagonal entries of the stored spectrum: pair (a, a), all l
    Nc, L = 8, 3
    idx = []
    pi = 0
    for a in range(Nc):
        for b in range(a, Nc):
            if a == b:
                idx += [pi * (L + 1) + l for l in range(L + 1)]
            pi += 1
    diag = ph[:, idx] * pn[:, None]
    ref = diag / np.linalg.norm(diag, axis=1, keepdims=True)
    assert np.abs(q - ref).max() <= 1e-12


def test_nu_full_orders_keep_the_kernel_and_zero_orders_sum_channels():
    soap = _soap()
    s, t = _cell(4), _cell(5)
    ph_s, ph_t = O.descriptor(soap, s)[0], O.descriptor(soap, t)[0]
    # nu_S = nu_R = 2: every ordered entry, so dot products equal the full descriptor's
    q_s = O.compressed_descriptor(soap, s, dict(recipe="nu", nu_S=2, nu_R=2))
    q_t = O.compressed_descriptor(soap, t, dict(recipe="nu", nu_S=2, nu_R=2))
    assert q_s.shape[1] == 8 * 8 * 4
    assert np.abs(q_s @ q_t.T - ph_s @ ph_t.T).max() <= 1e-12
    # nu_S = nu_R = 0: p_l = sum_m (sum_a c_{a,lm})^2, the element- and radius-blind density
    q0 = O.compressed_descriptor(soap, s, dict(recipe="nu", nu_S=0, nu_R=0))
    _, _, coef = O.descriptor(soap, s, with_coef=True)
    tot = coef[:, 0].sum(axis=1)  # [n][(L+1)^2]
    ref = np.stack([(tot[:, l * l:(l + 1) ** 2] ** 2).sum(1) for l in range(4)], axis=1)
    ref /= np.linalg.norm(ref, axis=1, keepdims=True)
    assert q0.shape[1] == 4 and np.abs(q0 - ref).max() <= 1e-12


def test_nu_one_orders_keep_the_first_index():
    """nu_S = 1 keeps the first species index and sums the second, nu_R = 1
    keeps the first radial index and sums the second (Sec. 3.3.3): closed
    forms from the expansion coefficients,
        nu_S = 1:  v[a][n][n'][l] = sum_m c^a_{n,lm} (sum_b c^b_{n',lm})
        nu_R = 1:  v[a][b][n][l]  = sum_m c^a_{n,lm} (sum_n' c^b_{n',lm}).
    Summing the other index of either pair gives the same numbers with the
    kept index moved to the other factor (p^{ab}_{nn'l} = p^{ba}_{n'nl}),
    which the invariance and full- and zero-order pins cannot see."""
    soap = _soap()
    s = _cell(8)
    Sn, N, L = 2, 4, 3
    _, _, coef = O.descriptor(soap, s, with_coef=True)
    c = coef[:, 0].reshape(-1, Sn, N, (L + 1) ** 2)  # [atom][species][n][lm]

    def by_l(x, y):  # sum over m within each l of x[..., lm] y[..., lm]
        return np.stack([(x[..., l * l:(l + 1) ** 2] * y[..., l * l:(l + 1) ** 2]).sum(-1) for l in range(L + 1)], -1)

    tot_s = c.sum(axis=1)  # [atom][n'][lm]
    ref_s = by_l(c[:, :, :, None, :], tot_s[:, None, None, :, :]).reshape(c.shape[0], -1)
    tot_r = c.sum(axis=2)  # [atom][b][lm]
    ref_r = by_l(c[:, :, None, :, :], tot_r[:, None, :, None, :]).reshape(c.shape[0], -1)
    for comp, ref in ((dict(recipe="nu", nu_S=1, nu_R=2), ref_s), (dict(recipe="nu", nu_S=2, nu_R=1), ref_r)):
        q = O.compressed_descriptor(soap, s, comp)
        ref = ref / np.linalg.norm(ref, axis=1, keepdims=True)
        assert q.shape == ref.shape and np.abs(q - ref).max() <= 1e-12


@pytest.mark.parametrize("comp", [
    dict(recipe="nu", nu_S=1, nu_R=1), dict(recipe="nu", nu_S=2, nu_R=0), dict(recipe="trivial"),
    dict(recipe="sketch", w=np.random.default_rng(1).normal(size=(5, 8)), u=np.random.default_rng(2).normal(size=(5, 8))),
])
def test_compressed_descriptors_are_rotation_invariant(comp):
    soap = _soap()
    s = _cell(6)
    th = 0.7
    R = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1.0]])
    R = R @ np.array([[1, 0, 0], [0, np.cos(0.4), -np.sin(0.4)], [0, np.sin(0.4), np.cos(0.4)]])
    r = S.Structure(s.pos @ R.T, s.species, s.cell @ R.T, s.pbc)
    assert np.abs(O.compressed_descriptor(soap, s, comp) - O.compressed_descriptor(soap, r, comp)).max() <= 1e-11


def test_matrix_identity_and_trivial_entries():
    soap = _soap()
    s = _cell(7)
    ph, _ = O.descriptor(soap, s)
    q = O.compressed_descriptor(soap, s, dict(recipe="matrix", P=np.eye(ph.shape[1])))
    assert np.abs(q - ph).max() <= 1e-13
    # trivial: entry (alpha, b, l) is P^{(alpha, n=0), b}_l of the ordered spectrum
    qt = O.compressed_descriptor(soap, s, dict(recipe="trivial"))
    _, _, coef = O.descriptor(soap, s, with_coef=True)
    c = coef[0, 0]
    v = np.array([[[c[a, l * l:(l + 1) ** 2] @ c[b, l * l:(l + 1) ** 2] for l in range(4)] for b in range(8)]
                  for a in (0, 4)]).ravel()
    assert np.abs(qt[0] - v / np.linalg.norm(v)).max() <= 1e-13


def test_identity_map_energies_equal_the_uncompressed_oracle():
    """With the identity matrix recipe the compressed descriptor is p_hat
    itself, so the compressed local energies (Eqs. 2, 13 on p~) equal the C
    oracle's local energies of the same model, two species and two GPs."""
    soap = _soap()
    s = _cell(9)
    ph, _ = O.descriptor(soap, s)
    rng = np.random.default_rng(9)
    X = [ph[:3] + 0.1 * rng.normal(size=(3, ph.shape[1])) for _ in range(2)]
    X = [x / np.linalg.norm(x, axis=1, keepdims=True) for x in X]
    model = O.Model(X, [rng.normal(size=3), rng.normal(size=3)], 1.2, 4)
    eps = O.compressed_local_energies(soap, dict(recipe="matrix", P=np.eye(ph.shape[1])), model, s)
    _, le, _, _ = O.predict(soap, model, s)
    assert np.abs(eps - le).max() <= 1e-12 * max(1.0, np.abs(le).max())
