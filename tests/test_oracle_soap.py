"""Pins of the oracle's SOAP descriptor (Eqs. 19-25) against invariances,
closed forms and reductions between its coupling variants."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2310_03921_gb300 import synth as S


def _rot(seed):
    q, _ = np.linalg.qr(np.random.default_rng(seed).normal(size=(3, 3)))
    return q * np.sign(np.linalg.det(q))


@pytest.mark.parametrize("reps,rc,count", [((2, 2, 2), 5.0, 28), ((1, 1, 1), 5.0, 28), ((1, 1, 1), 5.5, 34),
                                           ((1, 1, 2), 2.4, 4)])
def test_neighbour_count_diamond(reps, rc, count):
    """Undisplaced diamond (a = 5.431): shells at a*sqrt(3)/4 (4), a/sqrt(2) (12),
    a*sqrt(11)/4 (12) and a (6); cells smaller than 2 rc need several images."""
    s = S.diamond(reps)
    for i in range(s.n):
        j, sh, v = O.neighbours(s.pos, s.cell, s.pbc, rc, i)
        assert j.size == count
        r = np.linalg.norm(v, axis=1)
        assert np.all(r < rc) and np.all(r > 2.3)


@pytest.mark.parametrize("M", [((1, 0, 0), (1, 1, 0), (0, 1, 1)), ((1, 0, 0), (2, 1, 0), (0, -3, 1)),
                               ((1, 1, 1), (0, 1, 2), (0, 0, 1))])
def test_cell_choice_does_not_matter(M):
    """The same periodic crystal described by another cell: lattice vectors
    M a (M integer, det 1; rows of the cell are the lattice vectors), so the
    cell matrix is no longer symmetric and its perpendicular widths shrink
    below 2 r_c.  Pair counts (28 at r_c = 5, 34 at 5.5) and descriptors
    equal those of the cubic cell."""
    M = np.array(M, dtype=np.float64)
    assert round(abs(np.linalg.det(M))) == 1
    soap = O.Soap(4, 3, 5.0, 0.5)
    s = S.displaced_diamond(9, 3, (1, 1, 1), 0.1)
    t = S.Structure(s.pos, s.species, M @ s.cell, s.pbc)
    assert np.abs(t.cell - t.cell.T).max() > 1.0
    for rc, count in ((5.0, 28), (5.5, 34)):
        u = S.diamond((1, 1, 1))
        ut = S.Structure(u.pos, u.species, M @ u.cell, u.pbc)
        for i in range(u.n):
            assert O.neighbours(ut.pos, ut.cell, ut.pbc, rc, i)[0].size == count
    assert np.abs(O.descriptor(soap, t)[0] - O.descriptor(soap, s)[0]).max() < 1e-12


def test_neighbour_list_symmetric_with_images():
    s = S.displaced_diamond(9, 0, (1, 1, 1), 0.1)
    lists = [O.neighbours(s.pos, s.cell, s.pbc, 5.0, i) for i in range(s.n)]
    for i, (j, sh, v) in enumerate(lists):
        for jj, ss, vv in zip(j, sh, v):
            jr, sr, vr = lists[jj]
            hit = np.where((jr == i) & np.all(sr == -ss, axis=1))[0]
            assert hit.size == 1 and np.allclose(vr[hit[0]], -vv, atol=1e-12)


def test_descriptor_invariances():
    soap = O.Soap(6, 4, 5.0, 0.5)
    s = S.displaced_diamond(9, 1, (2, 2, 2), 0.15)
    p0, _ = O.descriptor(soap, s)
    assert np.allclose(np.linalg.norm(p0, axis=1), 1.0, atol=1e-14)      # k(rho, rho) = 1 (Eq. 24)
    R = _rot(5)
    rot = S.Structure(s.pos @ R.T, s.species, s.cell @ R.T, s.pbc)
    assert np.abs(O.descriptor(soap, rot)[0] - p0).max() < 1e-12
    tr = S.Structure(s.pos + np.array([0.37, -1.9, 12.3]), s.species, s.cell, s.pbc)
    assert np.abs(O.descriptor(soap, tr)[0] - p0).max() < 1e-12
    perm = np.random.default_rng(1).permutation(s.n)
    pm = S.Structure(s.pos[perm], s.species[perm], s.cell, s.pbc)
    assert np.abs(O.descriptor(soap, pm)[0] - p0[perm]).max() < 1e-12
    # wrapping an atom by a lattice vector changes nothing
    wr = S.Structure(s.pos.copy(), s.species, s.cell, s.pbc)
    wr.pos[5] += s.cell[1] - 2 * s.cell[2]
    assert np.abs(O.descriptor(soap, wr)[0] - p0).max() < 1e-12


def test_isolated_atom_closed_form():
    """An atom with no neighbour within the cutoff: only its own Gaussian
    contributes (Eq. 19 with r_j = 0 and f_cut(0) = 1), with weight
    central_weight and in the channels of its own species only, and
    i_l(0) = 0 for l > 0.  So c_{a,00} = w I_n0(0) / sqrt(4 pi) for a =
    (s_i, n), p_{ab0} = s_ab c_a c_b, and every other entry is 0; its forces
    and virial vanish."""
    N, L, cw = 4, 3, 0.7
    soap = O.Soap(N, L, 5.0, 0.5, central_weight=cw, n_species=2)
    s = S.Structure(np.array([[20.0, 20.0, 20.0]]), np.array([1], np.int32), np.eye(3) * 40.0, np.ones(3, np.int32))
    ph, pn = O.descriptor(soap, s)
    I, _ = O.radial_integrals(soap, 0.0)
    c = np.zeros(2 * N)
    c[N:] = cw * I[:, 0] / np.sqrt(4 * np.pi)
    p = np.array([(1.0 if a == b else np.sqrt(2.0)) * c[a] * c[b] * (l == 0)
                  for a in range(2 * N) for b in range(a, 2 * N) for l in range(L + 1)])
    assert np.abs(ph[0] * pn[0] - p).max() <= 1e-13 * np.abs(p).max()
    rng = np.random.default_rng(5)
    X = [rng.normal(size=(3, p.size)) for _ in range(2)]
    X = [x / np.linalg.norm(x, axis=1, keepdims=True) for x in X]
    E, le, F, V = O.predict(soap, O.Model(X, [rng.normal(size=3), rng.normal(size=3)], 1.1, 4), s)
    assert np.isfinite(E) and np.all(F == 0.0) and np.all(V == 0.0)


def _dimer(r, box=40.0):
    pos = np.array([[10.0, 10.0, 10.0], [10.0, 10.0, 10.0 + r]])
    return S.Structure(pos, np.zeros(2, np.int32), np.eye(3) * box, np.zeros(3, np.int32))


@pytest.mark.parametrize("r", [1.7, 3.2, 4.4])
def test_single_neighbour_closed_form(r):
    """One neighbour on +z, no central Gaussian: c_nlm = f I_nl Y_lm(z) with
    Y_lm(z) = delta_m0 sqrt((2l+1)/4pi), so p_nn'l = s_nn' f^2 I_nl I_n'l (2l+1)/(4pi)."""
    N, L = 6, 5
    soap = O.Soap(N, L, 5.0, 0.5, central_weight=0.0)
    ph, pn = O.descriptor(soap, _dimer(r), sel=[0])
    p = ph[0] * pn[0]
    I, _ = O.radial_integrals(soap, r)
    f = O.fcut(r, 5.0, 1.0)[0]
    ref, d = np.zeros(p.size), 0
    for a in range(N):
        for b in range(a, N):
            for l in range(L + 1):
                s = 1.0 if a == b else math.sqrt(2.0)
                ref[d] = s * f * f * I[a, l] * I[b, l] * (2 * l + 1) / (4 * math.pi)
                d += 1
    assert np.abs(p - ref).max() < 1e-13 * np.abs(ref).max()


def test_bessel_inequality_and_nested_basis():
    """sum c^2 <= int rho^2 (projection on an orthonormal set); with the
    Gram-Schmidt basis, raising n_max keeps the earlier coefficients."""
    s = S.displaced_diamond(9, 2, (2, 2, 2), 0.1)
    sig, rc = 0.5, 5.0
    small = O.Soap(6, 4, rc, sig)
    big = O.Soap(8, 6, rc, sig)
    _, _, c6 = O.descriptor(small, s, sel=[0, 7], with_coef=True)
    _, _, c8 = O.descriptor(big, s, sel=[0, 7], with_coef=True)
    assert np.abs(c8[:, 0, :6, :25] - c6[:, 0, :, :]).max() < 1e-12
    for t, i in enumerate([0, 7]):
        j, _, v = O.neighbours(s.pos, s.cell, s.pbc, rc, i)
        w = np.array([1.0] + [O.fcut(np.linalg.norm(x), rc, 1.0)[0] for x in v])
        cen = np.vstack([np.zeros(3), v])
        d2 = ((cen[:, None, :] - cen[None, :, :]) ** 2).sum(-1)
        norm2 = (w[:, None] * w[None, :] * (math.pi * sig * sig) ** 1.5 * np.exp(-d2 / (4 * sig * sig))).sum()
        s6, s8 = (c6[t] ** 2).sum(), (c8[t] ** 2).sum()
        assert s6 <= s8 * (1 + 1e-14) and s8 <= norm2


def test_species_coupling_reductions():
    rng_struct = S.random_packing(9, 0, 40, 0.05, 1.8, n_species=2)
    N, L = 4, 3
    single = O.Soap(N, L, 5.0, 0.5)
    full = O.Soap(N, L, 5.0, 0.5, n_species=2)
    # (a) all atoms species 0: the (0,0) species block of full coupling is the single-species p
    s0 = S.Structure(rng_struct.pos, np.zeros(40, np.int32), rng_struct.cell, rng_struct.pbc)
    p1, n1 = O.descriptor(single, s0)
    pf, nf = O.descriptor(full, s0)
    keep = [a < N and b < N for a in range(2 * N) for b in range(a, 2 * N) for _ in range(L + 1)]
    assert np.abs(pf[:, keep] * nf[:, None] - p1 * n1[:, None]).max() < 1e-12
    assert np.abs(pf[:, [not k for k in keep]]).max() == 0.0
    # (b) one embedded channel with unit weights: species become indistinguishable
    mix1 = O.Soap(N, L, 5.0, 0.5, n_species=2, mix_K=1, mix_w=np.ones((1, 2)))
    assert np.abs(O.descriptor(mix1, rng_struct)[0] - p1).max() < 1e-12
    # (c) identity embedding: p^k_nn'l is the diagonal (k,k) block of full coupling
    mixI = O.Soap(N, L, 5.0, 0.5, n_species=2, mix_K=2, mix_w=np.eye(2))
    pm, nm = O.descriptor(mixI, rng_struct)
    pf, nf = O.descriptor(full, rng_struct)
    blocks = []
    for k in range(2):
        blocks.append([(a // N == k and b // N == k) for a in range(2 * N) for b in range(a, 2 * N)
                       for _ in range(L + 1)])
    ref = np.concatenate([(pf * nf[:, None])[:, blocks[k]] for k in range(2)], axis=1)
    assert np.abs(pm * nm[:, None] - ref).max() < 1e-12


def test_embedding_weights_are_channel_by_species():
    """Eq. 25 with mix_w [K][n_species], row k the weights of embedded
    channel k: with w = [[1, 0], [1, 1]] channel 0 sees only species 0 (the
    (0, 0) block of full coupling) and channel 1 sees every atom alike (the
    single-species spectrum).  The weights are not symmetric, so reading them
    as [n_species][K] fails."""
    st = S.random_packing(9, 0, 40, 0.05, 1.8, n_species=2)
    N, L = 4, 3
    w = np.array([[1.0, 0.0], [1.0, 1.0]])
    pm, nm = O.descriptor(O.Soap(N, L, 5.0, 0.5, n_species=2, mix_K=2, mix_w=w), st)
    pf, nf = O.descriptor(O.Soap(N, L, 5.0, 0.5, n_species=2), st)
    blind = S.Structure(st.pos, np.zeros(st.n, np.int32), st.cell, st.pbc)
    ps, ns = O.descriptor(O.Soap(N, L, 5.0, 0.5), blind)
    block00 = [a < N and b < N for a in range(2 * N) for b in range(a, 2 * N) for _ in range(L + 1)]
    half = pm.shape[1] // 2
    p = pm * nm[:, None]
    assert np.abs(p[:, :half] - (pf * nf[:, None])[:, block00]).max() < 1e-12
    assert np.abs(p[:, half:] - ps * ns[:, None]).max() < 1e-12


def test_dimension_formula():
    assert O.Soap(6, 4, 5.0, 0.5).dim == 105
    assert O.Soap(8, 6, 5.0, 0.5).dim == 252
    assert O.Soap(8, 8, 5.0, 0.5).dim == 324
    assert O.Soap(10, 8, 4.5, 0.5).dim == 495
    assert O.Soap(8, 6, 5.0, 0.5, n_species=4, mix_K=4, mix_w=np.ones((4, 4))).dim == 1008
