"""GPU parity of the full path through the C-ABI against the FP64 oracle.

Tolerances: the plain FP64 path matches per-atom energies to 1e-6 eV and
forces to 1e-6 eV/A; the reduced-precision forms (BF16X3 tensor cores, FP32
CUDA cores) match force components to 1e-4 eV/A."""
import numpy as np
import pytest

import oracle as O
from paper_2310_03921_gb300 import synth as S
from _models import oracle_model

pytestmark = pytest.mark.gpu

TOL = {"fp64": dict(e=1e-6, f=1e-6, v=1e-5), "fp32": dict(e=1e-4, f=1e-4, v=1e-3),
       "bf16x3": dict(e=1e-4, f=1e-4, v=1e-3), "bf16x6": dict(e=1e-4, f=1e-4, v=1e-3)}


@pytest.fixture(scope="module")
def G():
    from paper_2310_03921_gb300 import build, gap
    build.build()
    return gap


def _gpu_model(G, index, soap_o, sparse, alpha, n_max=None, l_max=None, two_body=True):
    w = S.workload(index)
    sp = w.soap
    soap = G.Soap(n_max or sp.n_max, sp.l_max if l_max is None else l_max, sp.rc, sp.sigma, sp.d, sp.central_weight,
                  sp.n_species, sp.mix_K, sp.mix_w)
    tb = w.two_body if two_body else None
    return soap, G.Model(soap, sparse, alpha, w.delta, w.zeta, two_body=tb)


def _as_np(x):
    return x.cpu().numpy() if hasattr(x, "cpu") else x


def _oracle_batch(soap_o, model_o, structs):
    E, le, F, V = [], [], [], []
    for s in structs:
        e, l_, f, v = O.predict(soap_o, model_o, s)
        E.append(e); le.append(l_); F.append(f); V.append(v)
    return np.array(E), np.concatenate(le), np.concatenate(F), np.stack(V)


def _compare(out, ref, tol, n_atoms_per_cfg=None):
    E, le, F, V = ref
    assert np.abs(_as_np(out["local_e"]) - le).max() <= tol["e"]
    assert np.abs(_as_np(out["forces"]) - F).max() <= tol["f"]
    nat = n_atoms_per_cfg if n_atoms_per_cfg is not None else np.ones(len(E))
    assert np.all(np.abs(_as_np(out["energy"]) - E) <= tol["e"] * np.maximum(nat, 1))
    assert np.abs(_as_np(out["virial"]) - V).max() <= tol["v"] * max(1.0, np.abs(V).max())


@pytest.fixture(scope="module")
def c1(G):
    soap_o, model_o, sparse, alpha = oracle_model(0, 100)
    s = S.structures(0)[0]
    ref = O.predict(soap_o, model_o, s)
    soap, model = _gpu_model(G, 0, soap_o, sparse, alpha)
    return soap_o, model_o, soap, model, s, ref


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 2e-6), ("bf16x3", 2e-6)])
def test_descriptor_parity(G, c1, prec, tol):
    soap_o, _, soap, _, s, _ = c1
    ref, _ = O.descriptor(soap_o, s)
    got = soap.descriptor(G.Batch.from_synth(S.make_batch([s]), device="cuda"), precision=prec)
    assert np.abs(_as_np(got) - ref).max() < tol


def test_pair_counts_match_oracle(G, c1):
    soap_o, _, soap, _, s, _ = c1
    nd, npairs = soap.descriptor_sizes(G.Batch.from_synth(S.make_batch([s])))
    ref = sum(O.neighbours(s.pos, s.cell, s.pbc, 5.0, i)[0].size for i in range(s.n))
    assert nd == s.n and npairs == ref


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16x3", "bf16x6"])
def test_predict_c1(G, c1, prec):
    _, _, _, model, s, (E, le, F, V) = c1
    out = model.predict(G.Batch.from_synth(S.make_batch([s]), device="cuda"), precision=prec)
    _compare(out, (np.array([E]), le, F, V[None]), TOL[prec], [s.n])


def test_host_and_device_pointers_agree(G, c1):
    _, _, _, model, s, _ = c1
    b = S.make_batch([s])
    a = model.predict(G.Batch.from_synth(b), precision="fp64")
    d = model.predict(G.Batch.from_synth(b, device="cuda"), precision="fp64")
    for k in ("energy", "local_e", "forces", "virial"):
        assert np.array_equal(a[k], _as_np(d[k]))


def test_deterministic(G, c1):
    _, _, _, model, s, _ = c1
    b = G.Batch.from_synth(S.make_batch([s]), device="cuda")
    r1 = model.predict(b, precision="bf16x3")
    r2 = model.predict(b, precision="bf16x3")
    for k in ("energy", "forces", "virial"):
        assert np.array_equal(_as_np(r1[k]), _as_np(r2[k]))


def test_batch_of_strained_cells(G):
    soap_o, model_o, sparse, alpha = oracle_model(1, 64, n_cells=2)
    cells = S.structures(1, 4)
    ref = _oracle_batch(soap_o, model_o, cells)
    soap, model = _gpu_model(G, 1, soap_o, sparse, alpha)
    b = G.Batch.from_synth(S.make_batch(cells), device="cuda")
    nat = [c.n for c in cells]
    for prec in ("fp64", "bf16x3", "bf16x6"):
        _compare(model.predict(b, precision=prec), ref, TOL[prec], nat)


def test_small_cells_need_several_images(G, c1):
    soap_o, model_o, soap, model, _, _ = c1
    cells = [S.displaced_diamond(0, 50 + k, (1, 1, 1), 0.1) for k in range(3)]
    ref = _oracle_batch(soap_o, model_o, cells)
    b = G.Batch.from_synth(S.make_batch(cells), device="cuda")
    _compare(model.predict(b, precision="fp64"), ref, TOL["fp64"], [8, 8, 8])


def test_sheared_and_rotated_cells(G, c1):
    """The same crystals described by sheared cells (lattice vectors M a with
    M integer of determinant 1: cell matrices that are not symmetric, and
    perpendicular widths below 2 r_c) and by rotated sheared cells: energies,
    forces and virials against the oracle on those cells, and the sheared
    cells' results against the cubic cells' (the description of the crystal
    does not change it)."""
    soap_o, model_o, soap, model, _, _ = c1
    M = np.array([[1.0, 0.0, 0.0], [2.0, 1.0, 0.0], [0.0, -3.0, 1.0]])
    q, _ = np.linalg.qr(np.random.default_rng(21).normal(size=(3, 3)))
    base = [S.displaced_diamond(0, 60 + k, (1, 1, 2), 0.1) for k in range(2)]
    sheared = [S.Structure(c.pos, c.species, M @ c.cell, c.pbc) for c in base]
    rotated = [S.Structure(c.pos @ q.T, c.species, M @ c.cell @ q.T, c.pbc) for c in base]
    cells = sheared + rotated
    assert all(np.abs(c.cell - c.cell.T).max() > 1.0 for c in cells)
    ref = _oracle_batch(soap_o, model_o, cells)
    b = G.Batch.from_synth(S.make_batch(cells), device="cuda")
    nat = [c.n for c in cells]
    for prec in ("fp64", "bf16x3"):
        _compare(model.predict(b, precision=prec), ref, TOL[prec], nat)
    cubic = model.predict(G.Batch.from_synth(S.make_batch(base), device="cuda"), precision="fp64")
    shear = model.predict(G.Batch.from_synth(S.make_batch(sheared), device="cuda"), precision="fp64")
    assert np.abs(_as_np(shear["energy"]) - _as_np(cubic["energy"])).max() <= 1e-9
    assert np.abs(_as_np(shear["forces"]) - _as_np(cubic["forces"])).max() <= 1e-10
    assert np.abs(_as_np(shear["virial"]) - _as_np(cubic["virial"])).max() <= 1e-9


def test_slabs_and_clusters_with_atoms_outside_the_cell(G, c1):
    """Non-periodic directions: a slab (periodic in x and y only) whose atoms
    extend beyond both faces of the cell along z, and a cluster (no periodic
    direction) larger than its cell on every side.  The cells are wide enough
    for two neighbour bins per direction, so atoms outside the cell sit in
    clamped edge bins.  Energies, forces and virials against the oracle."""
    soap_o, model_o, soap, model, _, _ = c1
    d = S.displaced_diamond(0, 70, (2, 2, 3), 0.1)
    slab_cell = d.cell.copy()
    slab_cell[2, 2] = 11.0
    slab = S.Structure(d.pos - np.array([0.0, 0.0, 3.0]), d.species, slab_cell, np.array([1, 1, 0], np.int32))
    assert slab.pos[:, 2].min() < -2.0 and slab.pos[:, 2].max() > 12.0
    c = S.displaced_diamond(0, 71, (3, 3, 3), 0.1)
    cluster = S.Structure(c.pos - 3.0, c.species, 10.5 * np.eye(3), np.zeros(3, np.int32))
    assert cluster.pos.min() < -2.0 and cluster.pos.max() > 12.0
    cells = [slab, cluster]
    ref = _oracle_batch(soap_o, model_o, cells)
    b = G.Batch.from_synth(S.make_batch(cells), device="cuda")
    nd, npairs = soap.descriptor_sizes(G.Batch.from_synth(S.make_batch(cells)))
    assert npairs == sum(O.neighbours(x.pos, x.cell, x.pbc, 5.0, i)[0].size for x in cells for i in range(x.n))
    nat = [x.n for x in cells]
    for prec in ("fp64", "bf16x3"):
        _compare(model.predict(b, precision=prec), ref, TOL[prec], nat)


def test_mixed_species_compressed(G):
    soap_o, model_o, sparse, alpha = oracle_model(3, 24, n_cells=2)
    cells = S.structures(3, 3)
    ref = _oracle_batch(soap_o, model_o, cells)
    soap, model = _gpu_model(G, 3, soap_o, sparse, alpha)
    b = G.Batch.from_synth(S.make_batch(cells), device="cuda")
    nat = [c.n for c in cells]
    for prec in ("fp64", "bf16x3"):
        _compare(model.predict(b, precision=prec), ref, TOL[prec], nat)


def test_full_species_coupling(G):
    N, L = 4, 3
    soap_o = O.Soap(N, L, 5.0, 0.5, n_species=2)
    pool_cells = [S.random_packing(9, 100 + k, 60, 0.05, 1.8, n_species=2) for k in range(3)]
    P = [O.descriptor(soap_o, c)[0] for c in pool_cells]
    Z = np.concatenate([c.species for c in pool_cells])
    P = np.concatenate(P)
    sparse = [P[Z == 0][:20], P[Z == 1][:15]]
    alpha = [S.alpha_draw(9, 0, 20), S.alpha_draw(9, 1, 15)]
    model_o = O.Model(sparse, alpha, 1.0, 4)
    cells = [S.random_packing(9, 200 + k, 40 + 17 * k, 0.05, 1.8, n_species=2) for k in range(3)]
    ref = _oracle_batch(soap_o, model_o, cells)
    soap = G.Soap(N, L, 5.0, 0.5, n_species=2)
    model = G.Model(soap, sparse, alpha, 1.0, 4)
    b = G.Batch.from_synth(S.make_batch(cells), device="cuda")
    for prec in ("fp64", "bf16x3"):
        _compare(model.predict(b, precision=prec), ref, TOL[prec], [c.n for c in cells])


@pytest.mark.parametrize("N,L,S5,D", [(8, 4, 5, 4100), (8, 6, 4, 3696)])
def test_fully_coupled_many_species(G, N, L, S5, D):
    """Large fully coupled descriptors: the paper's five-element alloy SOAP
    (Sec. 4.3: n_max 8, l_max 4, five species, D = 4100, zeta 2) and four
    species at n_max 8, l_max 6 (D = 3696); energies and forces of
    random-packed boxes against the oracle, FP64 and BF16x3."""
    soap_o = O.Soap(N, L, 5.0, 0.5, n_species=S5)
    pool_cells = [S.random_packing(10, 100 + k, 80, 0.06, 2.0, n_species=S5) for k in range(2)]
    P = np.concatenate([O.descriptor(soap_o, c)[0] for c in pool_cells])
    Z = np.concatenate([c.species for c in pool_cells])
    sparse = [P[Z == z][:12] for z in range(S5)]
    alpha = [S.alpha_draw(10, z, sparse[z].shape[0]) for z in range(S5)]
    model_o = O.Model(sparse, alpha, 1.0, 2)
    cells = [S.random_packing(10, 200 + k, 30 + 11 * k, 0.06, 2.0, n_species=S5) for k in range(2)]
    ref = _oracle_batch(soap_o, model_o, cells)
    soap = G.Soap(N, L, 5.0, 0.5, n_species=S5)
    assert soap.dim == D
    model = G.Model(soap, sparse, alpha, 1.0, 2)
    b = G.Batch.from_synth(S.make_batch(cells), device="cuda")
    for prec in ("fp64", "bf16x3"):
        _compare(model.predict(b, precision=prec), ref, TOL[prec], [c.n for c in cells])


def test_two_body_plus_soap(G):
    soap_o, model_o, sparse, alpha = oracle_model(4, 40, n_cells=1)
    cells = [S.random_packing(4, 300 + k, 90, 0.1, 1.4) for k in range(2)]
    ref = _oracle_batch(soap_o, model_o, cells)
    soap, model = _gpu_model(G, 4, soap_o, sparse, alpha)
    b = G.Batch.from_synth(S.make_batch(cells), device="cuda")
    for prec in ("fp64", "bf16x3", "bf16x6"):
        _compare(model.predict(b, precision=prec), ref, TOL[prec], [c.n for c in cells])


def test_empty_and_ragged_batches(G, c1):
    _, model_o, soap, model, s, _ = c1
    empty = G.Batch(np.zeros((0, 3)), np.zeros(0, np.int32), np.zeros((0, 3, 3)), np.zeros((0, 3), np.int32),
                    np.zeros(1, np.int32))
    out = model.predict(empty, precision="bf16x3")
    assert out["energy"].shape == (0,)
    # a configuration without atoms between two real ones
    s0 = S.Structure(np.zeros((0, 3)), np.zeros(0, np.int32), s.cell, s.pbc)
    b = S.make_batch([s, s0, s])
    out = model.predict(G.Batch.from_synth(b, device="cuda"), precision="fp64")
    E = _as_np(out["energy"])
    assert E[1] == 0.0 and E[0] == E[2]


def test_invalid_species_is_an_error(G, c1):
    _, _, _, model, s, _ = c1
    b = S.make_batch([s])
    b.species[3] = 5
    with pytest.raises(G.GapError):
        model.predict(G.Batch.from_synth(b), precision="fp64")
    with pytest.raises(G.GapError):
        model.predict(G.Batch.from_synth(b, device="cuda"), precision="fp64")
