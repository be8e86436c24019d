"""Compressed descriptors (Sec. 3.3.3 tensor sketch and decomposition,
nu_R / nu_S correlation orders; the soap_turbo recipes of Sec. 3.3.4) on the
GPU through the C-ABI: the descriptors against the oracle's recipes written
from their definitions, the local energies against the oracle's, the forces
and virial of the library's backward kernels against central finite
differences of the oracle's energy (in positions and in strain), in FP64 and
in the split-BF16x3 form; and the K_NM rows of fitting (text after Eq. 4) on
compressed descriptors: energy rows against the oracle's kernel values,
force rows against central differences of those, and K_NM alpha against the
model's own energies and forces."""
import numpy as np
import pytest

import oracle as O
from paper_2310_03921_gb300 import synth as S

pytestmark = pytest.mark.gpu

RNG = np.random.default_rng(2024)
COMPS = {
    "sketch": dict(recipe="sketch", w=RNG.normal(size=(5, 8)), u=RNG.normal(size=(5, 8))),
    "decomposition": dict(recipe="decomposition", w=RNG.normal(size=(6, 8))),
    "nu11": dict(recipe="nu", nu_S=1, nu_R=1),
    "nu02": dict(recipe="nu", nu_S=0, nu_R=2),
    "nu20": dict(recipe="nu", nu_S=2, nu_R=0),
    "trivial": dict(recipe="trivial"),
    "matrix": dict(recipe="matrix", P=RNG.normal(size=(20, 144))),
}


@pytest.fixture(scope="module")
def G():
    from paper_2310_03921_gb300 import build, gap
    build.build()
    return gap


def _cell(seed, reps=(1, 1, 2), sig=0.15):
    s = S.displaced_diamond(0, seed, reps, sig)
    sp = S.SplitMix64(seed).integers(s.n, 0, 1).astype(np.int32)
    return S.Structure(s.pos, sp, s.cell, s.pbc)


def _pair(G, comp):
    so = O.Soap(4, 3, 5.0, 0.5, 1.0, n_species=2)
    sg = G.Soap(4, 3, 5.0, 0.5, 1.0, 1.0, 2)
    kw = {k: v for k, v in comp.items() if k != "recipe"}
    sg.set_compression(comp["recipe"], **kw)
    return so, sg


@pytest.mark.parametrize("name", list(COMPS))
def test_compressed_descriptor_matches_oracle(G, name):
    comp = COMPS[name]
    so, sg = _pair(G, comp)
    s = _cell(11)
    ref = O.compressed_descriptor(so, s, comp)
    assert sg.dim == ref.shape[1]
    b = G.Batch.from_synth(S.make_batch([s]), device="cuda")
    d64 = sg.descriptor(b, precision="fp64").cpu().numpy()
    d32 = sg.descriptor(b, precision="bf16x3").cpu().numpy()
    assert np.abs(d64 - ref).max() <= 1e-10
    assert np.abs(d32 - ref).max() <= 3e-5


def _model(G, so, sg, comp, M=24):
    pool = np.concatenate([O.compressed_descriptor(so, _cell(300 + c), comp) for c in range(4)])
    spec = np.concatenate([_cell(300 + c).species for c in range(4)])
    sparse, alpha = [], []
    for z in range(2):
        cand = pool[spec == z]
        idx = S.SplitMix64(S.seed_for(0, z, "sparse")).choice(cand.shape[0], min(M, cand.shape[0]))
        sparse.append(cand[idx])
        alpha.append(S.alpha_draw(0, z, idx.size))
    return O.Model(sparse, alpha, 1.0, 4), G.Model(sg, sparse, alpha, 1.0, 4)


def _energy(so, comp, mo, s):
    return O.compressed_local_energies(so, comp, mo, s).sum()


@pytest.mark.parametrize("name", ["sketch", "nu11", "trivial", "matrix"])
def test_compressed_energies_forces_virial(G, name):
    comp = COMPS[name]
    so, sg = _pair(G, comp)
    mo, mg = _model(G, so, sg, comp)
    s = _cell(12)
    le_ref = O.compressed_local_energies(so, comp, mo, s)
    h = 1e-4
    F_fd = np.zeros((s.n, 3))
    for i in range(s.n):
        for x in range(3):
            e = []
            for sgn in (1, -1):
                pos = s.pos.copy()
                pos[i, x] += sgn * h
                e.append(_energy(so, comp, mo, S.Structure(pos, s.species, s.cell, s.pbc)))
            F_fd[i, x] = -(e[0] - e[1]) / (2 * h)
    # virial V_ab = -dE/d e_ab for r -> (I + e) r (symmetric strain pairs)
    V_fd = np.zeros((3, 3))
    for a in range(3):
        for c in range(3):
            e = []
            for sgn in (1, -1):
                eps = np.eye(3)
                eps[a, c] += sgn * h
                e.append(_energy(so, comp, mo, S.Structure(s.pos @ eps.T, s.species, s.cell @ eps.T, s.pbc)))
            V_fd[a, c] = -(e[0] - e[1]) / (2 * h)
    b = G.Batch.from_synth(S.make_batch([s]), device="cuda")
    for prec, tol_e, tol_f in (("fp64", 1e-9, 2e-6), ("bf16x3", 2e-5, 1e-4)):
        out = mg.predict(b, precision=prec)
        le, F, V = (out[k].cpu().numpy() for k in ("local_e", "forces", "virial"))
        assert np.abs(le - le_ref).max() <= tol_e, (prec, np.abs(le - le_ref).max())
        assert np.abs(F - F_fd).max() <= tol_f, (prec, np.abs(F - F_fd).max())
        assert np.abs(V[0] - V_fd).max() <= 10 * tol_f * s.n, (prec, np.abs(V[0] - V_fd).max())


def test_compression_step_graph_and_limits(G):
    comp = COMPS["sketch"]
    so, sg = _pair(G, comp)
    mo, mg = _model(G, so, sg, comp)
    s = _cell(13)
    b = G.Batch.from_synth(S.make_batch([s]), device="cuda")
    ref = mg.predict(b, precision="bf16x3", local=False)
    graph = G.StepGraph(mg, b, precision="bf16x3")
    graph.launch()
    graph.status()
    assert np.array_equal(graph.outputs["forces"].cpu().numpy(), ref["forces"].cpu().numpy())
    # no change while a model holds the object
    with pytest.raises(G.GapError) as ei:
        sg.set_compression("trivial")
    assert ei.value.status == -1
    # the mixed (element-embedded) descriptor is not a compression target
    sm = G.Soap(4, 3, 5.0, 0.5, 1.0, 1.0, 4, 2, RNG.normal(size=(2, 4)))
    with pytest.raises(G.GapError):
        sm.set_compression("trivial")


def _energy_rows(so, comp, mo, s):
    """Energy row of one structure on compressed descriptors: sum over atoms
    of delta^2 (p~_i . x_m)^zeta for the sparse points of the atom's GP."""
    ph = O.compressed_descriptor(so, s, comp)
    d2, z = mo.c.delta ** 2, mo.c.zeta
    row = np.zeros(int(mo.offsets[-1]))
    for i in range(ph.shape[0]):
        g = int(s.species[i])
        a, b = int(mo.offsets[g]), int(mo.offsets[g + 1])
        row[a:b] += d2 * (mo.sparse[a:b] @ ph[i]) ** z
    return row


def _knm_fd(so, comp, mo, s, h=1e-4):
    """[1 + 3n][M] rows of one structure: the energy row, then the force rows
    -d(energy row)/d r_ja by central differences of the oracle."""
    rows = [_energy_rows(so, comp, mo, s)]
    for j in range(s.n):
        for x in range(3):
            e = []
            for sgn in (1, -1):
                pos = s.pos.copy()
                pos[j, x] += sgn * h
                e.append(_energy_rows(so, comp, mo, S.Structure(pos, s.species, s.cell, s.pbc)))
            rows.append(-(e[0] - e[1]) / (2 * h))
    return np.array(rows)


@pytest.mark.parametrize("name", list(COMPS))
def test_compressed_knm_rows(G, name):
    comp = COMPS[name]
    so, sg = _pair(G, comp)
    mo, mg = _model(G, so, sg, comp)
    cells = [_cell(21), _cell(22, reps=(1, 1, 1))]
    ref = np.concatenate([_knm_fd(so, comp, mo, c) for c in cells])
    b = G.Batch.from_synth(S.make_batch(cells), device="cuda")
    alpha = np.concatenate(mg._al)
    E_rows = np.cumsum([0] + [1 + 3 * c.n for c in cells])[:-1]
    F_rows = np.setdiff1d(np.arange(ref.shape[0]), E_rows)
    scale = np.abs(ref[F_rows]).max()
    # fp64 force rows: the central differences' own O(h^2) error (about 3e-8)
    for prec, tol_e, tol_f, tol_p in (("fp64", 1e-11, 2e-7, 1e-12), ("fp32", 2e-6, 6e-6, 2e-6),
                                      ("bf16x3", 5e-5, 5e-5, 2e-5), ("bf16x6", 5e-6, 1e-5, 5e-6)):
        K = mg.assemble_knm(b, precision=prec)
        K = K.cpu().numpy() if hasattr(K, "cpu") else K
        assert K.shape == ref.shape
        err_e = np.abs(K[E_rows] - ref[E_rows]).max() / np.abs(ref[E_rows]).max()
        err_f = np.abs(K[F_rows] - ref[F_rows]).max() / scale
        assert err_e <= tol_e, (prec, err_e)
        assert err_f <= tol_f, (prec, err_f)
        out = mg.predict(b, precision=prec)
        E, F = out["energy"].cpu().numpy(), out["forces"].cpu().numpy()
        a = 0
        for k, c in enumerate(cells):
            r = E_rows[k]
            assert abs(K[r] @ alpha - E[k]) <= tol_p * c.n
            assert np.abs((K[r + 1:r + 1 + 3 * c.n] @ alpha).reshape(-1, 3) - F[a:a + c.n]).max() <= tol_p
            a += c.n
