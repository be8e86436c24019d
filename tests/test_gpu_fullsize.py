"""Parity at the workloads' full sizes, in the launch configuration bench.py
times (device pointers, the BF16X3 tensor-core form), on outputs the FP64
oracle computes one by one: sampled atoms of the large cells, sampled cells
of the batches.  The models' sparse points are the oracle's own descriptors
of the seeded candidate cells."""
import numpy as np
import pytest

import oracle as O
from paper_2310_03921_gb300 import synth as S
from _models import oracle_model

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_2310_03921_gb300 import build, gap
    build.build()
    return gap


def _gpu_model(G, index, sparse, alpha):
    w = S.workload(index)
    soap = G.Soap.from_spec(w.soap)
    return soap, G.Model(soap, sparse, alpha, w.delta, w.zeta, two_body=w.two_body)


def _np(x):
    return x.cpu().numpy() if hasattr(x, "cpu") else x


def test_fit_workload_knm_rows_and_forces(G):
    """200 cells, M = 2000: K_NM rows of two sampled cells against the oracle,
    K_NM alpha against the model's own predict for all 200, E+F of the samples."""
    soap_o, model_o, sparse, alpha = oracle_model(1, 2000)
    cells = S.structures(1)
    soap, model = _gpu_model(G, 1, sparse, alpha)
    b = G.Batch.from_synth(S.make_batch(cells), device="cuda")
    K = _np(model.assemble_knm(b, precision="bf16x3"))
    out = model.predict(b, precision="bf16x3")
    E, F = _np(out["energy"]), _np(out["forces"])
    a = np.concatenate(alpha)
    starts = np.concatenate([[0], np.cumsum([1 + 3 * c.n for c in cells])])
    aoff = np.concatenate([[0], np.cumsum([c.n for c in cells])])
    assert np.abs(K[starts[:-1]] @ a - E).max() <= 1e-3
    assert np.abs((K[np.setdiff1d(np.arange(K.shape[0]), starts[:-1])] @ a).reshape(-1, 3) - F).max() <= 1e-4
    for c in (7, 151):
        ref = O.knm(soap_o, model_o, cells[c])
        got = K[starts[c]:starts[c + 1]]
        assert np.abs(got - ref).max() <= 5e-5 * np.abs(ref).max()
        Eo, leo, Fo, _ = O.predict(soap_o, model_o, cells[c])
        assert np.abs(F[aoff[c]:aoff[c + 1]] - Fo).max() <= 1e-4
        assert abs(E[c] - Eo) <= 1e-4 * cells[c].n


def test_md_cell_32768_sampled_atoms(G):
    soap_o, model_o, sparse, alpha = oracle_model(2, 4000)
    s = S.structures(2)[0]
    soap, model = _gpu_model(G, 2, sparse, alpha)
    out = model.predict(G.Batch.from_synth(S.make_batch([s]), device="cuda"), precision="bf16x3")
    le, F = _np(out["local_e"]), _np(out["forces"])
    sel = np.sort(S.SplitMix64(77).choice(s.n, 24))
    le_o, F_o = O.predict_sampled(soap_o, model_o, s, sel)
    assert np.abs(F[sel] - F_o).max() <= 1e-4
    assert np.abs(le[sel] - le_o).max() <= 1e-4
    assert np.abs(F.sum(0)).max() <= 1e-6 * s.n


def test_multispecies_batch_512_sampled_configs(G):
    soap_o, model_o, sparse, alpha = oracle_model(3, 3000)
    cells = S.structures(3)
    soap, model = _gpu_model(G, 3, sparse, alpha)
    out = model.predict(G.Batch.from_synth(S.make_batch(cells), device="cuda"), precision="bf16x3")
    E, F = _np(out["energy"]), _np(out["forces"])
    aoff = np.concatenate([[0], np.cumsum([c.n for c in cells])])
    for c in (0, 300, 511):
        Eo, _, Fo, _ = O.predict(soap_o, model_o, cells[c])
        assert np.abs(F[aoff[c]:aoff[c + 1]] - Fo).max() <= 1e-4
        assert abs(E[c] - Eo) <= 1e-4 * cells[c].n


def test_amorphous_110592_with_two_body_sampled_atoms(G):
    """Diverse environments and forces up to ~80 eV/A (two-body term)."""
    soap_o, model_o, sparse, alpha = oracle_model(4, 9000)
    s = S.structures(4)[0]
    soap, model = _gpu_model(G, 4, sparse, alpha)
    out = model.predict(G.Batch.from_synth(S.make_batch([s]), device="cuda"), precision="bf16x3")
    le, F = _np(out["local_e"]), _np(out["forces"])
    sel = np.sort(S.SplitMix64(78).choice(s.n, 12))
    le_o, F_o = O.predict_sampled(soap_o, model_o, s, sel)
    assert np.abs(F[sel] - F_o).max() <= 1e-4
    assert np.abs(le[sel] - le_o).max() <= 1e-4


def _clusters(s, centres, radius, h):
    """For each centre atom a of a cubic periodic cell: the atoms within
    `radius` of it (minimum image), as a non-periodic configuration with a
    first, then the same configuration with a moved by +-h along x, y, z.
    Only atoms within r_c of a change their local energy when a moves, and
    their environments lie within 2 r_c of a, so with radius >= 2 r_c the
    cluster's energy has the periodic cell's gradient with respect to a."""
    L = s.cell[0, 0]
    assert np.allclose(s.cell, L * np.eye(3))
    box = 2.0 * radius + 12.0
    pos, spec, cell, pbc, offs = [], [], [], [], [0]
    for a in centres:
        d = s.pos - s.pos[a]
        d -= L * np.round(d / L)
        near = np.nonzero(np.einsum("ij,ij->i", d, d) < radius * radius)[0]
        near = np.concatenate([[a], near[near != a]])
        base = d[near] + box / 2
        for k in range(7):
            p = base.copy()
            if k:
                p[0, (k - 1) // 2] += h if k % 2 else -h
            pos.append(p)
            spec.append(s.species[near])
            cell.append(box * np.eye(3))
            pbc.append([0, 0, 0])
            offs.append(offs[-1] + near.size)
    return (np.concatenate(pos), np.concatenate(spec).astype(np.int32), np.stack(cell), np.array(pbc, np.int32),
            np.array(offs, np.int32))


def test_md_cell_32768_forces_match_finite_differences_on_64_atoms(G):
    """The 32768-atom cell (n_max 8, l_max 8, M 4000): forces of 64 seeded
    random atoms, from the full-cell predict in the split-BF16x3 form and in
    FP64, against central finite differences (h = 5e-5 A) of FP64 energies,
    each through the atom's local cluster of radius 2 r_c + 0.5 A (all 448
    displaced clusters in one batched call)."""
    import torch
    _, _, sparse, alpha = oracle_model(2, 4000)
    s = S.structures(2)[0]
    w = S.workload(2)
    soap, model = _gpu_model(G, 2, sparse, alpha)
    full = G.Batch.from_synth(S.make_batch([s]), device="cuda")
    F_tc = _np(model.predict(full, precision="bf16x3", virial=False)["forces"])
    F_64 = _np(model.predict(full, precision="fp64", virial=False)["forces"])
    sel = S.SplitMix64(S.seed_for(2, 0, "count")).choice(s.n, 64)
    h = 5e-5
    pos, spec, cell, pbc, offs = _clusters(s, sel, 2.0 * w.soap.rc + 0.5, h)
    b = G.Batch(torch.as_tensor(pos, device="cuda"), torch.as_tensor(spec, device="cuda"), cell, pbc, offs)
    E = _np(model.predict(b, precision="fp64", local=False, forces=False, virial=False)["energy"]).reshape(64, 7)
    F_fd = -(E[:, 1::2] - E[:, 2::2]) / (2 * h)
    assert np.abs(F_64[sel] - F_fd).max() <= 2e-6
    assert np.abs(F_tc[sel] - F_fd).max() <= 1e-4
