"""Every tile variant of the tensor-core contractions against the FP64
oracle.  The tile autotuner picks one of four column tiles per shape by
timing, so a run normally exercises only the winners; here each variant is
forced in turn (128 x 256 and 128 x 128 tiles with two or three TMA stages,
and 128 x 192 with twelve epilogue warps) and the split-BF16x3 K_NM rows
(text after Eq. 4) and predictions (Eq. 3, forces and virial by the chain
rule of Sec. 3.4) are checked against the oracle.  M = 300 sparse points
leave a ragged last column tile for every width, and 240 atoms / 722 K_NM
rows a ragged last row tile."""
import numpy as np
import pytest

import oracle as O
from paper_2310_03921_gb300 import synth as S
from _models import oracle_model

pytestmark = pytest.mark.gpu

VARIANTS = [0, 1, 2, 3]


@pytest.fixture(scope="module")
def G():
    from paper_2310_03921_gb300 import build, gap
    build.build()
    return gap


@pytest.fixture(scope="module")
def case(G):
    soap_o, model_o, sparse, alpha = oracle_model(1, 300, n_cells=3)
    assert sparse[0].shape[0] == 300
    cells = S.structures(1, 2)
    w = S.workload(1)
    soap = G.Soap.from_spec(w.soap)
    model = G.Model(soap, sparse, alpha, w.delta, w.zeta)
    knm = np.concatenate([O.knm(soap_o, model_o, c) for c in cells])
    pred = [O.predict(soap_o, model_o, c) for c in cells]
    return model, cells, knm, pred


def _np(x):
    return x.cpu().numpy() if hasattr(x, "cpu") else x


def _forced(G, v, fn):
    G.test_tc_force_variant(v)
    try:
        return fn()
    finally:
        G.test_tc_force_variant(-1)


@pytest.mark.parametrize("v", VARIANTS)
def test_knm_rows_every_variant(G, case, v):
    model, cells, ref, _ = case
    b = G.Batch.from_synth(S.make_batch(cells), device="cuda")
    K = _np(_forced(G, v, lambda: model.assemble_knm(b, precision="bf16x3")))
    assert K.shape == ref.shape
    assert np.abs(K - ref).max() <= 5e-5 * np.abs(ref).max()
    r = 0
    for c in cells:  # energy rows relative to their own size
        assert np.abs(K[r] - ref[r]).max() <= 5e-5 * max(1.0, np.abs(ref[r]).max())
        r += 1 + 3 * c.n


@pytest.mark.parametrize("v", VARIANTS)
def test_predict_every_variant(G, case, v):
    model, cells, _, pred = case
    b = G.Batch.from_synth(S.make_batch(cells), device="cuda")
    out = _forced(G, v, lambda: model.predict(b, precision="bf16x3"))
    E = np.array([p[0] for p in pred])
    le = np.concatenate([p[1] for p in pred])
    F = np.concatenate([p[2] for p in pred])
    V = np.stack([p[3] for p in pred])
    nat = np.array([c.n for c in cells])
    assert np.abs(_np(out["local_e"]) - le).max() <= 1e-4
    assert np.abs(_np(out["forces"]) - F).max() <= 1e-4
    assert np.all(np.abs(_np(out["energy"]) - E) <= 1e-4 * nat)
    assert np.abs(_np(out["virial"]) - V).max() <= 1e-3 * max(1.0, np.abs(V).max())


def test_variants_agree_with_each_other(G, case):
    """The element-wise outputs do not depend on the tile: K_NM rows and forces
    of all variants within FP32 rounding of one another."""
    model, cells, _, _ = case
    b = G.Batch.from_synth(S.make_batch(cells), device="cuda")
    Ks, Fs = [], []
    for v in VARIANTS:
        Ks.append(_np(_forced(G, v, lambda: model.assemble_knm(b, precision="bf16x3"))))
        Fs.append(_np(_forced(G, v, lambda: model.predict(b, precision="bf16x3"))["forces"]))
    for K, F in zip(Ks[1:], Fs[1:]):
        assert np.abs(K - Ks[0]).max() <= 1e-6 * np.abs(Ks[0]).max()
        assert np.abs(F - Fs[0]).max() <= 1e-6 * max(1.0, np.abs(Fs[0]).max())


def test_force_variant_rejects_out_of_range(G):
    with pytest.raises(Exception):
        G.test_tc_force_variant(4)
    G.test_tc_force_variant(-1)
