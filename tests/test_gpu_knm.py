"""GPU parity of the K_NM rows (energy rows and force rows of L_hat K_NM,
text after Eq. 4) against the FP64 oracle, through the C-ABI."""
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


def _as_np(x):
    return x.cpu().numpy() if hasattr(x, "cpu") else x


def _oracle_rows(soap_o, model_o, cells):
    return np.concatenate([O.knm(soap_o, model_o, c) for c in cells])


@pytest.fixture(scope="module")
def c2(G):
    soap_o, model_o, sparse, alpha = oracle_model(1, 48, n_cells=1)
    cells = S.structures(1, 3)
    ref = _oracle_rows(soap_o, model_o, cells)
    w = S.workload(1)
    soap = G.Soap.from_spec(w.soap)
    model = G.Model(soap, sparse, alpha, w.delta, w.zeta)
    return soap_o, model_o, model, cells, ref


def _check(K, ref, cells, rel):
    scale_e = np.abs(ref).max()
    assert K.shape == ref.shape
    assert np.abs(K - ref).max() <= rel * scale_e
    # energy rows separately (they are large): relative to their own size
    r = 0
    for c in cells:
        assert np.abs(K[r] - ref[r]).max() <= rel * max(1.0, np.abs(ref[r]).max())
        r += 1 + 3 * c.n


@pytest.mark.parametrize("prec,rel", [("fp64", 1e-9), ("fp32", 2e-5), ("bf16x3", 5e-5), ("bf16x6", 2e-5)])
def test_knm_parity_strained_cells(G, c2, prec, rel):
    _, _, model, cells, ref = c2
    K = _as_np(model.assemble_knm(G.Batch.from_synth(S.make_batch(cells), device="cuda"), precision=prec))
    _check(K, ref, cells, rel)


def test_knm_times_alpha_equals_predict(G, c2):
    """Column sums against alpha reproduce the model's own energies and forces."""
    _, _, model, cells, _ = c2
    b = G.Batch.from_synth(S.make_batch(cells), device="cuda")
    alpha = np.concatenate(model._al)
    for prec, tol in (("fp64", 1e-8), ("bf16x3", 1e-4), ("bf16x6", 1e-4)):
        K = _as_np(model.assemble_knm(b, precision=prec))
        out = model.predict(b, precision=prec)
        E, F = _as_np(out["energy"]), _as_np(out["forces"])
        r, a = 0, 0
        for k, c in enumerate(cells):
            assert abs(K[r] @ alpha - E[k]) <= tol * c.n
            assert np.abs((K[r + 1:r + 1 + 3 * c.n] @ alpha).reshape(-1, 3) - F[a:a + c.n]).max() <= tol
            r += 1 + 3 * c.n
            a += c.n


def test_knm_host_pointers(G, c2):
    _, _, model, cells, ref = c2
    K = model.assemble_knm(G.Batch.from_synth(S.make_batch(cells)), precision="fp64")
    _check(K, ref, cells, 1e-9)


def test_knm_mixed_species(G):
    soap_o, model_o, sparse, alpha = oracle_model(3, 10, n_cells=1)
    cells = S.structures(3, 2)
    ref = _oracle_rows(soap_o, model_o, cells)
    w = S.workload(3)
    soap = G.Soap.from_spec(w.soap)
    model = G.Model(soap, sparse, alpha, w.delta, w.zeta)
    b = G.Batch.from_synth(S.make_batch(cells), device="cuda")
    for prec, rel in (("fp64", 1e-9), ("bf16x3", 5e-5)):
        _check(_as_np(model.assemble_knm(b, precision=prec)), ref, cells, rel)
