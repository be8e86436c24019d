"""Predictive variances of local energies (Sec. 3.1.2) through the C-ABI,
against the FP64 oracle's posterior variance.  The GPU keeps the posterior
factors from its own FP64 K_NM of the training cells (gap_assemble_knm);
the oracle uses its own K_NM of the same cells; both use the oracle's
sparse points and the same sigma and jitter."""
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


def _sigma(cells):
    return np.concatenate([np.concatenate([[0.001 * np.sqrt(c.n)], np.full(3 * c.n, 0.1)]) for c in cells])


def _case(G, index, M, train, probe, tol):
    soap_o, model_o, sparse, alpha = oracle_model(index, M)
    w = S.workload(index)
    soap = G.Soap.from_spec(w.soap)
    model = G.Model(soap, sparse, alpha, w.delta, w.zeta)
    sig = _sigma(train)
    K = model.assemble_knm(G.Batch.from_synth(S.make_batch(train), device="cuda"), precision="fp64")
    import torch
    model.set_posterior(K, torch.as_tensor(sig, device="cuda"), jitter=1e-8)
    K_o = np.concatenate([O.knm(soap_o, model_o, c) for c in train])
    d2 = w.delta ** 2
    for c in probe:
        ref = O.predict_variance(soap_o, model_o, c, K_o, sig, 1e-8)
        got = model.predict_variance(G.Batch.from_synth(S.make_batch([c]), device="cuda")).cpu().numpy()
        host = model.predict_variance(G.Batch.from_synth(S.make_batch([c])))
        assert np.array_equal(got, host)
        assert (got >= -1e-9 * d2).all() and (got <= d2 * (1 + 1e-9)).all()
        assert np.abs(got - ref).max() <= tol * d2, np.abs(got - ref).max()
    return model


def test_variance_small_fit_matches_oracle(G):
    train = [S.displaced_diamond(0, 600 + c, (1, 1, 2), 0.15) for c in range(4)]
    probe = [S.displaced_diamond(0, 700, (2, 2, 2), 0.1), S.displaced_diamond(0, 701, (1, 2, 2), 0.3)]
    _case(G, 0, 60, train, probe, 1e-8)


def test_variance_multispecies_blocks_match_oracle(G):
    """Four GPs (one per central species, compressed SOAP, D 1008): the
    block structure of U^-1 and the rows of R^-1 of each GP."""
    cells = S.structures(3)
    small = sorted(range(len(cells)), key=lambda k: cells[k].n)
    train = [cells[k] for k in small[:6]]
    probe = [cells[k] for k in small[6:8]]
    _case(G, 3, 40, train, probe, 1e-8)


def test_variance_fit_workload_scale(G):
    """M = 2000 sparse points and 20 cells of the fit workload (cond(A) of the
    order of the bench's fit): two probe cells of the batch."""
    cells = S.structures(1, 22)
    _case(G, 1, 2000, cells[:20], cells[20:22], 1e-6)


def test_variance_needs_a_posterior(G):
    _, _, sparse, alpha = oracle_model(0, 20)
    w = S.workload(0)
    soap = G.Soap.from_spec(w.soap)
    model = G.Model(soap, sparse, alpha, w.delta, w.zeta)
    with pytest.raises(G.GapError) as ei:
        model.predict_variance(G.Batch.from_synth(S.make_batch(S.structures(0)), device="cuda"))
    assert ei.value.status == -1
