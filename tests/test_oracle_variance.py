"""Pins of the oracle's predictive variance of a local energy (the
variances gp_predict returns, Sec. 3.1.2), read as the posterior variance of
the sparse GP of Eq. 4:
    var(x) = k(x, x) - k_x^T Kt^-1 k_x + k_x^T (A^T A)^-1 k_x.
The pins do not restate that formula: the kernel row against the C oracle's
local energies, the prior with no data, the textbook full-GP posterior when
the sparse points are themselves the observed points, monotone decrease as
data are added, and non-negativity on a fit with force rows."""
import numpy as np
import pytest

import oracle as O
from paper_2310_03921_gb300 import synth as S
from _models import oracle_model


@pytest.fixture(scope="module")
def setup():
    soap, model, sparse, alpha = oracle_model(0, 60)
    cells = [S.displaced_diamond(0, 500 + c, (1, 1, 2), 0.15) for c in range(3)]
    return soap, model, cells


def test_kernel_rows_reproduce_local_energies(setup):
    soap, model, cells = setup
    k, kxx = O.kernel_rows(soap, model, cells[0])
    _, le, _, _ = O.predict(soap, model, cells[0])
    assert np.abs(k @ model.alpha - le).max() <= 1e-12 * max(1.0, np.abs(le).max())
    assert np.allclose(kxx, model.c.delta ** 2, rtol=0, atol=1e-13)  # p_hat is normalised


def test_no_data_gives_the_prior(setup):
    soap, model, cells = setup
    var = O.predict_variance(soap, model, cells[1], np.zeros((0, 60)), np.zeros(0), 1e-8)
    assert np.allclose(var, model.c.delta ** 2, rtol=0, atol=1e-7)


def _diverse_model(M=8, zeta=2):
    """Sparse points from environments as different as the workloads have
    (diamond cells with large displacements, random packings), so that
    K_MM is well conditioned."""
    w = S.workload(0)
    soap = O.Soap(w.soap.n_max, w.soap.l_max, w.soap.rc, w.soap.sigma, w.soap.d)
    pool = np.concatenate([O.descriptor(soap, S.displaced_diamond(0, 900 + c, (1, 1, 1), 0.45))[0]
                           for c in range(4)])
    idx = S.SplitMix64(123).choice(pool.shape[0], M)
    X = pool[idx]
    return soap, O.Model([X], [np.zeros(M)], 1.3, zeta)


def test_sparse_points_observed_directly_is_the_full_gp():
    """When the observed data are the local energies at the sparse points
    themselves (K_NM = K_MM, noise sigma_n, no jitter), the sparse posterior
    is the exact GP posterior: var(x) = k(x,x) - k^T (K + sigma_n^2 I)^-1 k."""
    soap, model = _diverse_model()
    K = O.kmm(model, soap.dim)
    assert np.linalg.cond(K) < 1e8
    s = S.displaced_diamond(0, 77, (1, 1, 1), 0.3)
    for sn in (0.3, 0.05):
        var = O.predict_variance(soap, model, s, K, np.full(K.shape[0], sn), 0.0)
        k, kxx = O.kernel_rows(soap, model, s)
        ref = kxx - np.einsum("ij,ij->i", k, np.linalg.solve(K + sn ** 2 * np.eye(K.shape[0]), k.T).T)
        assert np.abs(var - ref).max() <= 1e-9 * kxx.max()


def test_variance_decreases_as_data_are_added(setup):
    soap, model, cells = setup
    K = [O.knm(soap, model, c) for c in cells]
    sig = [np.concatenate([[0.001 * np.sqrt(c.n)], np.full(3 * c.n, 0.1)]) for c in cells]
    probe = S.displaced_diamond(0, 640, (1, 1, 2), 0.15)
    v1 = O.predict_variance(soap, model, probe, K[0], sig[0], 1e-8)
    v2 = O.predict_variance(soap, model, probe, np.vstack(K[:2]), np.concatenate(sig[:2]), 1e-8)
    v3 = O.predict_variance(soap, model, probe, np.vstack(K), np.concatenate(sig), 1e-8)
    d2 = model.c.delta ** 2
    assert (v2 <= v1 + 1e-9 * d2).all() and (v3 <= v2 + 1e-9 * d2).all()
    assert (v3 < v1).any()
    assert (v3 >= -1e-9 * d2).all() and (v1 <= d2 + 1e-9).all()
