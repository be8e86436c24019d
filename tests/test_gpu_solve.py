"""GPU parity of the regularised least-squares fit (Eqs. 4-9) against the
oracle's QR solve, and a full fit (K_NM assembly + solve) on the GPU against
the same fit done by the oracle."""
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


@pytest.mark.parametrize("method", ["householder", "cholqr_tc"])
def test_solve_matches_oracle_qr(G, method):
    soap_o, model_o, sparse, alpha = oracle_model(0, 40)
    w = S.workload(0)
    soap = G.Soap.from_spec(w.soap)
    model = G.Model(soap, sparse, alpha, w.delta, w.zeta)
    rng = np.random.default_rng(3)
    R = 300
    K = rng.normal(size=(R, 40))
    y = rng.normal(size=R)
    sig = rng.uniform(0.05, 0.5, size=R)
    Kmm = O.kmm(model_o, soap_o.dim)
    ref = O.solve_qr(K, y, sig, Kmm, 1e-8)
    got = model.solve(K, y, sig, jitter=1e-8, method=method)
    assert np.abs(got - ref).max() <= 1e-8 * np.abs(ref).max()
    import torch
    got_d = model.solve(torch.as_tensor(K, device="cuda"), torch.as_tensor(y, device="cuda"),
                        torch.as_tensor(sig, device="cuda"), jitter=1e-8, method=method).cpu().numpy()
    assert np.abs(got_d - ref).max() <= 1e-8 * np.abs(ref).max()


@pytest.mark.parametrize("method", ["householder", "cholqr_tc"])
def test_full_fit_matches_oracle_fit(G, method):
    """Targets from a teacher model; K_NM and the solve on the GPU (FP64)
    against K_NM and the QR solve of the oracle; then the fitted models
    predict held-out cells identically."""
    soap_o, teacher_o, sparse, alpha = oracle_model(1, 24, n_cells=1)
    w = S.workload(1)
    cells = S.structures(1, 3)
    # oracle fit
    Ks, ys, sg = [], [], []
    for c in cells:
        Ks.append(O.knm(soap_o, teacher_o, c))
        E, _, F, _ = O.predict(soap_o, teacher_o, c)
        ys.append(np.concatenate([[E], F.reshape(-1)]))
        sg.append(np.concatenate([[1e-3 * np.sqrt(c.n)], np.full(3 * c.n, 0.1)]))
    K_o, y_o, s_o = np.concatenate(Ks), np.concatenate(ys), np.concatenate(sg)
    a_o = O.solve_qr(K_o, y_o, s_o, O.kmm(teacher_o, soap_o.dim), 1e-8)
    # GPU fit on the same targets
    soap = G.Soap.from_spec(w.soap)
    teacher = G.Model(soap, sparse, alpha, w.delta, w.zeta)
    b = G.Batch.from_synth(S.make_batch(cells))
    K_g = teacher.assemble_knm(b, precision="fp64")
    a_g = teacher.solve(K_g, y_o, s_o, jitter=1e-8, method=method)
    assert np.abs(K_g - K_o).max() <= 1e-9 * np.abs(K_o).max()
    held = S.displaced_diamond(1, 900, (2, 2, 2), 0.1)
    st_o = O.Model(sparse, [a_o], w.delta, w.zeta)
    E_o, _, F_o, _ = O.predict(soap_o, st_o, held)
    st_g = G.Model(soap, sparse, [a_g], w.delta, w.zeta)
    out = st_g.predict(G.Batch.from_synth(S.make_batch([held])), precision="fp64")
    assert abs(out["energy"][0] - E_o) <= 1e-6 * held.n
    assert np.abs(out["forces"] - F_o).max() <= 1e-6


@pytest.mark.parametrize("device", [False, True])
def test_fused_fit_matches_assemble_then_solve(G, device):
    """gap_fit (K_NM kept on the device, coefficients installed in the model)
    gives the coefficients of gap_assemble_knm + gap_solve on the same data,
    with host and with device arrays, and the model then predicts with them."""
    import torch
    _, _, sparse, alpha = oracle_model(1, 24, n_cells=1)
    w = S.workload(1)
    cells = S.structures(1, 3)
    soap = G.Soap.from_spec(w.soap)
    ref_model = G.Model(soap, sparse, alpha, w.delta, w.zeta)
    b = G.Batch.from_synth(S.make_batch(cells))
    rows = b.n_configs + 3 * b.n_atoms
    rng = np.random.default_rng(7)
    y = rng.normal(size=rows)
    sig = rng.uniform(0.05, 0.5, size=rows)
    K = ref_model.assemble_knm(b, precision="bf16x3")
    a_ref = ref_model.solve(K, y, sig, jitter=1e-8, method="cholqr_tc")
    model = G.Model(soap, sparse, alpha, w.delta, w.zeta)
    if device:
        bd = G.Batch.from_synth(S.make_batch(cells), device="cuda")
        a = model.fit(bd, torch.as_tensor(y, device="cuda"), torch.as_tensor(sig, device="cuda"), jitter=1e-8,
                      method="cholqr_tc", precision="bf16x3").cpu().numpy()
    else:
        a = model.fit(b, y, sig, jitter=1e-8, method="cholqr_tc", precision="bf16x3")
    assert np.abs(a - a_ref).max() <= 1e-10 * np.abs(a_ref).max()
    ref_model.set_alpha(a_ref)
    held = G.Batch.from_synth(S.make_batch([S.displaced_diamond(1, 901, (2, 2, 2), 0.1)]))
    o1 = ref_model.predict(held, precision="fp64")
    o2 = model.predict(held, precision="fp64")
    assert np.abs(o1["forces"] - o2["forces"]).max() <= 1e-9
    assert abs(o1["energy"][0] - o2["energy"][0]) <= 1e-9 * max(1.0, abs(o1["energy"][0]))


def test_singular_kmm(G):
    """Repeated sparse points make K_MM singular.  The Householder method
    needs U = chol(K_MM + jitter) and reports GAP_ENOTPD; CholeskyQR uses
    K_MM only through A^T A = K^T S^-1 K + K_MM, which the data rows keep
    positive definite, and returns the regularised least-squares solution
    (Eq. 4 written out)."""
    soap_o, model_o, sparse, alpha = oracle_model(0, 8)
    w = S.workload(0)
    soap = G.Soap.from_spec(w.soap)
    dup = [np.concatenate([sparse[0], sparse[0]])]          # repeated sparse points: K_MM singular
    model = G.Model(soap, dup, [np.concatenate([alpha[0], alpha[0]])], w.delta, w.zeta)
    rng = np.random.default_rng(1)
    K = rng.normal(size=(50, 16))
    y = rng.normal(size=50)
    with pytest.raises(G.GapError) as e:
        model.solve(K, y, np.ones(50), jitter=0.0, method="householder")
    assert e.value.status == -5
    got = model.solve(K, y, np.ones(50), jitter=0.0, method="cholqr_tc")
    Kmm = O.kmm(O.Model(dup, [np.zeros(16)], w.delta, w.zeta), soap_o.dim)
    ref = np.linalg.solve(K.T @ K + Kmm, K.T @ y)
    assert np.abs(got - ref).max() <= 1e-8 * np.abs(ref).max()


def _fit_system(K, y, sig, Kmm, jitter):
    """The stacked least-squares system [S^-1/2 K ; U], [S^-1/2 y ; 0] (Eqs. 5-9)."""
    U = np.linalg.cholesky(Kmm + jitter * np.eye(Kmm.shape[0])).T
    A = np.vstack([K / sig[:, None], U])
    b = np.concatenate([y / sig, np.zeros(U.shape[0])])
    return A, b


def test_ill_conditioned_fit_system(G):
    """Six strained cells, M = 2000 sparse points, jitter 1e-8: cond(A) ~ 1e10.
    alpha itself is ill-determined at this conditioning, so both solves are
    compared through what the fit fixes: the fitted values A alpha (the
    projection of b onto the range of A) and the residual norm, against the
    oracle's Householder QR."""
    soap_o, model_o, sparse, alpha = oracle_model(1, 2000)
    w = S.workload(1)
    cells = S.structures(1, 6)
    K = np.concatenate([O.knm(soap_o, model_o, c) for c in cells])
    rng = np.random.default_rng(17)
    y = rng.normal(size=K.shape[0]) + K @ alpha[0]
    sig = np.concatenate([np.r_[1e-3 * np.sqrt(c.n), np.full(3 * c.n, 0.1)] for c in cells])
    Kmm = O.kmm(model_o, soap_o.dim)
    ref = O.solve_qr(K, y, sig, Kmm, 1e-8)
    A, b = _fit_system(K, y, sig, Kmm, 1e-8)
    fit_ref = A @ ref
    soap = G.Soap.from_spec(w.soap)
    model = G.Model(soap, sparse, alpha, w.delta, w.zeta)
    for method in ("householder", "cholqr_tc"):
        a = model.solve(K, y, sig, jitter=1e-8, method=method)
        fit = A @ a
        assert np.linalg.norm(fit - fit_ref) <= 1e-6 * np.linalg.norm(b), method
        assert abs(np.linalg.norm(b - fit) - np.linalg.norm(b - fit_ref)) <= 1e-9 * np.linalg.norm(b), method
