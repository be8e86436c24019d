"""The differentiable energy (torch.autograd.Function around gap_predict):
gradients with respect to the positions are -F (Eq. 3), checked against
central finite differences of the energy on the GPU, against the oracle's
analytic forces, and for the chain rule through an upstream gradient; the
energy-only call (no gradient wanted) returns the same energies."""
import numpy as np
import pytest

import oracle as O
from paper_2310_03921_gb300 import synth as S
from _models import oracle_model

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import torch

    from paper_2310_03921_gb300 import build, gap
    build.build()
    soap_o, model_o, sparse, alpha = oracle_model(0, 100)
    w = S.workload(0)
    soap = gap.Soap.from_spec(w.soap)
    model = gap.Model(soap, sparse, alpha, w.delta, w.zeta)
    cells = [S.structures(0)[0], S.displaced_diamond(0, 77, (1, 1, 2), 0.1)]
    b = S.make_batch(cells)
    return torch, gap, soap_o, model_o, model, cells, b


def _pos(torch, b, grad=True):
    return torch.tensor(b.pos, dtype=torch.float64, device="cuda", requires_grad=grad)


def _args(torch, b):
    return (torch.as_tensor(b.species, dtype=torch.int32, device="cuda"), b.cell, b.pbc, b.config_offsets)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("bf16x3", 1e-9)])
def test_gradient_is_minus_forces(setup, prec, tol):
    torch, gap, _, _, model, _, b = setup
    pos = _pos(torch, b)
    E, V = gap.energy(model, pos, *_args(torch, b), precision=prec)
    (gpos,) = torch.autograd.grad(E.sum(), pos)
    ref = model.predict(gap.Batch.from_synth(b, device="cuda"), precision=prec)
    assert torch.equal(E, ref["energy"])
    assert torch.allclose(gpos, -ref["forces"], rtol=0, atol=tol)
    assert torch.allclose(V, ref["virial"], rtol=0, atol=tol)


def test_upstream_gradient_per_configuration(setup):
    torch, gap, _, _, model, cells, b = setup
    pos = _pos(torch, b)
    E, _ = gap.energy(model, pos, *_args(torch, b), precision="fp64")
    wts = torch.tensor([0.5, -2.0], dtype=torch.float64, device="cuda")
    (gpos,) = torch.autograd.grad((wts * E).sum(), pos)
    F = model.predict(gap.Batch.from_synth(b, device="cuda"), precision="fp64")["forces"]
    n0 = cells[0].n
    assert torch.allclose(gpos[:n0], 0.5 * -F[:n0], rtol=0, atol=1e-12)
    assert torch.allclose(gpos[n0:], -2.0 * -F[n0:], rtol=0, atol=1e-12)


def test_gradient_matches_finite_differences(setup):
    """Central differences of E (FP64 path, h = 1e-4 A) along random
    directions of single atoms against the autograd gradient."""
    torch, gap, _, _, model, _, b = setup
    args = _args(torch, b)
    pos = _pos(torch, b)
    E, _ = gap.energy(model, pos, *args, precision="fp64")
    (gpos,) = torch.autograd.grad(E.sum(), pos)
    rng = np.random.default_rng(11)
    h = 1e-4
    for atom in rng.choice(b.pos.shape[0], 6, replace=False):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        p = torch.tensor(b.pos, dtype=torch.float64, device="cuda")
        dd = torch.as_tensor(d, device="cuda")
        p[atom] += h * dd
        Ep, _ = gap.energy(model, p, *args, precision="fp64")
        p[atom] -= 2 * h * dd
        Em, _ = gap.energy(model, p, *args, precision="fp64")
        fd = float((Ep.sum() - Em.sum()) / (2 * h))
        assert abs(fd - float(gpos[atom] @ dd)) <= 1e-6


def test_gradient_matches_oracle_forces(setup):
    torch, gap, soap_o, model_o, model, cells, b = setup
    pos = _pos(torch, b)
    E, _ = gap.energy(model, pos, *_args(torch, b), precision="bf16x3")
    (gpos,) = torch.autograd.grad(E.sum(), pos)
    F_o = np.concatenate([O.predict(soap_o, model_o, c)[2] for c in cells])
    assert np.abs(-gpos.cpu().numpy() - F_o).max() <= 1e-4


def test_energy_only_without_gradient(setup):
    torch, gap, _, _, model, _, b = setup
    pos = _pos(torch, b, grad=False)
    E, V = gap.energy(model, pos, *_args(torch, b), precision="bf16x3")
    assert V is None and not E.requires_grad
    ref = model.predict(gap.Batch.from_synth(b, device="cuda"), precision="bf16x3")["energy"]
    assert torch.allclose(E, ref, rtol=0, atol=1e-9)


def test_soap_destroyed_before_model(setup):
    """A garbage collector may finalise the descriptor before the model built
    on it; the model keeps working and the release is deferred."""
    torch, gap, _, _, _, _, b = setup
    _, _, sparse, alpha = oracle_model(0, 100)
    w = S.workload(0)
    soap = gap.Soap.from_spec(w.soap)
    model = gap.Model(soap, sparse, alpha, w.delta, w.zeta)
    bb = gap.Batch.from_synth(b, device="cuda")
    ref = model.predict(bb, precision="fp64")["energy"].clone()
    soap.close()
    assert torch.equal(model.predict(bb, precision="fp64")["energy"], ref)
    model.close()
    fresh = gap.Soap.from_spec(w.soap)
    assert fresh.dim == soap_o_dim(w)


def soap_o_dim(w):
    return w.soap.n_max * (w.soap.n_max + 1) // 2 * (w.soap.l_max + 1)
