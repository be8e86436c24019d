"""The captured MD step (gap_step_graph): a CUDA graph of one predict of a
fixed batch layout.  Launches after moving the atoms in place must equal an
ordinary gap_predict of the new positions (the graph rebuilds the neighbour
lists inside), a launch whose positions exceed the pair capacity reports
GAP_ECAPACITY without touching memory outside the buffers, and the graph
recovers on the next launch."""
import numpy as np
import pytest

from paper_2310_03921_gb300 import synth as S
from _models import oracle_model

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import torch

    from paper_2310_03921_gb300 import build, gap
    build.build()
    _, _, sparse, alpha = oracle_model(0, 100)
    w = S.workload(0)
    soap = gap.Soap.from_spec(w.soap)
    model = gap.Model(soap, sparse, alpha, w.delta, w.zeta)
    cells = [S.structures(0)[0], S.displaced_diamond(0, 91, (1, 1, 1), 0.1)]
    return torch, gap, model, S.make_batch(cells)


def _same(out, ref, atol):
    import torch
    for k in ("energy", "forces", "virial"):
        assert torch.allclose(out[k], ref[k], rtol=0, atol=atol), k


@pytest.mark.parametrize("prec,atol", [("fp64", 1e-12), ("bf16x3", 1e-9)])
def test_graph_steps_match_predict(setup, prec, atol):
    torch, gap, model, b = setup
    batch = gap.Batch.from_synth(b, device="cuda")
    g = gap.StepGraph(model, batch, precision=prec, pair_capacity=1.3)
    assert g.kernels > 10
    rng = np.random.default_rng(4)
    for step in range(3):
        batch.pos.add_(torch.as_tensor(rng.normal(scale=0.03, size=b.pos.shape), device="cuda"))
        n0 = gap.launch_count()
        g.launch()
        g.status()
        assert gap.launch_count() - n0 == g.kernels
        ref = model.predict(gap.Batch(batch.pos.clone(), batch.species, b.cell, b.pbc, b.config_offsets),
                            precision=prec)
        _same(g.outputs, ref, atol)
    g.close()


def test_graph_sees_new_coefficients(setup):
    torch, gap, model, b = setup
    batch = gap.Batch.from_synth(b, device="cuda")
    g = gap.StepGraph(model, batch, precision="fp64")
    a0 = np.concatenate(model._al)
    try:
        model.set_alpha(2.0 * a0)
        g.launch()
        g.status()
        ref = model.predict(batch, precision="fp64")
        _same(g.outputs, ref, 1e-12)
    finally:
        model.set_alpha(a0)
        g.close()


def test_pair_capacity_overflow_is_reported_and_recoverable(setup):
    torch, gap, model, b = setup
    batch = gap.Batch.from_synth(b, device="cuda")
    g = gap.StepGraph(model, batch, precision="bf16x3", pair_capacity=1.0)
    ref = model.predict(batch, precision="bf16x3")
    saved = batch.pos.clone()
    # squeeze the first cell's atoms into one octant: many more pairs
    n0 = int(b.config_offsets[1])
    batch.pos[:n0].mul_(0.5)
    g.launch()
    with pytest.raises(gap.GapError) as e:
        g.status()
    assert e.value.status == -7
    batch.pos.copy_(saved)
    g.launch()
    g.status()
    _same(g.outputs, ref, 1e-9)
    g.close()


def test_graph_rejects_host_batches(setup):
    _, gap, model, b = setup
    with pytest.raises(ValueError):
        gap.StepGraph(model, gap.Batch.from_synth(b))
