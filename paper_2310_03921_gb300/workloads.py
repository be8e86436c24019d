"""Workload construction on the GPU path (sparse sets from the library's own
FP64 descriptors of seeded candidate cells, coefficients from the seeded
draws).  Shared by bench.py and profile_run.py."""
from __future__ import annotations

from . import synth


def model_for(index: int, gap, device: str, precision: str = "fp64"):
    """(workload, soap, model) with M random sparse points per central species
    taken among the descriptors of the workload's candidate cells."""
    w = synth.workload(index)
    soap = gap.Soap.from_spec(w.soap)
    cells = synth.sparse_candidate_structures(index)
    b = synth.make_batch(cells)
    pool = soap.descriptor(gap.Batch.from_synth(b, device=device), precision=precision)
    pool = pool.cpu().numpy() if hasattr(pool, "cpu") else pool
    sparse, alpha = [], []
    for s in range(w.soap.n_species):
        cand = pool[b.species == s]
        idx = synth.sparse_indices(index, s, cand.shape[0], min(w.M, cand.shape[0]))
        sparse.append(cand[idx])
        alpha.append(synth.alpha_draw(index, s, idx.size))
    model = gap.Model(soap, sparse, alpha, w.delta, w.zeta, two_body=w.two_body)
    return w, soap, model
