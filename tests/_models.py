"""Oracle-side model construction shared by the tests: sparse points are the
oracle's own descriptors of seeded candidate cells ('random' selection, Sec.
3.2.2), coefficients alpha are seeded draws.  Nothing here reads the CUDA path."""
import functools

import numpy as np

import oracle as O
from paper_2310_03921_gb300 import synth as S


def soap_of(spec, **over):
    kw = dict(n_max=spec.n_max, l_max=spec.l_max, rc=spec.rc, sigma=spec.sigma, d=spec.d,
              central_weight=spec.central_weight, n_species=spec.n_species, mix_K=spec.mix_K, mix_w=spec.mix_w)
    kw.update(over)
    return O.Soap(**kw)


@functools.lru_cache(maxsize=None)
def candidate_pool(index, n_max, l_max, n_cells=None):
    """Oracle descriptors of the candidate cells of a workload, per central species."""
    w = S.workload(index)
    soap = soap_of(w.soap, n_max=n_max, l_max=l_max)
    cells = S.sparse_candidate_structures(index)
    if n_cells is not None:
        cells = cells[:n_cells]
    ph = [O.descriptor(soap, c)[0] for c in cells]
    sp = [c.species for c in cells]
    P, Z = np.concatenate(ph), np.concatenate(sp)
    return tuple(P[Z == s] for s in range(w.soap.n_species))


def oracle_model(index, M, n_max=None, l_max=None, n_cells=None, two_body=True, zeta=None):
    """(soap, model, sparse list, alpha list) for a workload, optionally shrunk."""
    w = S.workload(index)
    n_max = n_max or w.soap.n_max
    l_max = l_max if l_max is not None else w.soap.l_max
    soap = soap_of(w.soap, n_max=n_max, l_max=l_max)
    pools = candidate_pool(index, n_max, l_max, n_cells)
    sparse, alpha = [], []
    for s, pool in enumerate(pools):
        idx = S.sparse_indices(index, s, pool.shape[0], min(M, pool.shape[0]))
        sparse.append(pool[idx])
        alpha.append(S.alpha_draw(index, s, idx.size))
    tb = w.two_body if two_body else None
    model = O.Model(sparse, alpha, w.delta, zeta or w.zeta, two_body=tb)
    return soap, model, sparse, alpha
