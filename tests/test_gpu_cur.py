"""'cur_points' selection (Sec. 3.2.2) on the GPU through the C-ABI against
the FP64 oracle: the leverage scores element by element, the rank k chosen
by default, and the selected rows.  Selection is decided by comparing FP64
scores, so rows whose oracle scores lie within the score tolerance of the
last selected score may legitimately differ; every other selected row must
be the oracle's."""
import numpy as np
import pytest

import oracle as O
from paper_2310_03921_gb300 import synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_2310_03921_gb300 import build, gap
    build.build()
    return gap


def _compare(G, X, m, k=0, device=False, tol=1e-6):
    ref_sel, ref_pi, ref_k = O.cur_select(X, m, k=k)
    if device:
        import torch
        sel, pi, ku = G.cur_select(torch.as_tensor(X, device="cuda"), m, k=k)
        sel, pi = sel.cpu().numpy(), pi.cpu().numpy()
    else:
        sel, pi, ku = G.cur_select(X, m, k=k)
    assert ku == ref_k
    scale = ref_pi.max()
    assert np.abs(pi - ref_pi).max() <= tol * scale, np.abs(pi - ref_pi).max() / scale
    assert sel.size == ref_sel.size and len(set(sel.tolist())) == sel.size
    s_last = ref_pi[ref_sel].min()
    for i in set(sel.tolist()) ^ set(ref_sel.tolist()):
        assert abs(ref_pi[i] - s_last) <= tol * scale, (i, ref_pi[i], s_last)
    # selection order: non-increasing GPU scores
    assert (np.diff(pi[sel]) <= 0).all()
    return sel, pi


def test_cur_random_design(G):
    rng = np.random.default_rng(7)
    X = rng.normal(size=(700, 24)) * np.logspace(0, -3, 24)
    for k, m in ((8, 40), (24, 100), (0, 60)):
        _compare(G, X, m, k=k, tol=1e-9)


def test_cur_duplicates_considered_once(G):
    rng = np.random.default_rng(8)
    X = rng.normal(size=(200, 10))
    X[[150, 170, 190]] = X[[3, 3, 40]]  # exact copies of rows 3 and 40
    sel, pi, _ = G.cur_select(X, 199, k=10)
    assert sel.size == 197  # three copies skipped
    for copy, orig in ((150, 3), (170, 3), (190, 40)):
        assert orig in sel.tolist() and copy not in sel.tolist()
        assert pi[copy] == pi[orig]


def test_cur_soap_descriptors_fit_workload(G):
    """Descriptors of the fit workload's candidate cells (D 252), default rank,
    on host and device arrays."""
    w = S.workload(1)
    soap = O.Soap(w.soap.n_max, w.soap.l_max, w.soap.rc, w.soap.sigma, w.soap.d)
    X = np.concatenate([O.descriptor(soap, c)[0] for c in S.sparse_candidate_structures(1)[:20]])
    _compare(G, X, 300)
    _compare(G, X, 1000, device=True)


def test_cur_bad_arguments(G):
    X = np.ones((10, 3))
    with pytest.raises(G.GapError):
        G.cur_select(X, 11)
    with pytest.raises(G.GapError):
        G.cur_select(np.zeros((10, 3)), 2)
