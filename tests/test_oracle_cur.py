"""Pins of the oracle's 'cur_points' selection (Sec. 3.2.2, CUR by rank-k
leverage scores): the scores sum to one, equal the diagonal of the hat
matrix divided by D at full rank (a normal-equations route, not the SVD),
are invariant to a rotation of the descriptor space and to scaling, single
out the rows of the dominant directions of a diagonal design, and the
selection follows the stated order and skips duplicates."""
import numpy as np

import oracle as O
from paper_2310_03921_gb300 import synth as S


def _desc(n_cells=3):
    w = S.workload(0)
    soap = O.Soap(w.soap.n_max, w.soap.l_max, w.soap.rc, w.soap.sigma, w.soap.d)
    return np.concatenate([O.descriptor(soap, c)[0] for c in S.sparse_candidate_structures(0)[:n_cells]])


def test_scores_sum_to_one_and_match_the_hat_matrix():
    rng = np.random.default_rng(3)
    X = rng.normal(size=(300, 12)) * np.logspace(0, -2, 12)
    for k in (1, 5, 12):
        _, pi, kk = O.cur_select(X, 10, k=k)
        assert kk == k and abs(pi.sum() - 1.0) <= 1e-12
    _, pi, _ = O.cur_select(X, 10, k=12)
    hat = np.einsum("ij,ij->i", X, np.linalg.solve(X.T @ X, X.T).T)
    assert np.abs(pi - hat / 12).max() <= 1e-12


def test_scores_invariant_to_rotation_and_scale():
    X = _desc()
    Q, _ = np.linalg.qr(np.random.default_rng(4).normal(size=(X.shape[1], X.shape[1])))
    c1, p1, k1 = O.cur_select(X, 40, k=30)
    c2, p2, k2 = O.cur_select(3.7 * X @ Q, 40, k=30)
    assert np.abs(p1 - p2).max() <= 1e-9 * p1.max()
    assert np.array_equal(c1, c2)


def test_diagonal_design_picks_the_dominant_directions():
    # rows c_j e_j (decreasing c_j), each twice, plus zero rows: at rank k the
    # scores are 1/(2k) on the rows of the k largest c_j and 0 elsewhere
    D, k = 8, 3
    c = np.linspace(5.0, 1.0, D)
    X = np.zeros((3 * D, D))
    for j in range(D):
        X[2 * j, j] = X[2 * j + 1, j] = c[j]
    chosen, pi, _ = O.cur_select(X, 3, k=k)
    assert np.allclose(pi[: 2 * k], 1.0 / (2 * k), atol=1e-14) and np.abs(pi[2 * k:]).max() <= 1e-14
    # duplicates considered once: rows 0, 2, 4 (not their copies 1, 3, 5);
    # the six scores are equal up to rounding, so any order among them holds
    assert sorted(chosen.tolist()) == [0, 2, 4]


def test_selection_order_and_default_rank():
    X = _desc()
    chosen, pi, k = O.cur_select(X, 50)
    s = np.linalg.svd(X, compute_uv=False)
    assert k == min(50, int((s >= 1e-4 * s[0]).sum()))
    # brute force: the 50 largest scores, ties by index
    ref = sorted(range(X.shape[0]), key=lambda i: (-pi[i], i))[:50]
    assert chosen.tolist() == ref
    assert len(set(chosen.tolist())) == 50
