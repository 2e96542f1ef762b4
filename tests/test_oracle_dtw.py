"""Pins of the oracle's DTW (Sec. 2: a distance with a lower bound) and of
LB_Keogh and its segment / iSAX forms, against things other than the oracle
itself: a hand-worked case, the Euclidean distance at band 0, brute force
over every warping path on tiny inputs, and the bound's definition."""
import itertools
from fractions import Fraction

import numpy as np
import pytest


@pytest.fixture(scope="module")
def O(oracle_lib):
    import oracle
    return oracle


def test_hand_worked_dtw(O):
    # cost matrix (q_i - x_j)^2; with band 1 the path (0,0) (0,1) (1,2) (2,3)
    # (3,3) costs 0 + 0 + 0 + 0 + 1; the diagonal (band 0) costs 0+1+1+1
    q = np.array([0, 1, 2, 3], np.float32)
    x = np.array([0, 0, 1, 2], np.float32)
    assert O.dtw2(q, x, 0) == 3.0
    assert O.dtw2(q, x, 1) == 1.0
    assert O.dtw2(q, x, 3) == 1.0


def _paths(n, band):
    """Every warping path from (0,0) to (n-1,n-1) inside the band."""
    def rec(i, j):
        if (i, j) == (n - 1, n - 1):
            yield [(i, j)]
            return
        for di, dj in ((1, 1), (1, 0), (0, 1)):
            a, b = i + di, j + dj
            if a < n and b < n and abs(a - b) <= band:
                for p in rec(a, b):
                    yield [(i, j)] + p
    return list(rec(0, 0))


@pytest.mark.parametrize("n,band", [(4, 1), (5, 2), (6, 1), (6, 5), (7, 2)])
def test_dtw_equals_brute_force_over_paths(O, n, band):
    rng = np.random.default_rng(n * 10 + band)
    paths = _paths(n, band)
    for _ in range(20):
        q = rng.standard_normal(n).astype(np.float32)
        x = rng.standard_normal(n).astype(np.float32)
        best = min(sum((Fraction(float(q[i])) - Fraction(float(x[j]))) ** 2 for i, j in p) for p in paths)
        assert O.dtw2(q, x, band) == pytest.approx(float(best), rel=1e-13, abs=1e-300)


def test_band_zero_is_squared_euclidean_and_self_distance_zero(O):
    rng = np.random.default_rng(3)
    for n in (16, 64, 256):
        for _ in range(10):
            q = rng.standard_normal(n).astype(np.float32)
            x = rng.standard_normal(n).astype(np.float32)
            assert O.dtw2(q, x, 0) == O.dist2(q, x)        # the same sum, the same order
            for band in (0, 3, 12):
                assert O.dtw2(q, q, band) == 0.0


def test_dtw_monotone_in_band_and_symmetric(O):
    rng = np.random.default_rng(4)
    for _ in range(30):
        q = np.cumsum(rng.standard_normal(64)).astype(np.float32)
        x = np.cumsum(rng.standard_normal(64)).astype(np.float32)
        vals = [O.dtw2(q, x, b) for b in (0, 1, 2, 4, 8, 16, 63)]
        assert all(a >= b for a, b in zip(vals, vals[1:]))
        assert O.dtw2(q, x, 5) == pytest.approx(O.dtw2(x, q, 5), rel=1e-12)


def test_envelope_definition(O):
    q = np.array([3, 1, 4, 1, 5, 9, 2, 6], np.float32)
    L, U = O.envelope(q, 1)
    np.testing.assert_array_equal(L, [1, 1, 1, 1, 1, 2, 2, 2])
    np.testing.assert_array_equal(U, [3, 4, 4, 5, 9, 9, 9, 6])


@pytest.mark.parametrize("n,band", [(16, 2), (32, 3), (64, 6)])
def test_lb_keogh_and_its_forms_bound_dtw(O, n, band):
    from oracle import tree
    rng = np.random.default_rng(n + band)
    X = np.cumsum(rng.standard_normal((160, n)), axis=1)
    X = ((X - X.mean(1, keepdims=True)) / X.std(1, keepdims=True)).astype(np.float32)
    Q = X[rng.integers(0, 160, 5)] + 0.5 * rng.standard_normal((5, n)).astype(np.float32)
    bp = O.isax_breakpoints_f32()
    root = tree.build_tree(X, 12)
    nodes = tree.nodes_preorder(root)
    syn = {id(nd): tree.node_synopsis(X, nd) for nd in nodes}
    for q in Q:
        d = np.array([O.dtw2(q, x, band) for x in X])
        for i, x in enumerate(X):
            assert O.lb_keogh(q, x, band) <= d[i] * (1 + 1e-12)
            assert O.lb_keogh_sax(q, band, O.isax_word(x, bp), bp) <= d[i] * (1 + 1e-12)
        for nd in nodes:
            lb = O.lb_keogh_eapca(q, band, nd.seg_end, syn[id(nd)])
            for i in tree.subtree_members(nd):
                assert lb <= d[i] * (1 + 1e-12)
        # band 0: LB_Keogh is the squared Euclidean distance itself
        assert O.lb_keogh(q, X[0], 0) == O.dist2(q, X[0])


def test_dtw_knn_brute_force(O):
    rng = np.random.default_rng(7)
    X = rng.standard_normal((300, 32)).astype(np.float32)
    X[200] = X[17]                                   # a tie: lower id first
    Q = np.stack([X[17], rng.standard_normal(32).astype(np.float32)])
    ids, d2 = O.dtw_knn(X, Q, 5, 3)
    for qi, q in enumerate(Q):
        d = np.array([O.dtw2(q, x, 3) for x in X])
        order = sorted(range(300), key=lambda i: (d[i], i))[:5]
        assert list(ids[qi]) == order
        np.testing.assert_array_equal(d2[qi], d[order])
    assert list(ids[0, :2]) == [17, 200]
