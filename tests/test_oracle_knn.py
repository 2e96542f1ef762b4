"""Pins for the oracle's distance and brute-force k-NN (Sec. 2: k-NN query
definition over the Euclidean distance; answers ordered by (D, id)).

Every check here is independent of the oracle's own code: closed forms,
numpy as a separate implementation, and properties of the definition.
"""
import numpy as np
import pytest

import oracle


def test_dist2_closed_forms(oracle_lib):
    n = 64
    z = np.zeros(n, np.float32)
    # distance to a unit vector is 1; to c*ones is n*c^2
    e = np.zeros(n, np.float32)
    e[17] = 1.0
    assert oracle.dist2(z, e) == 1.0
    c = np.full(n, 0.5, np.float32)
    assert oracle.dist2(z, c) == n * 0.25
    # sign matters only through the difference: (1 - (-2))^2 = 9
    a = np.zeros(n, np.float32)
    b = np.zeros(n, np.float32)
    a[3], b[3] = 1.0, -2.0
    assert oracle.dist2(a, b) == 9.0
    # index alignment: a shifted copy is not at distance 0
    x = np.arange(n, dtype=np.float32)
    assert oracle.dist2(x, x) == 0.0
    assert oracle.dist2(x, np.roll(x, 1)) == (n - 1) + (n - 1) ** 2


def test_dist2_matches_numpy(oracle_lib):
    rng = np.random.default_rng(5)
    for n in (16, 96, 256, 1024):
        q = rng.standard_normal(n).astype(np.float32)
        x = rng.standard_normal(n).astype(np.float32)
        ref = float(np.sum((q.astype(np.float64) - x.astype(np.float64)) ** 2))
        assert abs(oracle.dist2(q, x) - ref) <= 1e-12 * ref


def _numpy_knn(X, Q, k):
    d = ((Q[:, None, :].astype(np.float64) - X[None, :, :].astype(np.float64)) ** 2).sum(-1)
    ids = np.empty((Q.shape[0], k), np.int64)
    for i in range(Q.shape[0]):
        order = np.lexsort((np.arange(X.shape[0]), d[i]))
        ids[i] = order[:k]
    return ids, np.take_along_axis(d, ids, 1)


@pytest.mark.parametrize("N,n,nq,k", [(500, 16, 7, 1), (700, 64, 5, 10), (300, 256, 4, 100)])
def test_knn_matches_numpy(oracle_lib, N, n, nq, k):
    rng = np.random.default_rng(N + n)
    X = rng.standard_normal((N, n)).astype(np.float32)
    Q = rng.standard_normal((nq, n)).astype(np.float32)
    ids, d2 = oracle.knn(X, Q, k)
    rids, rd2 = _numpy_knn(X, Q, k)
    np.testing.assert_array_equal(ids, rids)
    np.testing.assert_allclose(d2, rd2, rtol=1e-12)
    assert np.all(np.diff(d2, axis=1) >= 0)


def test_knn_self_query_and_ties(oracle_lib):
    rng = np.random.default_rng(1)
    X = rng.standard_normal((200, 32)).astype(np.float32)
    X[150] = X[20]          # exact duplicate: equal distance, lower id first
    X[180] = X[20]
    ids, d2 = oracle.knn(X, X[[20, 7]], 4)
    assert list(ids[0, :3]) == [20, 150, 180]
    assert d2[0, 0] == d2[0, 1] == d2[0, 2] == 0.0
    assert ids[1, 0] == 7 and d2[1, 0] == 0.0


def test_knn_k_equals_n_is_full_sort(oracle_lib):
    rng = np.random.default_rng(2)
    X = rng.standard_normal((50, 16)).astype(np.float32)
    Q = rng.standard_normal((3, 16)).astype(np.float32)
    ids, d2 = oracle.knn(X, Q, 50)
    for i in range(3):
        assert sorted(ids[i]) == list(range(50))
        assert np.all(np.diff(d2[i]) >= 0)


def test_knn_stream_equals_single_pass(oracle_lib):
    rng = np.random.default_rng(3)
    X = rng.standard_normal((1000, 48)).astype(np.float32)
    X[999] = X[10]
    Q = np.concatenate([X[[10]], rng.standard_normal((5, 48)).astype(np.float32)])
    ids, d2 = oracle.knn(X, Q, 7)
    s = oracle.KnnStream(Q, 7, nthreads=3)
    for a in range(0, 1000, 137):
        s.update(X[a:a + 137], a)
    sids, sd2 = s.result()
    np.testing.assert_array_equal(ids, sids)
    np.testing.assert_array_equal(d2, sd2)
    assert list(ids[0, :2]) == [10, 999]


def test_knn_thread_count_invariant(oracle_lib):
    rng = np.random.default_rng(4)
    X = rng.standard_normal((400, 32)).astype(np.float32)
    Q = rng.standard_normal((9, 32)).astype(np.float32)
    a = oracle.knn(X, Q, 5, nthreads=1)
    b = oracle.knn(X, Q, 5, nthreads=4)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
