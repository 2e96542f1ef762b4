"""Exact k-NN under DTW (Sec. 2: a distance with a lower bound) through
hk_query_dtw against the oracle's brute force under the same DTW: ids
identical (ties to the lower id), distances within 1e-5 relative; band 0
gives the Euclidean answers; the leaf bound is the oracle's bit for bit
(through the answers it prunes by) and the stats show the bounds pruning."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hb():
    from paper_2212_13297_gb300 import build, binding
    build.build()
    binding.lib()
    assert torch.cuda.is_available(), "GPU test without a GPU"
    return binding


def _wl():
    from paper_2212_13297_gb300 import workload
    return workload


@pytest.mark.parametrize("N,n,tau,nq,k,band,sig", [
    (8000, 64, 100, 12, 1, 4, [0.1, 0.5]),
    (8000, 64, 100, 12, 10, 8, [0.5, 1.0]),
    (5000, 128, 80, 8, 5, 12, [0.05, 1.0]),
    (3000, 256, 60, 6, 20, 16, [0.3]),
    (6000, 16, 50, 10, 7, 3, [0.2, 1.0]),
    (20000, 64, 5000, 8, 10, 8, [0.5, 1.0]),     # leaves of thousands: several screening windows
])
def test_dtw_matches_bruteforce(hb, oracle_lib, N, n, tau, nq, k, band, sig):
    wl = _wl()
    X = wl.random_walk(N, n, seed=N + band, device="cuda")
    Q, _ = wl.queries(X, nq, sig, seed=band + 1)
    idx = hb.Index(X, tau)
    oids, od2 = oracle.dtw_knn(X.cpu().numpy(), Q.cpu().numpy(), k, band)
    for flags in (0, hb.HK_Q_NOSAX):
        ids, dist, st = idx.query_dtw(Q, k, band, flags=flags)
        np.testing.assert_array_equal(ids.cpu().numpy(), oids)
        np.testing.assert_allclose(dist.cpu().numpy(), np.sqrt(od2).astype(np.float32), rtol=1e-5)
        assert st["queries"] == nq and st["rescored"] >= nq * k
    assert st["series_sax_pruned"] + st["series_abandoned"] > 0   # the bounds pruned series


def test_dtw_band_zero_is_euclidean_and_ties(hb, oracle_lib):
    wl = _wl()
    X = wl.random_walk(6000, 64, seed=5, device="cuda")
    X[4000:4030] = X[11]                           # exact ties with row 11
    Q = torch.cat([X[[11]], wl.queries(X, 5, [0.3, 1.0], seed=6)[0]]).contiguous()
    idx = hb.Index(X, 80)
    ids0, d0, _ = idx.query_dtw(Q, 12, 0)
    ide, de, _ = idx.query(Q, 12)
    np.testing.assert_array_equal(ids0.cpu().numpy(), ide.cpu().numpy())
    np.testing.assert_array_equal(d0.cpu().numpy(), de.cpu().numpy())
    ids, d, _ = idx.query_dtw(Q, 40, 6)
    oids, od2 = oracle.dtw_knn(X.cpu().numpy(), Q.cpu().numpy(), 40, 6)
    np.testing.assert_array_equal(ids.cpu().numpy(), oids)
    assert list(ids[0, :3].cpu().numpy()) == [11, 4000, 4001]


def test_dtw_host_buffers_and_checks(hb, oracle_lib):
    wl = _wl()
    X = wl.random_walk(3000, 32, seed=8, device="cuda")
    Q, _ = wl.queries(X, 4, 0.5, seed=9)
    idx = hb.Index(X, 50)
    ids, d, _ = idx.query_dtw(Q.cpu().numpy(), 3, 5)
    oids, _ = oracle.dtw_knn(X.cpu().numpy(), Q.cpu().numpy(), 3, 5)
    np.testing.assert_array_equal(ids, oids)
    for band in (-1, 17, 32):
        with pytest.raises(hb.HerculesError) as e:
            idx.query_dtw(Q, 3, band)
        assert e.value.code == hb.HK_EINVAL
