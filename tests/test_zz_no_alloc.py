"""hk_scan_knn_noalloc, the exhaustive scan for callers that cannot allocate
device memory (for example when another allocator holds the GPU's memory, or
when cudaFree's device-wide wait is unacceptable): on consecutive calls that
share its fixed scratch array it must give the brute-force oracle's answers
and the same answers as hk_scan_knn, the entry point that allocates its work
space, and it must make no device allocation, also when a query has more
near-tied candidates than its pool holds (the exhaustive collect fallback).
Past the documented tie limit it returns HK_ENOMEM and the next call works.

Named to be collected last, so a run that stops at the first failure has
already run every other test.
"""
import ctypes

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


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def noalloc(hb, X, Q, k):
    nq = Q.shape[0]
    ids = torch.full((nq, k), -7, dtype=torch.int64, device="cuda")
    dist = torch.full((nq, k), -1.0, dtype=torch.float32, device="cuda")
    rc = hb.lib().hk_scan_knn_noalloc(_p(X), X.shape[0], X.shape[1], _p(Q), nq, k,
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                      _p(ids), _p(dist))
    assert rc == hb.HK_OK, hb.lib().hk_last_error()
    torch.cuda.synchronize()
    return ids.cpu().numpy(), dist.cpu().numpy()


def test_noalloc_matches_allocating_scan_twice(hb, oracle_lib):
    from paper_2212_13297_gb300 import workload
    X = workload.random_walk(50_000, 128, seed=41, device="cuda")
    X[20_000:20_100] = X[5]                       # 101 exact ties with row 5
    Q1, _ = workload.queries(X, 40, [0.05, 0.5, 1.0], seed=42)
    Q2 = torch.cat([X[[5, 5]], workload.queries(X, 6, 0.3, seed=43)[0]]).contiguous()
    cases = [(Q1, 10), (Q2, 17)]                   # second call: different sizes, ties
    Xh = X.cpu().numpy()
    for Q, k in cases:
        ref_ids, ref_dist = hb.scan_knn(X, Q, k)
        before = hb.device_allocs()
        ids, dist = noalloc(hb, X, Q, k)
        assert hb.device_allocs() == before, "the no-alloc entry point allocated device memory"
        np.testing.assert_array_equal(ids, ref_ids.cpu().numpy())
        np.testing.assert_allclose(dist, ref_dist.cpu().numpy(), rtol=1e-5, atol=0)
        oids, od2 = oracle.knn(Xh, Q.cpu().numpy(), k)
        np.testing.assert_array_equal(ids, oids)
        np.testing.assert_allclose(dist, np.sqrt(od2).astype(np.float32), rtol=1e-5)
    assert list(ids[0, :3]) == [5, 20_000, 20_001]


def test_noalloc_near_tie_fallback_allocates_nothing(hb, oracle_lib):
    """5,000 copies of one row overflow the 4,096-entry pool of the queries
    equal to it, so those queries take the exhaustive collect into the
    scratch's collection area."""
    from paper_2212_13297_gb300 import workload
    X = workload.random_walk(40_000, 64, seed=44, device="cuda")
    X[10_000:15_000] = X[7]
    Q = torch.cat([X[[7]], workload.queries(X, 5, [0.1, 1.0], seed=45)[0]]).contiguous()
    for k in (3, 40):
        before = hb.device_allocs()
        ids, dist = noalloc(hb, X, Q, k)
        assert hb.device_allocs() == before
        oids, od2 = oracle.knn(X.cpu().numpy(), Q.cpu().numpy(), k)
        np.testing.assert_array_equal(ids, oids)
        np.testing.assert_allclose(dist, np.sqrt(od2).astype(np.float32), rtol=1e-5)
    assert list(ids[0, :3]) == [7, 10_000, 10_001]


def test_noalloc_tie_limit(hb):
    """More near-tied candidates than the scratch's collection area holds
    (65,536): HK_ENOMEM with a message, and the next call still matches
    hk_scan_knn."""
    from paper_2212_13297_gb300 import workload
    L = hb.lib()
    X = workload.random_walk(1, 64, seed=46, device="cuda").repeat(70_000, 1).contiguous()
    q = X[:1].clone()
    ids = torch.zeros((1, 1), dtype=torch.int64, device="cuda")
    dist = torch.zeros((1, 1), device="cuda")
    rc = L.hk_scan_knn_noalloc(_p(X), 70_000, 64, _p(q), 1, 1, None, _p(ids), _p(dist))
    assert rc == hb.HK_ENOMEM
    assert b"near-tied" in L.hk_last_error()
    Y = workload.random_walk(20_000, 64, seed=47, device="cuda")
    Q, _ = workload.queries(Y, 4, 0.5, seed=48)
    got_ids, got_dist = noalloc(hb, Y, Q, 6)
    ref_ids, ref_dist = hb.scan_knn(Y, Q, 6)
    np.testing.assert_array_equal(got_ids, ref_ids.cpu().numpy())
    np.testing.assert_allclose(got_dist, ref_dist.cpu().numpy(), rtol=1e-5, atol=0)


def test_noalloc_rejects_oversized_and_host_buffers(hb):
    from paper_2212_13297_gb300 import workload
    X = workload.random_walk(1000, 64, seed=1, device="cuda")
    L = hb.lib()
    big_q = torch.zeros((65, 64), device="cuda")
    ids = torch.zeros((65, 1), dtype=torch.int64, device="cuda")
    dist = torch.zeros((65, 1), device="cuda")
    assert L.hk_scan_knn_noalloc(_p(X), 1000, 64, _p(big_q), 65, 1, None, _p(ids),
                                 _p(dist)) == hb.HK_EINVAL
    assert b"nq=65" in L.hk_last_error()
    q = torch.zeros((1, 64), device="cuda")
    assert L.hk_scan_knn_noalloc(_p(X), 1000, 64, _p(q), 1, 65, None, _p(ids),
                                 _p(dist)) == hb.HK_EINVAL
    host_ids = np.zeros((1, 1), np.int64)
    assert L.hk_scan_knn_noalloc(_p(X), 1000, 64, _p(q), 1, 1, None,
                                 ctypes.c_void_p(host_ids.ctypes.data), _p(dist)) == hb.HK_EINVAL
