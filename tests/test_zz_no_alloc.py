"""hk_scan_knn_noalloc, the exhaustive scan for callers that cannot allocate
device memory (for example when another allocator holds the GPU's memory, or
when cudaFree's device-wide wait is unacceptable): it must give the same
answers as hk_scan_knn, the entry point that allocates its work space, on
consecutive calls that share its fixed scratch array.

Named to be collected last, so a run that stops at the first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest

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


def test_noalloc_matches_allocating_scan_twice(hb):
    from paper_2212_13297_gb300 import workload
    X = workload.random_walk(50_000, 128, seed=41, device="cuda")
    X[20_000:20_100] = X[5]                       # 101 exact ties with row 5
    cases = []
    Q1, _ = workload.queries(X, 40, [0.05, 0.5, 1.0], seed=42)
    Q2 = torch.cat([X[[5, 5]], workload.queries(X, 6, 0.3, seed=43)[0]]).contiguous()
    cases = [(Q1, 10), (Q2, 17)]                   # second call: different sizes, ties
    for Q, k in cases:
        ref_ids, ref_dist = hb.scan_knn(X, Q, k)
        ids, dist = noalloc(hb, X, Q, k)
        np.testing.assert_array_equal(ids, ref_ids.cpu().numpy())
        np.testing.assert_allclose(dist, ref_dist.cpu().numpy(), rtol=1e-5, atol=0)
    assert list(ids[0, :3]) == [5, 20_000, 20_001]


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
