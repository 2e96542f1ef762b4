"""Failure paths, made to happen without faulting the GPU.

  * The tensor-core scan's bounded waits: a test hook makes one epilogue
    warp per CTA wait for a barrier nothing arrives at, with a 1 ms limit;
    the wait runs out, the CTA drains its copies and tensor-core operations
    in flight, frees its tensor memory and exits, and the call returns
    HK_ETIMEOUT.  The same index then answers exactly.
  * Device allocation failure: a test hook fails the library's next device
    allocation as a failed cudaMalloc would; build and query return
    HK_ENOMEM, and the next calls succeed with exact answers.
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
    yield binding
    binding.lib().hk_debug_tc_wait(0, 0)
    binding.lib().hk_debug_fail_device_alloc(-1)


def _wl():
    from paper_2212_13297_gb300 import workload
    return workload


def _exact(ids, dist, X, Q, k):
    oids, od2 = oracle.knn(X.cpu().numpy(), Q.cpu().numpy(), k)
    np.testing.assert_array_equal(ids.cpu().numpy(), oids)
    np.testing.assert_allclose(dist.cpu().numpy(), np.sqrt(od2).astype(np.float32), rtol=1e-5)


def test_tc_wait_runs_out_then_index_answers(hb, oracle_lib):
    wl = _wl()
    X = wl.random_walk(60_000, 256, seed=61, device="cuda")
    Q, _ = wl.queries(X, 40, [0.1, 0.5, 1.0], seed=62)
    idx = hb.Index(X, 1000, flags=hb.HK_BUILD_FP16)
    L = hb.lib()
    assert L.hk_debug_tc_wait(1_000_000, 1) == hb.HK_OK
    try:
        with pytest.raises(hb.HerculesError) as e:
            idx.query(Q, 10, flags=hb.HK_Q_BF16)
        assert e.value.code == hb.HK_ETIMEOUT
        # flag 2: a wait ran out; flag 4 would mean a drain missed its deadline
        assert "flag 2)" in str(e.value), str(e.value)
    finally:
        assert L.hk_debug_tc_wait(0, 0) == hb.HK_OK
    torch.cuda.synchronize()
    ids, dist, _ = idx.query(Q, 10, flags=hb.HK_Q_BF16)
    _exact(ids, dist, X, Q, 10)
    ids, dist, _ = idx.query(Q, 10)
    _exact(ids, dist, X, Q, 10)
    idx.close()


def test_injected_allocation_failure(hb, oracle_lib):
    wl = _wl()
    L = hb.lib()
    X = wl.random_walk(30_000, 128, seed=63, device="cuda")
    before = hb.device_allocs()
    assert L.hk_debug_fail_device_alloc(2) == hb.HK_OK   # the third allocation fails
    with pytest.raises(hb.HerculesError) as e:
        hb.Index(X, 500)
    assert e.value.code == hb.HK_ENOMEM and "injected" in str(e.value)
    assert hb.device_allocs() == before + 3
    idx = hb.Index(X, 500)                                # the hook was one-shot
    Q, _ = wl.queries(X, 8, [0.2, 1.0], seed=64)
    ids, dist, _ = idx.query(Q, 5)
    _exact(ids, dist, X, Q, 5)
    # a larger batch grows the work space: fail its first allocation
    Q2, _ = wl.queries(X, 300, [0.2, 1.0], seed=65)
    assert L.hk_debug_fail_device_alloc(0) == hb.HK_OK
    with pytest.raises(hb.HerculesError) as e:
        idx.query(Q2, 5)
    assert e.value.code == hb.HK_ENOMEM
    ids, dist, _ = idx.query(Q2, 5)
    _exact(ids, dist, X, Q2, 5)
    # the exhaustive scan's temporary buffers
    assert L.hk_debug_fail_device_alloc(0) == hb.HK_OK
    with pytest.raises(hb.HerculesError) as e:
        hb.scan_knn(X.cpu().numpy(), Q.cpu().numpy(), 3)
    assert e.value.code == hb.HK_ENOMEM
    ids, dist = hb.scan_knn(X, Q, 3)
    _exact(ids, dist, X, Q, 3)
    idx.close()
