"""Parity at the benchmark workloads' full sizes, in the launch configuration
bench.py times (collection, batch, form, options), against the brute-force
oracle, which streams the same seeded collection block by block so host
memory never holds it whole.  Ids must be identical, distances within 1e-5
relative (the answer definition of Sec. 2: the k smallest (D, id) pairs).

Checked queries:
  mid        10M x 256, leaf 10K, 100 queries (sigma 0.01 / 0.1 / 0.5 / 1.0),
             k = 1 and 10, float32 path: every query;
  precision  10M x 256, leaf 10K, 1,024 queries (sigma uniform in [0.01, 1]),
             k = 100, tensor-core form on a float16 and on a bfloat16 copy and
             the float32 path: every query;
  large      100M x 256, leaf 100K, the benchmark's first batch of 2,000 hard
             queries (sigma 0.5 / 1.0), k = 10, float16 tensor-core form and
             float32 path: every 8th query of the batch (250), or every
             HK_FULLSIZE_STRIDE-th when that variable is set;
  served mix the four collections of workload.SERVED_MIX behind one server
             (tensor-core form where n <= 256, float32 for n = 1024), 48
             requests per collection with k cycling over 1, 10, 100, submitted
             in interleaved waves while earlier batches run: every request;
  n = 1024   200K x 1024 random walks, leaf 2,000, float32 path, k = 1, 10, 100:
             every query.
The oracle runs on all host cores (its threads split the queries).
"""
import gc
import os
import time

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


def _release():
    gc.collect()                 # indexes and tensors of earlier tests
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def _need(nbytes):
    _release()
    free, _ = torch.cuda.mem_get_info()
    if free < nbytes:
        pytest.skip("needs %.0f GB of free device memory" % (nbytes / 1e9))


def _oracle_rw(N, n, seed, Qs, k):
    """Oracle answer over random_walk(N, n, seed), regenerated block by block."""
    s = oracle.KnnStream(Qs, k)
    for a, rows in _wl().random_walk_chunks(N, n, seed=seed, device="cuda"):
        s.update(rows.cpu().numpy(), a)
    return s.result()


def _oracle_dev(X, Qs, k, rows=1 << 18):
    """Oracle answer over a device-resident collection, copied block by block."""
    s = oracle.KnnStream(Qs, k)
    for a in range(0, X.shape[0], rows):
        s.update(X[a:a + rows].cpu().numpy(), a)
    return s.result()


def _check(ids, dist, oids, od2, what):
    ids = ids.cpu().numpy() if hasattr(ids, "cpu") else ids
    dist = dist.cpu().numpy() if hasattr(dist, "cpu") else dist
    bad = np.nonzero((ids != oids).any(axis=1))[0]
    assert bad.size == 0, "%s: %d queries differ, first rows %s" % (what, bad.size, bad[:8].tolist())
    np.testing.assert_allclose(dist, np.sqrt(od2).astype(np.float32), rtol=1e-5, err_msg=what)


def test_mid_every_query(hb, oracle_lib):
    wl = _wl()
    N, n, tau = 10_000_000, 256, 10_000
    _need(N * n * 4 * 2.2)
    X = wl.random_walk(N, n, seed=0, device="cuda")
    Q, _ = wl.queries(X, 100, [0.01, 0.1, 0.5, 1.0], seed=1)
    idx = hb.Index(X, tau)
    del X
    _release()
    oids, od2 = _oracle_rw(N, n, 0, Q.cpu().numpy(), 10)
    for k in (1, 10):
        ids, dist, st = idx.query(Q, k, flags=hb.HK_Q_TIMING)
        assert st["queries"] == 100
        _check(ids, dist, oids[:, :k], od2[:, :k], "mid k=%d" % k)
    idx.close()


def test_precision_every_query(hb, oracle_lib):
    wl = _wl()
    N, n, tau, B, k = 10_000_000, 256, 10_000, 1024, 100
    _need(N * n * 4 * 3.3)
    X = wl.random_walk(N, n, seed=0, device="cuda")
    Q, _ = wl.queries(X, B, wl.uniform_sigmas(B, 0.01, 1.0, seed=1), seed=1)
    i16 = hb.Index(X, tau, flags=hb.HK_BUILD_FP16)
    ib16 = hb.Index(X, tau, flags=hb.HK_BUILD_BF16)
    del X
    _release()
    oids, od2 = _oracle_rw(N, n, 0, Q.cpu().numpy(), k)
    for name, idx, flags in (("float16 copy", i16, hb.HK_Q_BF16 | hb.HK_Q_TIMING),
                             ("bfloat16 copy", ib16, hb.HK_Q_BF16),
                             ("float32 path", i16, hb.HK_Q_TIMING)):
        ids, dist, st = idx.query(Q, k, flags=flags)
        assert st["queries"] == B
        _check(ids, dist, oids, od2, "precision, " + name)
    i16.close()
    ib16.close()


def test_large_bench_batch(hb, oracle_lib):
    wl = _wl()
    N, n, tau, B, k = 100_000_000, 256, 100_000, 2000, 10
    stride = int(os.environ.get("HK_FULLSIZE_STRIDE", "8"))
    _need(N * n * 4 * 2.6)
    X = wl.random_walk(N, n, seed=0, device="cuda")
    Q_all, _ = wl.queries(X, 10_000, [0.5, 1.0], seed=1)   # bench.py's 10K queries
    Q = Q_all[:B].contiguous()                            # its first 2,000-query step
    idx = hb.Index(X, tau, flags=hb.HK_BUILD_FP16)
    del X
    _release()
    rows = np.arange(0, B, stride)
    t0 = time.perf_counter()
    oids, od2 = _oracle_rw(N, n, 0, Q.cpu().numpy()[rows], k)
    print("oracle: %d queries over %d series in %.0f s" % (rows.size, N, time.perf_counter() - t0))
    for name, flags in (("float16 tensor-core form", hb.HK_Q_BF16 | hb.HK_Q_TIMING),
                        ("float32 path", hb.HK_Q_TIMING)):
        ids, dist, st = idx.query(Q, k, flags=flags)
        assert st["queries"] == B
        _check(ids.cpu().numpy()[rows], dist.cpu().numpy()[rows], oids, od2, "large, " + name)
    idx.close()


def test_served_mix_every_request(hb, oracle_lib):
    """Requests of all four collections, k in {1, 10, 100}, submitted in
    interleaved waves (later waves arrive while earlier batches are on the
    GPU); each answer equals the oracle's for that request alone."""
    wl = _wl()
    per, waves = 48, 4
    total = sum(N * n * 4 for _, N, n, _, _ in wl.SERVED_MIX)
    _need(total * 2.6)
    Xs, idxs, Qs = [], [], []
    for ci, (name, N, n, kind, tau) in enumerate(wl.SERVED_MIX):
        X = wl.collection(kind, N, n, seed=10 + ci, device="cuda")
        Q, _ = wl.queries(X, per, wl.uniform_sigmas(per, 0.01, 1.0, seed=20 + ci), seed=20 + ci,
                          norm=wl.query_norm(kind))
        Xs.append(X)
        Qs.append(Q.cpu().numpy())
        idxs.append(hb.Index(X, tau, flags=hb.HK_BUILD_FP16 if n <= 256 else 0))
    sv = hb.Server(max_batch=1024, query_flags=hb.HK_Q_BF16, workers=2)
    colls = [sv.add(ix) for ix in idxs]
    rng = np.random.default_rng(2)
    order = [(ci, i) for ci in range(len(Xs)) for i in range(per)]
    rng.shuffle(order)
    ks = (1, 10, 100)
    tickets = {}
    for w in range(waves):
        for ci, i in order[w::waves]:
            tickets[(ci, i)] = sv.submit(colls[ci], Qs[ci][i], ks[i % 3])
        time.sleep(0.002)
    got = {}
    for key, t in tickets.items():
        r = None
        while r is None:
            r = sv.poll(t, ks[key[1] % 3], timeout_us=30_000_000)
        got[key] = r
    st = sv.stats()
    sv.close()
    assert st["errors"] == 0 and st["served"] == len(order)
    for ci, (name, N, n, kind, tau) in enumerate(wl.SERVED_MIX):
        oids, od2 = _oracle_dev(Xs[ci], Qs[ci], 100)
        for i in range(per):
            k = ks[i % 3]
            ids, dist, _ = got[(ci, i)]
            _check(ids[None, :], dist[None, :], oids[i:i + 1, :k], od2[i:i + 1, :k],
                   "%s, request %d (k=%d)" % (name, i, k))
    for ix in idxs:
        ix.close()


def test_n1024_float32_path(hb, oracle_lib):
    wl = _wl()
    N, n = 200_000, 1024
    X = wl.random_walk(N, n, seed=31, device="cuda")
    Q, _ = wl.queries(X, 48, [0.01, 0.1, 0.5, 1.0], seed=32)
    idx = hb.Index(X, 2000)
    oids, od2 = oracle.knn(X.cpu().numpy(), Q.cpu().numpy(), 100)
    for k in (1, 10, 100):
        ids, dist, _ = idx.query(Q, k)
        _check(ids, dist, oids[:, :k], od2[:, :k], "n=1024 k=%d" % k)
    # the exhaustive scan on the same collection
    ids, dist = hb.scan_knn(X, Q, 10)
    _check(ids, dist, oids[:, :10], od2[:, :10], "n=1024 scan")
    idx.close()
