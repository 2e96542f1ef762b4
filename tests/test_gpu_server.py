"""The continuous-batching server: every request's answer equals the answer
of the same query alone (hk_query, and the brute-force oracle), whatever
batch it was answered in; bounded waits; argument checks."""
import threading

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


@pytest.fixture(scope="module")
def two_collections(hb):
    from paper_2212_13297_gb300 import workload as wl
    X1 = wl.random_walk(30_000, 64, seed=101, device="cuda")
    X2 = wl.gaussian(20_000, 128, seed=102, device="cuda", l2=True)
    i1 = hb.Index(X1, 300)
    i2 = hb.Index(X2, 300, flags=hb.HK_BUILD_FP16)
    Q1, _ = wl.queries(X1, 120, [0.05, 0.5, 1.0], seed=103)
    Q2, _ = wl.queries(X2, 80, [0.01, 0.1], seed=104, norm="l2")
    return dict(X=[X1, X2], idx=[i1, i2], Q=[Q1.cpu().numpy(), Q2.cpu().numpy()])


@pytest.mark.parametrize("flags", [0, "bf16"])
def test_mixed_requests_equal_their_answers_alone(hb, oracle_lib, two_collections, flags):
    c = two_collections
    qflags = hb.HK_Q_BF16 if flags == "bf16" else 0
    sv = hb.Server(max_batch=64, max_wait_us=200, query_flags=qflags, workers=2)
    coll = [sv.add(c["idx"][0]), sv.add(c["idx"][1])]
    rng = np.random.default_rng(7)
    reqs = []
    for i in range(120):
        reqs.append((0, i, int(rng.choice([1, 5, 20]))))
    for i in range(80):
        reqs.append((1, i, int(rng.choice([1, 10]))))
    rng.shuffle(reqs)
    tickets = [None] * len(reqs)

    def submit(part):
        for j in part:
            cidx, qi, k = reqs[j]
            tickets[j] = sv.submit(coll[cidx], c["Q"][cidx][qi], k)

    ths = [threading.Thread(target=submit, args=(range(p, len(reqs), 2),)) for p in range(2)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    got = []
    for j, (cidx, qi, k) in enumerate(reqs):
        r = sv.poll(tickets[j], k, timeout_us=30_000_000)
        assert r is not None
        got.append(r)
    st = sv.stats()
    assert st["served"] == len(reqs) and st["errors"] == 0 and st["pending"] == 0
    assert st["batches"] < len(reqs)          # requests were batched
    sv.close()
    # alone: the same query through hk_query
    for j, (cidx, qi, k) in enumerate(reqs):
        ids, dist, _ = c["idx"][cidx].query(c["Q"][cidx][qi:qi + 1], k)
        np.testing.assert_array_equal(got[j][0], ids[0])
        np.testing.assert_array_equal(got[j][1], dist[0])
    # and a sample against the oracle
    for cidx in (0, 1):
        Xh = c["X"][cidx].cpu().numpy()
        qs = [j for j, r in enumerate(reqs) if r[0] == cidx][:12]
        for j in qs:
            _, qi, k = reqs[j]
            oids, _ = oracle.knn(Xh, c["Q"][cidx][qi:qi + 1], k)
            np.testing.assert_array_equal(got[j][0], oids[0])


def test_poll_timeout_and_budget_cap(hb, two_collections):
    c = two_collections
    # a worker that lingers 300 ms for more requests: a 1 ms poll times out
    sv = hb.Server(max_batch=512, max_wait_us=300_000, workers=1)
    coll = sv.add(c["idx"][0])
    t = sv.submit(coll, c["Q"][0][0], 5)
    assert sv.poll(t, 5, timeout_us=1000) is None
    r = sv.poll(t, 5, timeout_us=10_000_000)
    assert r is not None and r[2] > 0
    sv.close()
    # a device budget that fits only a few queries caps the batch size
    sv = hb.Server(max_batch=512, max_wait_us=50_000, hbm_budget=64 << 20, workers=1)
    coll = sv.add(c["idx"][0])
    ts = [sv.submit(coll, c["Q"][0][i], 3) for i in range(60)]
    for i, t in enumerate(ts):
        ids, _, _ = sv.poll(t, 3, timeout_us=30_000_000)
        ref, _, _ = c["idx"][0].query(c["Q"][0][i:i + 1], 3)
        np.testing.assert_array_equal(ids, ref[0])
    st = sv.stats()
    assert st["max_batch"] < 60
    sv.close()


def test_server_rejects_bad_requests(hb, two_collections):
    c = two_collections
    sv = hb.Server(workers=1)
    coll = sv.add(c["idx"][0])
    q = c["Q"][0][0].copy()
    q[3] = np.nan
    with pytest.raises(hb.HerculesError) as e:
        sv.submit(coll, q, 1)
    assert e.value.code == hb.HK_EINVAL
    with pytest.raises(hb.HerculesError):
        sv.submit(coll + 5, c["Q"][0][0], 1)
    with pytest.raises(hb.HerculesError):
        sv.submit(coll, c["Q"][0][0], 2000)
    with pytest.raises(hb.HerculesError):
        sv.poll(987654, 1, timeout_us=10)
    sv.close()


def test_persistent_scan_admits_batches_midflight(hb, oracle_lib):
    """Persistent form: requests for three collections of different series
    lengths (64, 128, 256; float16 copies) arrive in waves while earlier
    batches are on the GPU; their tensor-core scans run as jobs of resident
    launches, batches admitted mid-flight joining a running launch and
    several collections sharing one.  Every answer equals the same query's
    answer alone (hk_query) and the oracle's."""
    import time
    from paper_2212_13297_gb300 import workload as wl
    Xs = [wl.random_walk(40_000, 64, seed=111, device="cuda"),
          wl.gaussian(30_000, 128, seed=112, device="cuda", l2=True),
          wl.random_walk(30_000, 256, seed=113, device="cuda")]
    norms = ["z", "l2", "z"]
    idxs = [hb.Index(X, 400, flags=hb.HK_BUILD_FP16) for X in Xs]
    Qs = [wl.queries(X, 90, [0.05, 0.5, 1.0], seed=114 + i, norm=norms[i])[0].cpu().numpy()
          for i, X in enumerate(Xs)]
    sv = hb.Server(max_batch=24, query_flags=hb.HK_Q_BF16, workers=4, persistent=1)
    colls = [sv.add(ix) for ix in idxs]
    rng = np.random.default_rng(9)
    reqs = [(c, i, int(rng.choice([1, 10, 50]))) for c in range(3) for i in range(90)]
    rng.shuffle(reqs)
    tickets = []
    for w0 in range(0, len(reqs), 45):          # six waves, a few ms apart
        for c, i, k in reqs[w0:w0 + 45]:
            tickets.append(sv.submit(colls[c], Qs[c][i], k))
        time.sleep(0.004)
    got = []
    for t, (c, i, k) in zip(tickets, reqs):
        r = sv.poll(t, k, timeout_us=60_000_000)
        assert r is not None
        got.append(r)
    st = sv.stats()
    sv.close()
    assert st["errors"] == 0 and st["served"] == len(reqs)
    assert st["scan_jobs"] >= st["batches"] > 0
    assert st["scan_launches"] < st["scan_jobs"]        # launches took several batches' scans
    assert st["scan_jobs_inflight"] > 0                # scans admitted while a launch ran
    assert st["scan_max_collections"] >= 2             # collections of different n in one launch
    for (c, i, k), r in zip(reqs, got):
        ids, dist, _ = idxs[c].query(Qs[c][i:i + 1], k, flags=hb.HK_Q_BF16)
        np.testing.assert_array_equal(r[0], ids[0])
        np.testing.assert_array_equal(r[1], dist[0])
    for c in range(3):
        sel = [j for j, rq in enumerate(reqs) if rq[0] == c][:20]
        qs = np.stack([Qs[c][reqs[j][1]] for j in sel])
        oids, _ = oracle.knn(Xs[c].cpu().numpy(), qs, 50)
        for row, j in enumerate(sel):
            k = reqs[j][2]
            np.testing.assert_array_equal(got[j][0], oids[row, :k])


def test_budget_admits_as_memory_frees(hb, two_collections):
    """A device budget that holds only a few queries' work spaces: workers
    admit what fits beside the batches in flight and wait for memory to free
    up; every request is answered and the budget is never exceeded."""
    c = two_collections
    budget = 96 << 20
    sv = hb.Server(max_batch=256, hbm_budget=budget, workers=3)
    coll = sv.add(c["idx"][0])
    ts = [sv.submit(coll, c["Q"][0][i % 120], 3) for i in range(150)]
    for i, t in enumerate(ts):
        ids, _, _ = sv.poll(t, 3, timeout_us=60_000_000)
        ref, _, _ = c["idx"][0].query(c["Q"][0][(i % 120):(i % 120) + 1], 3)
        np.testing.assert_array_equal(ids, ref[0])
    st = sv.stats()
    sv.close()
    assert st["errors"] == 0 and st["served"] == 150
    assert 0 < st["budget_peak"] <= budget
    assert st["max_batch"] < 150


def test_persistent_scan_relaunches_after_idle(hb, oracle_lib, two_collections):
    """The resident launch leaves after a short idle period; a batch that
    arrives later starts another launch.  A collection without a 16-bit copy
    (float32 path) is served beside it."""
    import time
    c = two_collections
    sv = hb.Server(max_batch=16, query_flags=hb.HK_Q_BF16, workers=2, persistent=1)
    coll16 = sv.add(c["idx"][1])                 # float16 copy: tensor-core scans
    coll32 = sv.add(c["idx"][0])                 # no 16-bit copy: float32 path
    got = []
    for wave in range(3):
        ts = [(sv.submit(coll16, c["Q"][1][wave * 10 + i], 7), 1, wave * 10 + i) for i in range(10)]
        ts += [(sv.submit(coll32, c["Q"][0][wave * 10 + i], 4), 0, wave * 10 + i) for i in range(5)]
        for t, ci, qi in ts:
            k = 7 if ci == 1 else 4
            r = sv.poll(t, k, timeout_us=60_000_000)
            assert r is not None
            got.append((ci, qi, k, r))
        time.sleep(0.05)                         # far longer than the launch's idle period
    st = sv.stats()
    sv.close()
    assert st["errors"] == 0 and st["scan_launches"] >= 3
    for ci, qi, k, r in got:
        flags = hb.HK_Q_BF16 if ci == 1 else 0
        ids, dist, _ = c["idx"][ci].query(c["Q"][ci][qi:qi + 1], k, flags=flags)
        np.testing.assert_array_equal(r[0], ids[0])
        np.testing.assert_array_equal(r[1], dist[0])


def test_collection_opts_and_tuned_configuration(hb, two_collections):
    """hk_server_add_opts: each collection's batches run with its own query
    configuration -- here hk_tune's choice for the float16 collection and two
    hand-set ones for the float32 collection -- and every answer equals
    hk_query's for the same query with the same options; invalid options are
    refused when the collection is added."""
    c = two_collections
    keys = ("l_max", "eapca_th", "sax_th", "flags", "query_group", "series_tile")
    tuned = c["idx"][1].tune(c["Q"][1][:32], 10)
    tuned = {k: tuned[k] for k in keys}
    hand = [dict(query_group=2, series_tile=4096, eapca_th=1.01, flags=hb.HK_Q_NOSAX),
            dict(flags=hb.HK_Q_TREE, l_max=2)]
    sv = hb.Server(max_batch=32, max_wait_us=200, workers=2)
    setups = [(1, tuned), (0, hand[0]), (0, hand[1])]
    coll = [sv.add(c["idx"][i], opts=o) for i, o in setups]
    reqs = [(s, qi, k) for s in range(3) for qi, k in zip(range(40), [1, 10, 3, 10] * 10)]
    tickets = [sv.submit(coll[s], c["Q"][setups[s][0]][qi], k) for s, qi, k in reqs]
    got = [sv.poll(t, k, timeout_us=30_000_000) for t, (_, _, k) in zip(tickets, reqs)]
    st = sv.stats()
    assert st["served"] == len(reqs) and st["errors"] == 0
    sv.close()
    for (s, qi, k), r in zip(reqs, got):
        i, o = setups[s]
        ids, dist, _ = c["idx"][i].query(c["Q"][i][qi:qi + 1], k, **o)
        np.testing.assert_array_equal(r[0], ids[0])
        np.testing.assert_array_equal(r[1], dist[0])
    sv = hb.Server()
    for i, o in [(0, dict(flags=hb.HK_Q_BF16)),                       # no 16-bit copy
                 (1, dict(flags=hb.HK_Q_BF16 | hb.HK_Q_NOPRUNE)),
                 (0, dict(flags=hb.HK_Q_TREE | hb.HK_Q_NOPRUNE)),
                 (0, dict(query_group=-1)), (0, dict(l_max=-2))]:
        with pytest.raises(hb.HerculesError) as e:
            sv.add(c["idx"][i], opts=o)
        assert e.value.code == hb.HK_EINVAL
    sv.close()
