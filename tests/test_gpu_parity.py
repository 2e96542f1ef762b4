"""Parity of the CUDA path with the oracle, through the C ABI.

Tree: the GPU's level-by-level build must produce exactly the tree that
sequential insertion (Algorithm InsertSeriesToNode) gives, with identical
segmentations, synopses (binary64, bit for bit) and iSAX words.
Bounds: LB_EAPCA bit for bit; LB_SAX as a certified lower value.
Answers: ids identical to the brute-force oracle (ties to the lower id) and
distances within 1e-5 relative (they are the same binary64 values rounded to
float32, so in practice equal).
"""
import numpy as np
import pytest

import oracle
from oracle import tree as otree

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


def check_answers(ids, dist, X_host, Q_host, k):
    oids, od2 = oracle.knn(X_host, Q_host, k)
    odist = np.sqrt(od2).astype(np.float32)
    ids = ids.cpu().numpy() if hasattr(ids, "cpu") else ids
    dist = dist.cpu().numpy() if hasattr(dist, "cpu") else dist
    np.testing.assert_array_equal(ids, oids)
    np.testing.assert_allclose(dist, odist, rtol=1e-5, atol=0)
    return oids, odist


def leaves_from_export(ex):
    out = []
    for p in range(len(ex["nseg"])):
        a, b = ex["leaf_off"][p], ex["leaf_off"][p + 1]
        out.append((ex["perm"][a:b].tolist(), ex["seg_end"][p, :ex["nseg"][p]].tolist()))
    return out


@pytest.mark.parametrize("N,n,tau,eval_cap", [(2500, 64, 60, 0), (1800, 96, 40, 0),
                                              (2000, 16, 30, 0), (3000, 64, 200, 25)])
def test_tree_synopses_and_words_match_oracle(hb, oracle_lib, N, n, tau, eval_cap):
    X = _wl().random_walk(N, n, seed=N + n, device="cuda")
    Xh = X.cpu().numpy()
    idx = hb.Index(X, tau, eval_cap=eval_cap)
    ex = idx.export()
    root = otree.build_tree(Xh, tau, eval_cap=eval_cap or otree.EVAL_CAP)
    oleaves = otree.leaves_inorder(root)
    gleaves = leaves_from_export(ex)
    assert len(gleaves) == len(oleaves)
    for (members, seg), ol in zip(gleaves, oleaves):
        assert members == ol.members
        assert seg == ol.seg_end
    for p, ol in enumerate(oleaves):
        env = otree.leaf_synopsis(Xh, ol)
        np.testing.assert_array_equal(ex["env"][p, :len(ol.seg_end)], env)
    bp = oracle.isax_breakpoints_f32()
    for pos in range(0, N, 7):
        np.testing.assert_array_equal(ex["sax"][pos], oracle.isax_word(Xh[ex["perm"][pos]], bp))
    info = idx.info()
    assert info["leaves"] == len(oleaves) and info["N"] == N


def test_lb_eapca_bit_exact_and_lb_sax_certified(hb, oracle_lib):
    N, n, tau = 4000, 64, 100
    wl = _wl()
    X = wl.random_walk(N, n, seed=3, device="cuda")
    Xh = X.cpu().numpy()
    Q, _ = wl.queries(X, 12, [0.1, 0.5, 1.0], seed=4)
    Qh = Q.cpu().numpy()
    idx = hb.Index(X, tau)
    ex = idx.export()
    lb = idx.debug_lb_eapca(Q)
    for p in range(len(ex["nseg"])):
        seg = ex["seg_end"][p, :ex["nseg"][p]]
        env = ex["env"][p, :len(seg)]
        for qi in range(len(Qh)):
            assert lb[qi, p] == oracle.lb_eapca(Qh[qi], seg, env)
    lbs = idx.debug_lb_sax(Q)
    bp = oracle.isax_breakpoints_f32()
    for qi in range(len(Qh)):
        pq = oracle.paa(Qh[qi])
        for pos in range(0, N, 13):
            ref = oracle.lb_sax(pq, ex["sax"][pos], n, bp)
            assert lbs[qi, pos] <= ref
            # float32 arithmetic rounded down at every step from the PAA
            # bracketed in float32: a few float32 roundings relative, plus
            # the PAA's own rounding (absolute, at most w * 2^-12 here)
            assert lbs[qi, pos] >= ref * (1 - 2.0**-14) - (n // 16) * 2.0**-12
            # and it lower-bounds the true distance
            assert lbs[qi, pos] <= oracle.dist2(Qh[qi], Xh[ex["perm"][pos]])


@pytest.mark.parametrize("N,n,tau,nq,k,sig", [
    (20000, 64, 200, 16, 1, 0.1),
    (20000, 64, 200, 16, 10, 0.5),
    (5000, 256, 100, 8, 100, 1.0),
    (6000, 96, 150, 9, 5, 0.2),
    (3000, 16, 50, 8, 3, 0.3),
])
def test_query_matches_bruteforce(hb, oracle_lib, N, n, tau, nq, k, sig):
    wl = _wl()
    X = wl.random_walk(N, n, seed=N + k, device="cuda")
    Q, _ = wl.queries(X, nq, sig, seed=k)
    idx = hb.Index(X, tau)
    ids, dist, st = idx.query(Q, k)
    check_answers(ids, dist, X.cpu().numpy(), Q.cpu().numpy(), k)
    assert st["queries"] == nq


def test_query_flags_same_answer(hb, oracle_lib):
    wl = _wl()
    X = wl.random_walk(15000, 128, seed=9, device="cuda")
    Q, _ = wl.queries(X, 12, [0.01, 0.3, 1.0], seed=9)
    idx = hb.Index(X, 120)
    Xh, Qh = X.cpu().numpy(), Q.cpu().numpy()
    variants = [dict(), dict(flags=hb.HK_Q_NOSAX), dict(flags=hb.HK_Q_NOTHRESH),
                dict(flags=hb.HK_Q_NOPRUNE), dict(l_max=7), dict(query_group=1),
                dict(query_group=4, series_tile=64), dict(eapca_th=0.99)]
    for v in variants:
        ids, dist, st = idx.query(Q, 8, **v)
        check_answers(ids, dist, Xh, Qh, 8)
    _, _, st = idx.query(Q, 8, flags=hb.HK_Q_NOPRUNE)
    assert st["series_candidate"] == 15000 * 12


def test_gaussian_l2_collection(hb, oracle_lib):
    wl = _wl()
    X = wl.gaussian(12000, 96, seed=5, device="cuda", l2=True)
    Q, _ = wl.queries(X, 10, [0.01, 0.05], seed=6, norm="l2")
    idx = hb.Index(X, 100)
    ids, dist, _ = idx.query(Q, 10)
    check_answers(ids, dist, X.cpu().numpy(), Q.cpu().numpy(), 10)


def test_duplicates_ties_and_fallback(hb, oracle_lib):
    wl = _wl()
    X = wl.random_walk(5000, 64, seed=11, device="cuda")
    X[1000:1150] = X[17]          # 151 identical series
    X[4000] = X[17]
    Q = X[[17, 17, 3]].clone()
    idx = hb.Index(X, 80)
    ids, dist, st = idx.query(Q, 10)
    oids, _ = check_answers(ids, dist, X.cpu().numpy(), Q.cpu().numpy(), 10)
    assert list(oids[0]) == [17] + list(range(1000, 1009))
    # 153 exact ties exceed a work item's list (k + 32 entries): those
    # queries are finished by the exhaustive collection
    assert st["fallback_queries"] == 2
    ids, dist, st = idx.query(Q, 200)
    check_answers(ids, dist, X.cpu().numpy(), Q.cpu().numpy(), 200)


def test_scan_knn_matches_bruteforce(hb, oracle_lib):
    wl = _wl()
    X = wl.random_walk(30000, 128, seed=21, device="cuda")
    Q, _ = wl.queries(X, 10, [0.1, 1.0], seed=22)
    for k in (1, 7, 64):
        ids, dist = hb.scan_knn(X, Q, k)
        check_answers(ids, dist, X.cpu().numpy(), Q.cpu().numpy(), k)


def test_small_config_bruteforce_parity(hb, oracle_lib):
    """100,000 random walks x 256, leaf capacity 1,000, 10 queries with
    N(0, 0.1^2) noise, k = 1 (and k = 10)."""
    wl = _wl()
    X = wl.random_walk(100_000, 256, seed=0, device="cuda")
    Q, _ = wl.queries(X, 10, 0.1, seed=1)
    idx = hb.Index(X, 1000)
    Xh, Qh = X.cpu().numpy(), Q.cpu().numpy()
    for k in (1, 10):
        ids, dist, st = idx.query(Q, k)
        check_answers(ids, dist, Xh, Qh, k)


def test_host_buffers_and_replay(hb, oracle_lib):
    wl = _wl()
    X = wl.random_walk(8000, 64, seed=31, device="cuda")
    Q, _ = wl.queries(X, 6, 0.4, seed=32)
    Xh, Qh = X.cpu().numpy(), Q.cpu().numpy()
    idx = hb.Index(Xh, 100)              # host collection
    ids, dist, _ = idx.query(Qh, 5)      # host queries and outputs
    assert isinstance(ids, np.ndarray)
    check_answers(ids, dist, Xh, Qh, 5)
    ids2, dist2, _ = idx.query(Qh, 5)
    np.testing.assert_array_equal(ids, ids2)
    np.testing.assert_array_equal(dist, dist2)


def test_edge_cases(hb, oracle_lib):
    wl = _wl()
    # one series
    X = wl.random_walk(1, 32, seed=1, device="cuda")
    idx = hb.Index(X, 10)
    ids, dist, _ = idx.query(X.clone(), 1)
    assert ids.item() == 0 and dist.item() == 0.0
    # k = N, a single leaf and leaves of one series
    X = wl.random_walk(40, 32, seed=2, device="cuda")
    Q, _ = wl.queries(X, 3, 0.5, seed=3)
    for tau in (1, 5, 100):
        idx = hb.Index(X, tau)
        ids, dist, _ = idx.query(Q, 40)
        check_answers(ids, dist, X.cpu().numpy(), Q.cpu().numpy(), 40)
    # the longest series
    X = wl.random_walk(300, 4096, seed=4, device="cuda")
    Q, _ = wl.queries(X, 2, 0.2, seed=5)
    idx = hb.Index(X, 50)
    ids, dist, _ = idx.query(Q, 3)
    check_answers(ids, dist, X.cpu().numpy(), Q.cpu().numpy(), 3)
    # a constant collection: no split is possible, one over-full leaf
    X = torch.zeros((500, 16), device="cuda")
    idx = hb.Index(X, 10)
    assert idx.info()["leaves"] == 1
    ids, dist, _ = idx.query(torch.ones((1, 16), device="cuda"), 4)
    assert ids.cpu().tolist() == [[0, 1, 2, 3]]


def test_largest_k_and_many_candidates_at_the_bound(hb, oracle_lib):
    """k = HK_MAX_K = 1024.  One query equals a row copied 2,000 times, so
    more than 1,024 candidates sit at the final bound (the selection over the
    pool in global memory); the others leave about k (the shared-memory
    sort).  Plain and precision forms."""
    wl = _wl()
    X = wl.random_walk(6000, 64, seed=21, device="cuda")
    X[1000:3000] = X[17]
    Q = torch.cat([X[[17]], wl.queries(X, 3, [0.3, 1.0], seed=22)[0]]).contiguous()
    for qflags, bflags in ((0, 0), (hb.HK_Q_BF16, hb.HK_BUILD_FP16)):
        idx = hb.Index(X, 200, flags=bflags)
        ids, dist, _ = idx.query(Q, 1024, flags=qflags)
        check_answers(ids, dist, X.cpu().numpy(), Q.cpu().numpy(), 1024)
        assert ids[0].cpu().tolist() == [17] + list(range(1000, 2023))


def test_rejects_nonfinite_and_bad_k(hb):
    wl = _wl()
    X = wl.random_walk(100, 32, seed=1, device="cuda")
    idx = hb.Index(X, 10)
    Q = X[:2].clone()
    Q[1, 5] = float("nan")
    with pytest.raises(hb.HerculesError) as e:
        idx.query(Q, 1)
    assert e.value.code == hb.HK_EINVAL
    with pytest.raises(hb.HerculesError):
        idx.query(X[:1].clone(), 101)
    Xb = X.clone()
    Xb[3, 3] = float("inf")
    with pytest.raises(hb.HerculesError):
        hb.Index(Xb, 10)
