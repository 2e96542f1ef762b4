"""Precision form: tensor-core distances with a certified bound.

The bound is pinned pair by pair: for every query and series, the
tensor-core value D~ = |q|^2 + |x|^2 - 2 q^.x^ must lie within E of the exact
squared distance (binary64 from numpy, a separate implementation), so the
candidate filter never drops a true neighbour.  Answers through the
precision form must equal the brute-force oracle's.
"""
import zlib

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


@pytest.mark.parametrize("fmt", ["bf16", "fp16"])
@pytest.mark.parametrize("N,n,kind", [(3000, 256, "rw"), (2500, 64, "rw"), (2000, 96, "gauss"),
                                      (1800, 128, "rw")])
def test_tc_distance_within_certified_bound(hb, N, n, kind, fmt):
    wl = _wl()
    X = wl.random_walk(N, n, seed=N, device="cuda") if kind == "rw" else \
        wl.gaussian(N, n, seed=N, device="cuda")
    Q, _ = wl.queries(X, 9, [0.01, 0.5, 1.0], seed=3, norm="z" if kind == "rw" else None)
    idx = hb.Index(X, 100, flags=hb.HK_BUILD_BF16 if fmt == "bf16" else hb.HK_BUILD_FP16)
    assert idx.info()["has_bf16"] == 1
    ex = idx.export()
    lo, up = idx.debug_tc_dist(Q)
    Xl = X.cpu().numpy().astype(np.float64)[ex["perm"]]
    Qh = Q.cpu().numpy().astype(np.float64)
    exact = ((Qh[:, None, :] - Xl[None, :, :]) ** 2).sum(-1)
    assert np.isfinite(lo).all() and np.isfinite(up).all(), "some pairs were not computed"
    assert (lo <= exact).all(), float((lo - exact).max())
    assert (up >= exact).all(), float((exact - up).max())
    # the interval is not vacuous: its half-width stays small next to typical
    # distances, and the bfloat16 rounding uses a visible part of it
    half = (up.astype(np.float64) - lo) / 2
    mid = (up.astype(np.float64) + lo) / 2
    assert float(np.median(half / exact)) < (0.05 if fmt == "bf16" else 0.008)
    assert (0.01 if fmt == "bf16" else 0.002) < float(np.median(np.abs(mid - exact) / half)) < 0.5


@pytest.mark.parametrize("N,n,tau,nq,k,sig,fmt", [
    (20000, 256, 300, 20, 10, [0.5, 1.0], "bf16"),
    (20000, 256, 300, 150, 1, [0.3, 1.0], "bf16"),
    (15000, 64, 200, 30, 50, [0.1, 1.0], "bf16"),
    (12000, 96, 150, 16, 5, [0.5], "bf16"),
    (20000, 256, 300, 150, 10, [0.01, 0.5, 1.0], "fp16"),
    (15000, 128, 200, 30, 50, [0.1, 1.0], "fp16"),
])
def test_tc_query_matches_bruteforce(hb, oracle_lib, N, n, tau, nq, k, sig, fmt):
    wl = _wl()
    X = wl.random_walk(N, n, seed=N + n, device="cuda")
    Q, _ = wl.queries(X, nq, sig, seed=k)
    idx = hb.Index(X, tau, flags=hb.HK_BUILD_BF16 if fmt == "bf16" else hb.HK_BUILD_FP16)
    ids, dist, st = idx.query(Q, k, flags=hb.HK_Q_BF16)
    oids, od2 = oracle.knn(X.cpu().numpy(), Q.cpu().numpy(), k)
    np.testing.assert_array_equal(ids.cpu().numpy(), oids)
    np.testing.assert_allclose(dist.cpu().numpy(), np.sqrt(od2).astype(np.float32), rtol=1e-5)
    assert st["tc_pairs"] > 0
    # the plain path gives the same answer
    ids2, _, _ = idx.query(Q, k)
    np.testing.assert_array_equal(ids2.cpu().numpy(), oids)


def test_tc_ties_and_flag_checks(hb, oracle_lib):
    wl = _wl()
    X = wl.random_walk(6000, 128, seed=8, device="cuda")
    X[3000:3040] = X[9]
    Q = torch.cat([X[[9]], wl.queries(X, 3, 0.7, seed=2)[0]]).contiguous()
    idx = hb.Index(X, 100, flags=hb.HK_BUILD_BF16)
    ids, dist, _ = idx.query(Q, 20, flags=hb.HK_Q_BF16)
    oids, _ = oracle.knn(X.cpu().numpy(), Q.cpu().numpy(), 20)
    np.testing.assert_array_equal(ids.cpu().numpy(), oids)
    plain = hb.Index(X, 100)
    with pytest.raises(hb.HerculesError) as e:
        plain.query(Q, 5, flags=hb.HK_Q_BF16)
    assert e.value.code == hb.HK_EINVAL


@pytest.mark.parametrize("fmt", ["bf16", "fp16"])
def test_tc_long_items_match_bruteforce(hb, oracle_lib, fmt):
    """Items spanning many tiles (so the producer, MMA and epilogue run
    several tiles apart) on hard queries with bounds tightening in flight."""
    wl = _wl()
    X = wl.random_walk(400_000, 256, seed=77, device="cuda")
    Q, _ = wl.queries(X, 160, [0.5, 1.0], seed=78)
    idx = hb.Index(X, 20_000, flags=hb.HK_BUILD_BF16 if fmt == "bf16" else hb.HK_BUILD_FP16)
    ids, dist, st = idx.query(Q, 10, flags=hb.HK_Q_BF16)
    sel = np.arange(0, 160, 8)
    oids, od2 = oracle.knn(X.cpu().numpy(), Q.cpu().numpy()[sel], 10)
    np.testing.assert_array_equal(ids.cpu().numpy()[sel], oids)
    np.testing.assert_allclose(dist.cpu().numpy()[sel], np.sqrt(od2).astype(np.float32), rtol=1e-5)


def test_fp16_range_checked(hb):
    wl = _wl()
    X = wl.random_walk(2000, 64, seed=5, device="cuda")
    Xb = X.clone()
    Xb[7, 3] = 70000.0
    with pytest.raises(hb.HerculesError) as e:
        hb.Index(Xb, 100, flags=hb.HK_BUILD_FP16)
    assert e.value.code == hb.HK_EINVAL
    idx = hb.Index(X, 100, flags=hb.HK_BUILD_FP16)
    Q = X[:2].clone()
    Q[1, 0] = -1e5
    with pytest.raises(hb.HerculesError):
        idx.query(Q, 3, flags=hb.HK_Q_BF16)


@pytest.mark.parametrize("fmt", ["bf16", "fp16"])
def test_tc_edge_cases(hb, oracle_lib, fmt):
    """The precision form at its edges: one series, k = N with leaves of one
    series up to a single leaf, the shortest series (16 points), a lone
    query, and batches that cross the 128-row query block."""
    wl = _wl()
    bf = hb.HK_BUILD_BF16 if fmt == "bf16" else hb.HK_BUILD_FP16
    X = wl.random_walk(1, 32, seed=11, device="cuda")
    idx = hb.Index(X, 10, flags=bf)
    ids, dist, _ = idx.query(X.clone(), 1, flags=hb.HK_Q_BF16)
    assert ids.item() == 0 and dist.item() == 0.0
    X = wl.random_walk(40, 32, seed=12, device="cuda")
    Q, _ = wl.queries(X, 3, 0.5, seed=13)
    for tau in (1, 5, 100):
        idx = hb.Index(X, tau, flags=bf)
        ids, dist, _ = idx.query(Q, 40, flags=hb.HK_Q_BF16)
        oids, od2 = oracle.knn(X.cpu().numpy(), Q.cpu().numpy(), 40)
        np.testing.assert_array_equal(ids.cpu().numpy(), oids)
        np.testing.assert_allclose(dist.cpu().numpy(), np.sqrt(od2).astype(np.float32), rtol=1e-5)
    X = wl.random_walk(3000, 16, seed=14, device="cuda")
    idx = hb.Index(X, 100, flags=bf)
    for nq in (1, 129, 300):
        Q, _ = wl.queries(X, nq, [0.2, 1.0], seed=nq)
        ids, dist, _ = idx.query(Q, 7, flags=hb.HK_Q_BF16)
        oids, od2 = oracle.knn(X.cpu().numpy(), Q.cpu().numpy(), 7)
        np.testing.assert_array_equal(ids.cpu().numpy(), oids)
        np.testing.assert_allclose(dist.cpu().numpy(), np.sqrt(od2).astype(np.float32), rtol=1e-5)


def _adversarial(kind, N, n, fmt, rng):
    """Rows and queries that stress the float32 accumulation and the 16-bit
    rounding: every pair's interval must still hold the exact distance."""
    big = 2.0e4 if fmt == "fp16" else 1.0e15     # float16 holds up to 65504
    if kind == "cancel":          # q ~ x with large norms: D << |q||x|
        X = rng.standard_normal((N, n)) * big / 4
        src = rng.integers(0, N, 24)
        Q = X[src] * (1 + 1e-3 * rng.standard_normal((24, n)))
    elif kind == "alternating":   # products alternate in sign along the sum
        mag = np.abs(rng.standard_normal((N, n))) * big / 8
        X = mag * np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
        Q = np.abs(rng.standard_normal((24, n))) * big / 8
        Q[12:] *= np.where(np.arange(n) % 2 == 0, -1.0, 1.0)
    elif kind == "near_max":      # magnitudes close to the format's largest
        # bfloat16: large, yet squared distances stay inside float32's range
        top = 65504.0 if fmt == "fp16" else 1.0e17
        X = rng.choice([-1.0, 1.0], (N, n)) * rng.uniform(0.9, 1.0, (N, n)) * top
        Q = rng.choice([-1.0, 1.0], (24, n)) * rng.uniform(0.9, 1.0, (24, n)) * top
    elif kind == "wide_range":    # signs and binary exponents spread over 2^-12 .. 2^12
        X = rng.choice([-1.0, 1.0], (N, n)) * np.exp2(rng.integers(-12, 13, (N, n)))
        Q = rng.choice([-1.0, 1.0], (24, n)) * np.exp2(rng.integers(-12, 13, (24, n)))
    elif kind == "tiny":          # float16 subnormal range and below
        X = rng.standard_normal((N, n)) * 1e-6
        Q = rng.standard_normal((24, n)) * 1e-6
    else:
        raise ValueError(kind)
    return X.astype(np.float32), Q.astype(np.float32)


@pytest.mark.parametrize("fmt", ["bf16", "fp16"])
@pytest.mark.parametrize("kind", ["cancel", "alternating", "near_max", "wide_range", "tiny"])
@pytest.mark.parametrize("n", [16, 64, 256])
def test_tc_bound_adversarial(hb, kind, n, fmt):
    rng = np.random.default_rng(zlib.crc32(("%s/%d/%s" % (kind, n, fmt)).encode()))
    X, Q = _adversarial(kind, 700, n, fmt, rng)
    Xd = torch.from_numpy(X).cuda()
    idx = hb.Index(Xd, 64, flags=hb.HK_BUILD_BF16 if fmt == "bf16" else hb.HK_BUILD_FP16)
    ex = idx.export()
    lo, up = idx.debug_tc_dist(torch.from_numpy(Q).cuda())
    Xl = X.astype(np.float64)[ex["perm"]]
    exact = ((Q.astype(np.float64)[:, None, :] - Xl[None, :, :]) ** 2).sum(-1)
    assert not np.isnan(lo).any() and not np.isnan(up).any(), "some pairs were not computed"
    lo64, up64 = lo.astype(np.float64), up.astype(np.float64)
    assert (lo64 <= exact).all(), (kind, float((lo64 - exact).max()))
    assert (up64 >= exact).all(), (kind, float((exact - up64).max()))


def test_tc_candidate_list_overflow_reruns_exactly(hb, oracle_lib):
    """A query whose certified band admits more candidates than its list
    holds (300,000 copies of one row: every copy is a candidate) is rerun on
    the float32 path and still gets the exact answer, ties to the lower id."""
    wl = _wl()
    base = wl.random_walk(1, 16, seed=31, device="cuda")
    other = wl.random_walk(2000, 16, seed=32, device="cuda")
    X = torch.cat([other[:1000], base.repeat(300_000, 1), other[1000:]]).contiguous()
    Q = torch.cat([base, wl.queries(other, 2, 0.5, seed=33)[0]]).contiguous()
    idx = hb.Index(X, 10_000, flags=hb.HK_BUILD_FP16)
    ids, dist, st = idx.query(Q, 3, flags=hb.HK_Q_BF16)
    oids, od2 = oracle.knn(X.cpu().numpy(), Q.cpu().numpy(), 3)
    np.testing.assert_array_equal(ids.cpu().numpy(), oids)
    np.testing.assert_allclose(dist.cpu().numpy(), np.sqrt(od2).astype(np.float32), rtol=1e-5)
    assert list(ids[0].cpu().numpy()) == [1000, 1001, 1002]
    assert st["retried_queries"] >= 1
