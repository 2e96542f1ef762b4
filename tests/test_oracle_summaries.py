"""Pins for the oracle's summaries and lower bounds:
EAPCA segment statistics and LB_EAPCA (Sec. 2, Sec. 3.2), PAA, iSAX and
LB_SAX (Sec. 2, Sec. 3.4).

Closed forms, scipy/numpy as separate implementations, the no-false-dismissal
property of both bounds (Sec. 2: the filtering step prunes without false
dismissals), and special cases where a bound is attained exactly.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import tree as otree


# ---------------------------------------------------------------- segment stats
def test_seg_stats_closed_forms(oracle_lib):
    x = np.full(40, 1.75, np.float32)
    mu, sd = oracle.seg_stats(x, 3, 29)
    assert mu == 1.75 and sd == 0.0
    ramp = np.arange(64, dtype=np.float32)
    for a, b in [(0, 64), (5, 21), (10, 11)]:
        l = b - a
        mu, sd = oracle.seg_stats(ramp, a, b)
        assert mu == pytest.approx((a + b - 1) / 2, abs=1e-13)
        assert sd == pytest.approx(math.sqrt((l * l - 1) / 12.0), abs=1e-12)
    # only the requested range counts
    y = np.zeros(32, np.float32)
    y[:8] = 100.0
    assert oracle.seg_stats(y, 8, 32) == (0.0, 0.0)


def test_seg_stats_match_numpy(oracle_lib):
    rng = np.random.default_rng(7)
    x = rng.standard_normal(256).astype(np.float32)
    for a, b in [(0, 256), (0, 64), (64, 96), (200, 256), (17, 18)]:
        mu, sd = oracle.seg_stats(x, a, b)
        seg = x[a:b].astype(np.float64)
        assert mu == pytest.approx(seg.mean(), rel=1e-13, abs=1e-15)
        assert sd == pytest.approx(seg.std(ddof=0), rel=1e-12, abs=1e-15)


# ---------------------------------------------------------------- LB_EAPCA
def _envelope(X, rows, seg_end):
    env = np.empty((len(seg_end), 4))
    a = 0
    for j, b in enumerate(seg_end):
        mu, sd = oracle.seg_stats_rows(X, rows, a, b)
        env[j] = (mu.min(), mu.max(), sd.min(), sd.max())
        a = b
    return env


def test_lb_eapca_attained_on_piecewise_constant(oracle_lib):
    # q and x constant on every segment: D = sum_i l_i (mu_q - mu_x)^2 = LB.
    seg_end = [3, 8, 16, 32]
    lens = [3, 5, 8, 16]
    qv = [0.5, -1.0, 2.0, 0.25]
    xv = [-0.5, -1.0, 0.0, 1.25]
    q = np.concatenate([np.full(l, v, np.float32) for l, v in zip(lens, qv)])
    x = np.concatenate([np.full(l, v, np.float32) for l, v in zip(lens, xv)])
    env = _envelope(x[None], [0], seg_end)
    d = oracle.dist2(q, x)
    assert d == 3 * 1.0 + 0 + 8 * 4.0 + 16 * 1.0
    assert oracle.lb_eapca(q, seg_end, env) == d


def test_lb_eapca_std_term(oracle_lib):
    # q alternates +-a on a segment (mean 0, std a); x is 0 there.
    # D = l a^2 = l [(0-0)^2 + (a-0)^2] = LB: pins the std term and its weight.
    a = 1.5
    q = np.zeros(32, np.float32)
    q[8:16] = a * np.array([1, -1] * 4, np.float32)
    x = np.zeros(32, np.float32)
    seg_end = [8, 16, 24, 32]
    env = _envelope(x[None], [0], seg_end)
    assert oracle.dist2(q, x) == 8 * a * a
    assert oracle.lb_eapca(q, seg_end, env) == 8 * a * a


def test_lb_eapca_zero_inside_envelope(oracle_lib):
    rng = np.random.default_rng(11)
    X = rng.standard_normal((20, 64)).astype(np.float32)
    seg_end = [16, 32, 48, 64]
    env = _envelope(X, np.arange(20), seg_end)
    for i in range(20):
        assert oracle.lb_eapca(X[i], seg_end, env) == 0.0


def test_lb_eapca_direction(oracle_lib):
    # a query above the mean range is at distance (mu_q - mu_max), not
    # (mu_q - mu_min): shift a constant query past a one-member envelope.
    x = np.zeros(16, np.float32)
    env = _envelope(x[None], [0], [4, 8, 12, 16])
    env[:, 0] = -1.0          # mu range [-1, 0]
    for c in (0.5, -1.5):
        q = np.full(16, c, np.float32)
        expect = 16 * (0.5 ** 2)
        assert oracle.lb_eapca(q, [4, 8, 12, 16], env) == expect


@pytest.mark.parametrize("n", [16, 32, 64, 256])
def test_lb_eapca_never_exceeds_distance(oracle_lib, n):
    """No false dismissals (Sec. 2) on every query-series pair of a tiny set,
    with synopses over multi-member nodes of various segmentations."""
    rng = np.random.default_rng(n)
    X = np.cumsum(rng.standard_normal((120, n)), axis=1).astype(np.float32)
    Q = (X[:12] + rng.standard_normal((12, n)) * 2).astype(np.float32)
    segs = [otree.root_segmentation(n),
            sorted(set(otree.root_segmentation(n) + [n // 8, 3 * n // 8 + 1])),
            list(range(n // 16, n + 1, n // 16))]
    for seg_end in segs:
        for grp in np.array_split(np.arange(120), 6):
            env = _envelope(X, grp, seg_end)
            for q in Q:
                lb = oracle.lb_eapca(q, seg_end, env)
                for r in grp:
                    d = oracle.dist2(q, X[r])
                    assert lb <= d * (1 + 1e-12), (lb, d)


# ---------------------------------------------------------------- PAA / iSAX
def test_paa_closed_form(oracle_lib):
    x = np.arange(64, dtype=np.float32)
    p = oracle.paa(x, 16)
    np.testing.assert_array_equal(p, np.arange(16) * 4 + 1.5)


def test_breakpoints_match_scipy_and_symmetry(oracle_lib):
    stats = pytest.importorskip("scipy.stats")
    bp = oracle.isax_breakpoints()
    ref = stats.norm.ppf(np.arange(1, 256) / 256.0)
    np.testing.assert_allclose(bp, ref, rtol=0, atol=1e-13)
    assert bp[127] == 0.0                            # beta_128 = 0
    np.testing.assert_array_equal(bp, -bp[::-1])     # beta_{256-j} = -beta_j
    assert np.all(np.diff(bp) > 0)
    # Phi(beta_j) = j/256 with the library's erfc
    for j in (1, 2, 64, 128, 200, 255):
        phi = 0.5 * math.erfc(-bp[j - 1] / math.sqrt(2.0))
        assert phi == pytest.approx(j / 256.0, abs=1e-15)


def test_isax_symbol_rules(oracle_lib):
    bp = oracle.isax_breakpoints_f32()
    assert oracle.isax_symbol(-1e30, bp) == 0
    assert oracle.isax_symbol(1e30, bp) == 255
    assert oracle.isax_symbol(0.0, bp) == 128           # on beta_128: upper cell
    for j in (1, 50, 255):
        b = float(bp[j - 1])
        assert oracle.isax_symbol(b, bp) == j          # on a breakpoint: goes up
        assert oracle.isax_symbol(np.nextafter(b, -np.inf), bp) == j - 1
    vals = np.linspace(-4, 4, 301)
    syms = [oracle.isax_symbol(v, bp) for v in vals]
    assert syms == sorted(syms)


def test_lb_sax_exact_value(oracle_lib):
    # n = 16: segment length 1.  x's first segment sits in cell s; a query
    # value above the cell is at distance (p - beta_{s+1}), below it at
    # (beta_s - p); other segments inside their cells contribute 0.
    bp = oracle.isax_breakpoints_f32()
    x = np.zeros(16, np.float32)
    x[0] = 0.3
    sym = oracle.isax_word(x, bp)
    s = int(sym[0])
    assert bp[s - 1] <= 0.3 < bp[s]
    paa_q = oracle.paa(x, 16).copy()
    paa_q[0] = 2.0
    assert oracle.lb_sax(paa_q, sym, 16, bp) == pytest.approx((2.0 - float(bp[s])) ** 2, rel=1e-15)
    paa_q[0] = -1.0
    assert oracle.lb_sax(paa_q, sym, 16, bp) == pytest.approx((float(bp[s - 1]) + 1.0) ** 2, rel=1e-15)
    # weight n/w: the same cell distance on n = 64 counts 4 times
    assert oracle.lb_sax(paa_q, sym, 64, bp) == pytest.approx(4 * (float(bp[s - 1]) + 1.0) ** 2, rel=1e-15)


def test_lb_sax_zero_for_self(oracle_lib):
    bp = oracle.isax_breakpoints_f32()
    rng = np.random.default_rng(3)
    for _ in range(20):
        x = rng.standard_normal(128).astype(np.float32)
        assert oracle.lb_sax(oracle.paa(x), oracle.isax_word(x, bp), 128, bp) == 0.0


@pytest.mark.parametrize("n", [16, 32, 64, 256])
def test_lb_sax_never_exceeds_distance(oracle_lib, n):
    bp = oracle.isax_breakpoints_f32()
    rng = np.random.default_rng(100 + n)
    X = rng.standard_normal((150, n)).astype(np.float32)
    X = ((X - X.mean(1, keepdims=True)) / X.std(1, keepdims=True)).astype(np.float32)
    words = [oracle.isax_word(x, bp) for x in X]
    Q = X[:10] + rng.standard_normal((10, n)).astype(np.float32) * 0.7
    for q in Q:
        pq = oracle.paa(q)
        for x, w in zip(X, words):
            lb = oracle.lb_sax(pq, w, n, bp)
            assert lb <= oracle.dist2(q, x) * (1 + 1e-12)
