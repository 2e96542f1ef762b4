"""Oracle for Hercules exact k-NN (Echihabi et al., PVLDB 15(10), 2022).

TEST INFRASTRUCTURE ONLY.  A plain, slow, obviously correct CPU restatement of
what the query path computes, in binary64.  Only tests/, the smoke check and
the benchmark's CPU-baseline leg may import it; the product path never does,
and the CUDA library shares no code, header, table or constant generator with
it.  Each function cites the passage it follows:

  dist2, knn, KnnStream    Sec. 2: k-NN query over the Euclidean distance;
                           answer ordered by (squared distance, id)
  seg_stats, seg_stats_rows  Sec. 3.2: EAPCA segment mean and population std
  lb_eapca                 Sec. 2 / Sec. 3.4 (Approx-kNN, FindCandidateLeaves):
                           LB_EAPCA of a query to a node synopsis
  paa                      Sec. 2: PAA with 16 equal segments
  isax_breakpoints         Sec. 2: alphabet 256, standard normal quantiles
  isax_symbol, isax_word   Sec. 2: iSAX symbols of PAA values
  lb_sax                   Sec. 3.4 (CSWorker, CRWorker): LB_SAX
  dtw2, dtw_knn, DtwKnnStream  Sec. 2: DTW (squared point costs, Sakoe-Chiba
                           band) as a distance with a lower bound, and k-NN
                           under it
  envelope, lb_keogh, lb_keogh_eapca, lb_keogh_sax
                           LB_Keogh (Keogh & Ratanamahatana 2005, the bound
                           the paper cites for DTW) and its forms against a
                           node synopsis and an iSAX word
  tree.build_tree          Sec. 3.2 and Algorithm InsertSeriesToNode (Sec. 3.3):
                           sequential insertion with H/V node splits; the split
                           policy, which the paper leaves to DSTree, is the
                           reading given in tree.py

Every function has parity pins in tests/test_oracle_*.py (closed forms,
library routines, invariants, the paper's worked split example).
"""
import ctypes
import os

import numpy as np

from . import build as _build

_LIB = None

W_PAA = 16          # PAA / iSAX segments (Sec. 2)
ALPHABET = 256      # iSAX alphabet (Sec. 2)


def _lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        f32p = ctypes.POINTER(ctypes.c_float)
        f64p = ctypes.POINTER(ctypes.c_double)
        i64p = ctypes.POINTER(ctypes.c_int64)
        i32p = ctypes.POINTER(ctypes.c_int32)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        L.hko_dist2.restype = ctypes.c_double
        L.hko_dist2.argtypes = [f32p, f32p, ctypes.c_int]
        L.hko_knn_init.restype = None
        L.hko_knn_init.argtypes = [ctypes.c_int, ctypes.c_int, i64p, f64p]
        L.hko_knn_update.restype = ctypes.c_int
        L.hko_knn_update.argtypes = [f32p, ctypes.c_int64, ctypes.c_int64,
                                     ctypes.c_int, f32p, ctypes.c_int,
                                     ctypes.c_int, i64p, f64p, ctypes.c_int]
        L.hko_seg_stats.restype = None
        L.hko_seg_stats.argtypes = [f32p, ctypes.c_int, ctypes.c_int, f64p, f64p]
        L.hko_seg_stats_rows.restype = None
        L.hko_seg_stats_rows.argtypes = [f32p, i64p, ctypes.c_int64, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_int, f64p, f64p]
        L.hko_lb_eapca.restype = ctypes.c_double
        L.hko_lb_eapca.argtypes = [f32p, ctypes.c_int, i32p, f64p]
        L.hko_paa.restype = None
        L.hko_paa.argtypes = [f32p, ctypes.c_int, ctypes.c_int, f64p]
        L.hko_isax_bp.restype = None
        L.hko_isax_bp.argtypes = [f64p]
        L.hko_isax_symbol.restype = ctypes.c_int
        L.hko_isax_symbol.argtypes = [ctypes.c_double, f32p]
        L.hko_lb_sax.restype = ctypes.c_double
        L.hko_lb_sax.argtypes = [f64p, u8p, ctypes.c_int, ctypes.c_int, f32p]
        L.hko_dtw2.restype = ctypes.c_double
        L.hko_dtw2.argtypes = [f32p, f32p, ctypes.c_int, ctypes.c_int]
        L.hko_dtw_knn_update.restype = ctypes.c_int
        L.hko_dtw_knn_update.argtypes = [f32p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, f32p,
                                         ctypes.c_int, ctypes.c_int, ctypes.c_int, i64p, f64p,
                                         ctypes.c_int]
        L.hko_envelope.restype = None
        L.hko_envelope.argtypes = [f32p, ctypes.c_int, ctypes.c_int, f32p, f32p]
        L.hko_lb_keogh.restype = ctypes.c_double
        L.hko_lb_keogh.argtypes = [f32p, f32p, ctypes.c_int, ctypes.c_int]
        L.hko_lb_keogh_eapca.restype = ctypes.c_double
        L.hko_lb_keogh_eapca.argtypes = [f32p, ctypes.c_int, ctypes.c_int, ctypes.c_int, i32p, f64p]
        L.hko_lb_keogh_sax.restype = ctypes.c_double
        L.hko_lb_keogh_sax.argtypes = [f32p, ctypes.c_int, ctypes.c_int, u8p, f32p]
        _LIB = L
    return _LIB


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)))


def dist2(q, x) -> float:
    """Squared Euclidean distance, binary64, summed in index order."""
    q = _f32(q)
    x = _f32(x)
    assert q.shape == x.shape and q.ndim == 1
    return _lib().hko_dist2(_p(q, ctypes.c_float), _p(x, ctypes.c_float), q.size)


class KnnStream:
    """Brute-force k-NN over a collection fed in consecutive blocks.

    Every series is offered, in id order, to each query's running list of the
    k smallest (D, id) pairs (Sec. 2).  Feeding the collection in blocks gives
    the same lists as feeding it whole.
    """

    def __init__(self, Q, k: int, nthreads: int | None = None):
        self.Q = _f32(Q)
        assert self.Q.ndim == 2
        self.nq, self.n = self.Q.shape
        self.k = int(k)
        self.nthreads = nthreads or default_threads()
        self.ids = np.empty((self.nq, self.k), dtype=np.int64)
        self.d2 = np.empty((self.nq, self.k), dtype=np.float64)
        _lib().hko_knn_init(self.nq, self.k, _p(self.ids, ctypes.c_int64),
                            _p(self.d2, ctypes.c_double))
        self.next_id = 0

    def update(self, Xblock, id0: int | None = None):
        X = _f32(Xblock)
        assert X.ndim == 2 and X.shape[1] == self.n
        if id0 is None:
            id0 = self.next_id
        rc = _lib().hko_knn_update(_p(X, ctypes.c_float), int(id0), X.shape[0],
                                   self.n, _p(self.Q, ctypes.c_float), self.nq,
                                   self.k, _p(self.ids, ctypes.c_int64),
                                   _p(self.d2, ctypes.c_double), self.nthreads)
        if rc != 0:
            raise RuntimeError("hko_knn_update failed: %d" % rc)
        self.next_id = int(id0) + X.shape[0]

    def result(self):
        """(ids [nq,k] int64, squared distances [nq,k] float64)."""
        return self.ids.copy(), self.d2.copy()


def knn(X, Q, k: int, nthreads: int | None = None):
    """Exact k-NN by brute force: (ids, squared distances), ascending (D, id)."""
    s = KnnStream(Q, k, nthreads)
    s.update(X, 0)
    return s.result()


def seg_stats(x, a: int, b: int):
    """(mean, population std) of x[a:b] in binary64, two passes (Sec. 3.2)."""
    x = _f32(x)
    mu = ctypes.c_double()
    sd = ctypes.c_double()
    _lib().hko_seg_stats(_p(x, ctypes.c_float), a, b, ctypes.byref(mu),
                         ctypes.byref(sd))
    return mu.value, sd.value


def seg_stats_rows(X, rows, a: int, b: int):
    """seg_stats of X[rows[i], a:b] for every i: (mu[], sd[])."""
    X = _f32(X)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    mu = np.empty(rows.size, dtype=np.float64)
    sd = np.empty(rows.size, dtype=np.float64)
    _lib().hko_seg_stats_rows(_p(X, ctypes.c_float), _p(rows, ctypes.c_int64),
                              rows.size, X.shape[1], a, b,
                              _p(mu, ctypes.c_double), _p(sd, ctypes.c_double))
    return mu, sd


def lb_eapca(q, seg_end, env) -> float:
    """Squared LB_EAPCA of query q to a synopsis env[m][4] =
    (mu_min, mu_max, sd_min, sd_max) over segmentation seg_end (Sec. 2)."""
    q = _f32(q)
    se = np.ascontiguousarray(seg_end, dtype=np.int32)
    env = np.ascontiguousarray(env, dtype=np.float64).reshape(-1)
    assert env.size == 4 * se.size and se[-1] == q.size
    return _lib().hko_lb_eapca(_p(q, ctypes.c_float), se.size,
                               _p(se, ctypes.c_int32), _p(env, ctypes.c_double))


def paa(x, w: int = W_PAA):
    """PAA: means of w equal segments, binary64 (Sec. 2)."""
    x = _f32(x)
    assert x.size % w == 0
    out = np.empty(w, dtype=np.float64)
    _lib().hko_paa(_p(x, ctypes.c_float), x.size, w, _p(out, ctypes.c_double))
    return out


def isax_breakpoints():
    """beta_1..beta_255 with Phi(beta_j) = j/256, binary64 (Sec. 2)."""
    out = np.empty(ALPHABET - 1, dtype=np.float64)
    _lib().hko_isax_bp(_p(out, ctypes.c_double))
    return out


def isax_breakpoints_f32():
    """The breakpoint table as float32, the form both encode and LB_SAX use."""
    return isax_breakpoints().astype(np.float32)


def isax_symbol(v: float, bp32) -> int:
    bp32 = _f32(bp32)
    return _lib().hko_isax_symbol(float(v), _p(bp32, ctypes.c_float))


def isax_word(x, bp32, w: int = W_PAA):
    """iSAX word (w uint8 symbols) of series x (Sec. 2)."""
    p = paa(x, w)
    return np.array([isax_symbol(v, bp32) for v in p], dtype=np.uint8)


def lb_sax(paa_q, sym, n: int, bp32) -> float:
    """Squared LB_SAX of a query PAA to an iSAX word (Sec. 3.4)."""
    pq = np.ascontiguousarray(paa_q, dtype=np.float64)
    sym = np.ascontiguousarray(sym, dtype=np.uint8)
    bp32 = _f32(bp32)
    return _lib().hko_lb_sax(_p(pq, ctypes.c_double), _p(sym, ctypes.c_uint8),
                             sym.size, n, _p(bp32, ctypes.c_float))


def exact_answer(X, Q, k: int, nthreads: int | None = None):
    """The answer the query path must return: ids ascending by (D, id) and
    the reported Euclidean distances sqrt(D) rounded to float32."""
    ids, d2 = knn(X, Q, k, nthreads)
    return ids, np.sqrt(d2).astype(np.float32), d2


# ---- DTW with a Sakoe-Chiba band (Sec. 2: any distance with a lower bound)

def dtw2(q, x, band: int) -> float:
    """DTW with squared point costs and a Sakoe-Chiba band of half-width
    `band`, binary64 (the dynamic programme in hk_oracle.c)."""
    q = _f32(q)
    x = _f32(x)
    assert q.shape == x.shape and q.ndim == 1 and band >= 0
    return _lib().hko_dtw2(_p(q, ctypes.c_float), _p(x, ctypes.c_float), q.size, int(band))


class DtwKnnStream(KnnStream):
    """Brute-force k-NN under DTW(band), fed block by block like KnnStream."""

    def __init__(self, Q, k: int, band: int, nthreads: int | None = None):
        super().__init__(Q, k, nthreads)
        self.band = int(band)

    def update(self, Xblock, id0: int | None = None):
        X = _f32(Xblock)
        assert X.ndim == 2 and X.shape[1] == self.n
        if id0 is None:
            id0 = self.next_id
        rc = _lib().hko_dtw_knn_update(_p(X, ctypes.c_float), int(id0), X.shape[0], self.n,
                                       _p(self.Q, ctypes.c_float), self.nq, self.k, self.band,
                                       _p(self.ids, ctypes.c_int64), _p(self.d2, ctypes.c_double),
                                       self.nthreads)
        if rc != 0:
            raise RuntimeError("hko_dtw_knn_update failed: %d" % rc)
        self.next_id = int(id0) + X.shape[0]


def dtw_knn(X, Q, k: int, band: int, nthreads: int | None = None):
    """Exact k-NN under DTW(band): (ids, squared DTW values), ascending (D, id)."""
    s = DtwKnnStream(Q, k, band, nthreads)
    s.update(X, 0)
    return s.result()


def envelope(q, band: int):
    """(L, U): min and max of q over each window j-band .. j+band."""
    q = _f32(q)
    L = np.empty_like(q)
    U = np.empty_like(q)
    _lib().hko_envelope(_p(q, ctypes.c_float), q.size, int(band), _p(L, ctypes.c_float),
                        _p(U, ctypes.c_float))
    return L, U


def lb_keogh(q, x, band: int) -> float:
    """LB_Keogh^2(q, x) for DTW(band)."""
    q = _f32(q)
    x = _f32(x)
    return _lib().hko_lb_keogh(_p(q, ctypes.c_float), _p(x, ctypes.c_float), q.size, int(band))


def lb_keogh_eapca(q, band: int, seg_end, env) -> float:
    """LB_Keogh of q against a node synopsis env[m][4] over seg_end."""
    q = _f32(q)
    se = np.ascontiguousarray(seg_end, dtype=np.int32)
    env = np.ascontiguousarray(env, dtype=np.float64).reshape(-1)
    return _lib().hko_lb_keogh_eapca(_p(q, ctypes.c_float), q.size, int(band), se.size,
                                     _p(se, ctypes.c_int32), _p(env, ctypes.c_double))


def lb_keogh_sax(q, band: int, sym, bp32) -> float:
    """LB_Keogh of q against an iSAX word (16 symbols)."""
    q = _f32(q)
    sym = np.ascontiguousarray(sym, dtype=np.uint8)
    bp32 = _f32(bp32)
    return _lib().hko_lb_keogh_sax(_p(q, ctypes.c_float), q.size, int(band), _p(sym, ctypes.c_uint8),
                                   _p(bp32, ctypes.c_float))
