"""ctypes binding of the C ABI in include/hercules_gb300.h.

Argument marshalling only: every step of index building and query answering
runs in the CUDA library.  There is no CPU fallback; if the library has not
been built, loading it raises.

Raw entry points keep their C names (hk_build, hk_query, ...).  `Index` and
`scan_knn` wrap them for torch tensors and numpy arrays.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libhercules_gb300.so")

HK_OK = 0
HK_EINVAL = -1
HK_ENOMEM = -2
HK_ECUDA = -3
HK_ETIMEOUT = -4
HK_EBUSY = -5
HK_EINTERNAL = -6
HK_EIO = -7

HK_BUILD_ADOPT = 1
HK_BUILD_BF16 = 2
HK_BUILD_FP16 = 4
HK_Q_NOSAX = 1
HK_Q_NOTHRESH = 2
HK_Q_NOPRUNE = 4
HK_Q_TIMING = 8
HK_Q_BF16 = 16
HK_Q_GRAPH = 32
HK_Q_TREE = 64


class hk_build_opts(ctypes.Structure):
    _fields_ = [("leaf_capacity", ctypes.c_int32), ("eval_cap", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("reserved", ctypes.c_int32)]


class hk_query_opts(ctypes.Structure):
    _fields_ = [("l_max", ctypes.c_int32), ("eapca_th", ctypes.c_float),
                ("sax_th", ctypes.c_float), ("flags", ctypes.c_uint32),
                ("query_group", ctypes.c_int32), ("series_tile", ctypes.c_int32)]


class hk_query_stats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in (
        "queries", "leaves_total", "leaves_approx", "leaves_candidate", "series_candidate",
        "series_sax_pruned", "series_abandoned", "series_full", "points_computed", "rescored",
        "fallback_queries", "retried_queries", "work_items", "skip_sequential", "scan_ns", "kernel_launches",
        "scan_bytes", "tc_pairs", "tc_candidates", "tc_ns", "tc_bytes", "tc_approx_pairs",
        "tc_approx_ns", "tc_approx_bytes", "tc_leaf_bytes", "lb_evaluations")]

    def as_dict(self):
        return {f[0]: getattr(self, f[0]) for f in self._fields_}


class hk_index_info(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("n", ctypes.c_int32), ("leaf_capacity", ctypes.c_int32),
                ("leaves", ctypes.c_int64), ("max_segments", ctypes.c_int32),
                ("depth", ctypes.c_int32), ("distinct_segments", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("has_bf16", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class hk_tune_result(ctypes.Structure):
    _fields_ = [("opts", hk_query_opts), ("ms_per_query", ctypes.c_double), ("tried", ctypes.c_int32),
                ("tensor_cores", ctypes.c_int32)]


class hk_server_opts(ctypes.Structure):
    _fields_ = [("max_batch", ctypes.c_int32), ("max_wait_us", ctypes.c_int32),
                ("hbm_budget", ctypes.c_int64), ("query_flags", ctypes.c_uint32),
                ("workers", ctypes.c_int32), ("persistent", ctypes.c_int32)]


class hk_server_stats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in (
        "batches", "served", "max_batch", "errors", "pending", "busy_ns", "budget_peak",
        "scan_launches", "scan_jobs", "scan_jobs_inflight", "scan_max_collections")]


class HerculesError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("hercules error %d: %s" % (code, msg))
        self.code = code


_lib = None

# every symbol include/hercules_gb300.h declares
EXPORTS = ["hk_build", "hk_free", "hk_index_info_get", "hk_query", "hk_query_dtw", "hk_scan_knn",
           "hk_scan_knn_noalloc",
           "hk_isax_breakpoints", "hk_index_export", "hk_index_export_tree", "hk_debug_lb_eapca",
           "hk_debug_lb_sax",
           "hk_debug_tc_dist", "hk_server_create", "hk_server_add", "hk_server_add_opts", "hk_submit", "hk_poll",
           "hk_server_stats_get", "hk_server_destroy", "hk_tune", "hk_save", "hk_load",
           "hk_query_opts_default", "hk_debug_device_allocs", "hk_debug_fail_device_alloc",
           "hk_debug_tc_wait", "hk_last_error", "hk_version"]


def lib():
    """The loaded library (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("CUDA library not built: %s missing (run "
                               "__graft_entry__.build())" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        vp = ctypes.c_void_p
        i64p = ctypes.POINTER(ctypes.c_int64)
        L.hk_build.argtypes = [vp, ctypes.c_int64, ctypes.c_int32,
                               ctypes.POINTER(hk_build_opts), vp, ctypes.POINTER(vp)]
        L.hk_free.argtypes = [vp]
        L.hk_index_info_get.argtypes = [vp, ctypes.POINTER(hk_index_info)]
        L.hk_query.argtypes = [vp, vp, ctypes.c_int32, ctypes.c_int32,
                               ctypes.POINTER(hk_query_opts), vp, vp, vp,
                               ctypes.POINTER(hk_query_stats)]
        L.hk_query_dtw.argtypes = [vp, vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                   ctypes.POINTER(hk_query_opts), vp, vp, vp, ctypes.POINTER(hk_query_stats)]
        L.hk_scan_knn.argtypes = [vp, ctypes.c_int64, ctypes.c_int32, vp, ctypes.c_int32,
                                  ctypes.c_int32, vp, vp, vp]
        L.hk_scan_knn_noalloc.argtypes = [vp, ctypes.c_int64, ctypes.c_int32, vp, ctypes.c_int32,
                                          ctypes.c_int32, vp, vp, vp]
        L.hk_isax_breakpoints.argtypes = [vp]
        L.hk_index_export.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.hk_index_export_tree.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.hk_debug_lb_eapca.argtypes = [vp, vp, ctypes.c_int32, vp]
        L.hk_debug_lb_sax.argtypes = [vp, vp, ctypes.c_int32, vp]
        L.hk_debug_tc_dist.argtypes = [vp, vp, ctypes.c_int32, vp, vp]
        L.hk_server_create.argtypes = [ctypes.POINTER(hk_server_opts), ctypes.POINTER(vp)]
        L.hk_server_add.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_int32)]
        L.hk_server_add_opts.argtypes = [vp, vp, ctypes.POINTER(hk_query_opts), ctypes.POINTER(ctypes.c_int32)]
        L.hk_submit.argtypes = [vp, ctypes.c_int32, vp, ctypes.c_int32,
                                ctypes.POINTER(ctypes.c_uint64)]
        L.hk_poll.argtypes = [vp, ctypes.c_uint64, vp, vp, ctypes.c_int32,
                              ctypes.POINTER(ctypes.c_int64)]
        L.hk_server_stats_get.argtypes = [vp, ctypes.POINTER(hk_server_stats)]
        L.hk_server_destroy.argtypes = [vp]
        L.hk_tune.argtypes = [vp, vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint32, vp,
                              ctypes.POINTER(hk_tune_result)]
        L.hk_save.argtypes = [vp, ctypes.c_char_p]
        L.hk_load.argtypes = [ctypes.c_char_p, vp, ctypes.POINTER(vp)]
        L.hk_query_opts_default.argtypes = [ctypes.POINTER(hk_query_opts)]
        L.hk_debug_device_allocs.argtypes = [i64p]
        L.hk_debug_fail_device_alloc.argtypes = [ctypes.c_int64]
        L.hk_debug_tc_wait.argtypes = [ctypes.c_uint64, ctypes.c_int32]
        L.hk_last_error.restype = ctypes.c_char_p
        L.hk_version.restype = ctypes.c_char_p
        for name in EXPORTS:
            if name not in ("hk_last_error", "hk_version"):
                getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(rc):
    if rc != HK_OK:
        raise HerculesError(rc, lib().hk_last_error().decode())


def _ptr(a):
    """Address of a torch tensor or numpy array (contiguous)."""
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous()
        return ctypes.c_void_p(a.data_ptr())
    assert a.flags["C_CONTIGUOUS"]
    return ctypes.c_void_p(a.ctypes.data)


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    try:
        import torch
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return ctypes.c_void_p(0)


def query_opts_default():
    """The options a NULL hk_query_opts stands for, as a dict."""
    o = hk_query_opts()
    _check(lib().hk_query_opts_default(ctypes.byref(o)))
    return {f[0]: getattr(o, f[0]) for f in o._fields_}


def device_allocs():
    """Device allocations the library has made in this process so far."""
    c = ctypes.c_int64()
    _check(lib().hk_debug_device_allocs(ctypes.byref(c)))
    return c.value


def isax_breakpoints():
    out = np.empty(255, np.float32)
    _check(lib().hk_isax_breakpoints(_ptr(out)))
    return out


def _is_cuda(t):
    return hasattr(t, "is_cuda") and t.is_cuda


def _out_like(like, shape, np_dtype, torch_dtype):
    if _is_cuda(like):
        import torch
        return torch.empty(shape, dtype=torch_dtype, device=like.device)
    return np.empty(shape, np_dtype)


class Index:
    """A Hercules index resident on the current GPU (owns its device memory)."""

    def __init__(self, X, leaf_capacity: int, eval_cap: int = 0, flags: int = 0, stream=None):
        N, n = X.shape
        o = hk_build_opts(int(leaf_capacity), int(eval_cap), int(flags), 0)
        h = ctypes.c_void_p()
        _check(lib().hk_build(_ptr(X), N, n, ctypes.byref(o), _stream(stream), ctypes.byref(h)))
        self._h = h
        self.N, self.n = N, n

    def close(self):
        if getattr(self, "_h", None):
            lib().hk_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def save(self, path):
        """hk_save: write the index to a file."""
        _check(lib().hk_save(self._h, os.fsencode(path)))

    @classmethod
    def load(cls, path, stream=None):
        """hk_load: an index read from a file written by save()."""
        h = ctypes.c_void_p()
        _check(lib().hk_load(os.fsencode(path), _stream(stream), ctypes.byref(h)))
        self = cls.__new__(cls)
        self._h = h
        i = self.info()
        self.N, self.n = i["N"], i["n"]
        return self

    def info(self):
        i = hk_index_info()
        _check(lib().hk_index_info_get(self._h, ctypes.byref(i)))
        return {f[0]: getattr(i, f[0]) for f in i._fields_ if f[0] != "reserved"}

    def query(self, Q, k: int, l_max=0, eapca_th=-1.0, sax_th=-1.0, flags=0, query_group=0,
              series_tile=0, stream=None, out=None):
        """(ids [nq,k] int64, dist [nq,k] float32, stats dict).  Outputs live
        where Q lives (device tensors for a CUDA Q, numpy otherwise) unless
        out=(ids, dist) is given."""
        nq = Q.shape[0]
        assert Q.shape[1] == self.n
        if out is None:
            ids = _out_like(Q, (nq, k), np.int64, _torch_dtype("int64"))
            dist = _out_like(Q, (nq, k), np.float32, _torch_dtype("float32"))
        else:
            ids, dist = out
        o = hk_query_opts(int(l_max), float(eapca_th), float(sax_th), int(flags),
                          int(query_group), int(series_tile))
        st = hk_query_stats()
        _check(lib().hk_query(self._h, _ptr(Q), nq, int(k), ctypes.byref(o), _stream(stream),
                              _ptr(ids), _ptr(dist), ctypes.byref(st)))
        return ids, dist, st.as_dict()

    def query_dtw(self, Q, k: int, band: int, l_max=0, flags=0, stream=None, out=None):
        """Exact k-NN under DTW with a Sakoe-Chiba band: (ids, dist, stats)
        as query()."""
        nq = Q.shape[0]
        assert Q.shape[1] == self.n
        if out is None:
            ids = _out_like(Q, (nq, k), np.int64, _torch_dtype("int64"))
            dist = _out_like(Q, (nq, k), np.float32, _torch_dtype("float32"))
        else:
            ids, dist = out
        o = hk_query_opts(int(l_max), -1.0, -1.0, int(flags), 0, 0)
        st = hk_query_stats()
        _check(lib().hk_query_dtw(self._h, _ptr(Q), nq, int(k), int(band), ctypes.byref(o), _stream(stream),
                                  _ptr(ids), _ptr(dist), ctypes.byref(st)))
        return ids, dist, st.as_dict()

    def tune(self, Q, k: int, keep_flags=0, stream=None):
        """hk_tune: the fastest query configuration on the sample batch Q, as a
        dict of hk_query keyword arguments plus ms_per_query / tried /
        tensor_cores."""
        r = hk_tune_result()
        _check(lib().hk_tune(self._h, _ptr(Q), Q.shape[0], int(k), int(keep_flags), _stream(stream),
                             ctypes.byref(r)))
        o = r.opts
        return dict(l_max=o.l_max, eapca_th=o.eapca_th, sax_th=o.sax_th, flags=o.flags,
                    query_group=o.query_group, series_tile=o.series_tile,
                    ms_per_query=r.ms_per_query, tried=r.tried, tensor_cores=r.tensor_cores)

    def export(self):
        """Leaf layout as numpy arrays (see hk_index_export)."""
        info = self.info()
        L = info["leaves"]
        perm = np.empty(self.N, np.int64)
        leaf_off = np.empty(L + 1, np.int64)
        nseg = np.empty(L, np.int32)
        seg_end = np.empty((L, 64), np.int32)
        env = np.empty((L, 64, 4), np.float64)
        sax = np.empty((self.N, 16), np.uint8)
        _check(lib().hk_index_export(self._h, _ptr(perm), _ptr(leaf_off), _ptr(nseg),
                                     _ptr(seg_end), _ptr(env), _ptr(sax)))
        return dict(perm=perm, leaf_off=leaf_off, nseg=nseg, seg_end=seg_end, env=env, sax=sax)

    def export_tree(self):
        """The whole tree as numpy arrays (see hk_index_export_tree)."""
        T = 2 * self.info()["leaves"] - 1
        out = dict(parent=np.empty(T, np.int32), left=np.empty(T, np.int32), right=np.empty(T, np.int32),
                   beg=np.empty(T, np.int64), end=np.empty(T, np.int64), nseg=np.empty(T, np.int32),
                   seg_end=np.empty((T, 64), np.int32), env=np.empty((T, 64, 4), np.float64))
        _check(lib().hk_index_export_tree(self._h, *[_ptr(out[k]) for k in
                                                     ("parent", "left", "right", "beg", "end", "nseg",
                                                      "seg_end", "env")]))
        return out

    def debug_lb_eapca(self, Q):
        L = self.info()["leaves"]
        out = np.empty((Q.shape[0], L), np.float64)
        _check(lib().hk_debug_lb_eapca(self._h, _ptr(Q), Q.shape[0], _ptr(out)))
        return out

    def debug_tc_dist(self, Q):
        """Certified interval (lo [nq, N], up [nq, N]) of the tensor-core
        form around every squared distance, leaf order."""
        lo = np.empty((Q.shape[0], self.N), np.float32)
        up = np.empty((Q.shape[0], self.N), np.float32)
        _check(lib().hk_debug_tc_dist(self._h, _ptr(Q), Q.shape[0], _ptr(lo), _ptr(up)))
        return lo, up

    def debug_lb_sax(self, Q):
        out = np.empty((Q.shape[0], self.N), np.float32)
        _check(lib().hk_debug_lb_sax(self._h, _ptr(Q), Q.shape[0], _ptr(out)))
        return out


def _torch_dtype(name):
    import torch
    return getattr(torch, name)


def scan_knn(X, Q, k: int, stream=None):
    """Exhaustive exact k-NN (the parallel-scan baseline), no index."""
    N, n = X.shape
    nq = Q.shape[0]
    ids = _out_like(Q, (nq, k), np.int64, _torch_dtype("int64"))
    dist = _out_like(Q, (nq, k), np.float32, _torch_dtype("float32"))
    _check(lib().hk_scan_knn(_ptr(X), N, n, _ptr(Q), nq, int(k), _stream(stream), _ptr(ids),
                             _ptr(dist)))
    return ids, dist


class Server:
    """Continuous-batching server over registered indexes (hk_server_*)."""

    def __init__(self, max_batch=0, max_wait_us=0, hbm_budget=0, query_flags=0, workers=0, persistent=0):
        o = hk_server_opts(int(max_batch), int(max_wait_us), int(hbm_budget), int(query_flags),
                           int(workers), int(persistent))
        h = ctypes.c_void_p()
        _check(lib().hk_server_create(ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        self._n = {}

    def add(self, index, opts=None):
        """Register an index; opts (hk_query keyword arguments, e.g. the
        dict Index.tune returns) become that collection's query configuration
        (hk_server_add_opts)."""
        if opts is not None:
            o = hk_query_opts(int(opts.get("l_max", 0)), float(opts.get("eapca_th", -1.0)),
                              float(opts.get("sax_th", -1.0)), int(opts.get("flags", 0)),
                              int(opts.get("query_group", 0)), int(opts.get("series_tile", 0)))
            c = ctypes.c_int32()
            _check(lib().hk_server_add_opts(self._h, index._h, ctypes.byref(o), ctypes.byref(c)))
            self._n[c.value] = index.n
            return c.value
        c = ctypes.c_int32()
        _check(lib().hk_server_add(self._h, index._h, ctypes.byref(c)))
        self._n[c.value] = index.n
        return c.value

    def submit(self, coll, q, k):
        q = np.ascontiguousarray(q, dtype=np.float32)
        t = ctypes.c_uint64()
        _check(lib().hk_submit(self._h, int(coll), _ptr(q), int(k), ctypes.byref(t)))
        return t.value

    def poll(self, ticket, k, timeout_us=1_000_000):
        """(ids, dist, latency_ns), or None if not done within the timeout."""
        ids = np.empty(k, np.int64)
        dist = np.empty(k, np.float32)
        lat = ctypes.c_int64()
        rc = lib().hk_poll(self._h, ctypes.c_uint64(ticket), _ptr(ids), _ptr(dist),
                           int(timeout_us), ctypes.byref(lat))
        if rc == HK_ETIMEOUT:
            return None
        _check(rc)
        return ids, dist, lat.value

    def stats(self):
        st = hk_server_stats()
        _check(lib().hk_server_stats_get(self._h, ctypes.byref(st)))
        return {f[0]: getattr(st, f[0]) for f in st._fields_}

    def close(self):
        if getattr(self, "_h", None):
            lib().hk_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
