"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/hercules_gb300.h declares; host-only entry points and argument
checks work without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hercules_gb300.h")


@pytest.fixture(scope="session")
def hk():
    from paper_2212_13297_gb300 import build, binding
    build.build()
    return binding


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hk_[a-z0-9_]+)\s*\(", text)))


def test_exports_every_declared_symbol(hk):
    L = hk.lib()
    names = declared_symbols()
    assert len(names) >= 10
    for name in names:
        assert hasattr(L, name), name
    assert sorted(hk.EXPORTS) == names


def test_version_and_breakpoints_match_oracle(hk, oracle_lib):
    assert b"sm_103a" in hk.lib().hk_version()
    bp = hk.isax_breakpoints()
    import oracle
    np.testing.assert_array_equal(bp, oracle.isax_breakpoints_f32())


def test_argument_checks_without_gpu(hk):
    L = hk.lib()
    h = ctypes.c_void_p()
    X = np.zeros((4, 16), np.float32)
    o = hk.hk_build_opts(10, 0, 0, 0)
    for N, n in [(4, 15), (4, 8), (4, 4100), (0, 16), (-1, 16)]:
        rc = L.hk_build(X.ctypes.data_as(ctypes.c_void_p), N, n, ctypes.byref(o), None,
                        ctypes.byref(h))
        assert rc == hk.HK_EINVAL
        assert L.hk_last_error()
    bad = hk.hk_build_opts(0, 0, 0, 0)
    rc = L.hk_build(X.ctypes.data_as(ctypes.c_void_p), 4, 16, ctypes.byref(bad), None,
                    ctypes.byref(h))
    assert rc == hk.HK_EINVAL and b"leaf_capacity" in L.hk_last_error()
    assert L.hk_build(None, 4, 16, ctypes.byref(o), None, ctypes.byref(h)) == hk.HK_EINVAL
    ids = np.zeros(4, np.int64)
    d = np.zeros(4, np.float32)
    assert L.hk_query(None, X.ctypes.data_as(ctypes.c_void_p), 1, 1, None, None,
                      ids.ctypes.data_as(ctypes.c_void_p), d.ctypes.data_as(ctypes.c_void_p),
                      None) == hk.HK_EINVAL
    assert L.hk_scan_knn(X.ctypes.data_as(ctypes.c_void_p), 4, 16,
                         X.ctypes.data_as(ctypes.c_void_p), 1, 5, None,
                         ids.ctypes.data_as(ctypes.c_void_p),
                         d.ctypes.data_as(ctypes.c_void_p)) == hk.HK_EINVAL   # k > N
    assert L.hk_free(None) == hk.HK_OK


def test_binding_structs_match_header(hk):
    text = open(HEADER).read()

    def fields(struct_name):
        body = text[:text.index("} %s;" % struct_name)]
        body = body[body.rindex("typedef struct {"):]
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        return re.findall(r"\b(?:u?int\d+_t|float|double|hk_\w+)\s+(\w+)(?:\[\d+\])?;", body)

    for cname, pyc in [("hk_build_opts", hk.hk_build_opts), ("hk_query_opts", hk.hk_query_opts),
                       ("hk_query_stats", hk.hk_query_stats), ("hk_index_info", hk.hk_index_info),
                       ("hk_tune_result", hk.hk_tune_result), ("hk_server_opts", hk.hk_server_opts),
                       ("hk_server_stats", hk.hk_server_stats)]:
        assert [f[0] for f in pyc._fields_] == fields(cname), cname
        assert ctypes.sizeof(pyc) >= 4 * len(pyc._fields_), cname
