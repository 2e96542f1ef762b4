"""Index persistence (hk_save / hk_load).  Files that are not index files, or
are damaged, are rejected before any device memory is touched, so those
checks run without a GPU; the round trip runs on the GPU."""
import os

import numpy as np
import pytest


@pytest.fixture(scope="module")
def hb():
    from paper_2212_13297_gb300 import build, binding
    build.build()
    binding.lib()
    return binding


def test_load_rejects_missing_and_foreign_files(hb, tmp_path):
    with pytest.raises(hb.HerculesError) as e:
        hb.Index.load(tmp_path / "nope.hkidx")
    assert e.value.code == hb.HK_EIO
    bad = tmp_path / "foreign.hkidx"
    bad.write_bytes(b"PK\x03\x04 not an index" + bytes(200))
    with pytest.raises(hb.HerculesError) as e:
        hb.Index.load(bad)
    assert e.value.code == hb.HK_EINVAL
    # the right tag but a header that describes no valid index
    hdr = tmp_path / "header.hkidx"
    hdr.write_bytes(b"HKIDX002" + np.array([0, 7, 0, 0, 0, 0, 0, 0, 0, 0, 9], np.int64).tobytes()
                    + np.float64(0).tobytes() + np.int64(1).tobytes())
    with pytest.raises(hb.HerculesError) as e:
        hb.Index.load(hdr)
    assert e.value.code == hb.HK_EINVAL


@pytest.mark.gpu
@pytest.mark.parametrize("flags", [0, "fp16"])
def test_save_load_round_trip(hb, oracle_lib, tmp_path, flags):
    torch = pytest.importorskip("torch")
    import oracle
    from paper_2212_13297_gb300 import workload as wl
    X = wl.random_walk(30_000, 128, seed=61, device="cuda")
    f = hb.HK_BUILD_FP16 if flags == "fp16" else 0
    idx = hb.Index(X, 300, flags=f)
    path = tmp_path / "idx.hkidx"
    idx.save(path)
    idx2 = hb.Index.load(path)
    a, b = idx.info(), idx2.info()
    for key in ("N", "n", "leaves", "max_segments", "depth", "distinct_segments", "has_bf16", "device_bytes"):
        assert a[key] == b[key], key
    ea, eb = idx.export(), idx2.export()
    for key in ea:
        np.testing.assert_array_equal(ea[key], eb[key])
    Q, _ = wl.queries(X, 24, [0.1, 0.5, 1.0], seed=62)
    qf = hb.HK_Q_BF16 if flags == "fp16" else 0
    ids1, d1, _ = idx.query(Q, 10, flags=qf)
    ids2, d2, _ = idx2.query(Q, 10, flags=qf)
    np.testing.assert_array_equal(ids1.cpu().numpy(), ids2.cpu().numpy())
    np.testing.assert_array_equal(d1.cpu().numpy(), d2.cpu().numpy())
    oids, _ = oracle.knn(X.cpu().numpy(), Q.cpu().numpy(), 10)
    np.testing.assert_array_equal(ids2.cpu().numpy(), oids)
    # a damaged copy (one flipped byte in the raw series) fails its checksum
    raw = bytearray(path.read_bytes())
    raw[200] ^= 0x40
    bad = tmp_path / "flipped.hkidx"
    bad.write_bytes(bytes(raw))
    with pytest.raises(hb.HerculesError) as e:
        hb.Index.load(bad)
    assert e.value.code == hb.HK_EINVAL
    # a truncated copy
    short = tmp_path / "short.hkidx"
    short.write_bytes(bytes(raw[: len(raw) // 2]))
    with pytest.raises(hb.HerculesError) as e:
        hb.Index.load(short)
    assert e.value.code == hb.HK_EINVAL
