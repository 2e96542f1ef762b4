"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times (collection, batch, form, options): a sample of each batch's queries is
checked against the brute-force oracle, which streams the same seeded
collection block by block, so host memory never holds it whole.  Ids must be
identical, distances within 1e-5 relative."""
import gc

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


def _oracle_stream(N, n, seed, Qs, k):
    s = oracle.KnnStream(Qs, k)
    for a, rows in _wl().random_walk_chunks(N, n, seed=seed, device="cuda"):
        s.update(rows.cpu().numpy(), a)
    return s.ids.copy(), s.d2.copy()


# name: N, n, leaf capacity, batch, sigmas, ks, form, sampled rows of the batch
SIZES = {
    "large": (100_000_000, 256, 100_000, 1000, [0.5, 1.0], [10], "fp16", [0, 333, 666, 999]),
    "mid": (10_000_000, 256, 10_000, 100, [0.01, 0.1, 0.5, 1.0], [1, 10], "plain", [0, 13, 26, 39, 52, 65, 78, 99]),
    "precision": (10_000_000, 256, 10_000, 1024, "uniform", [100], "fp16", [0, 511, 1023]),
}


@pytest.mark.parametrize("name", ["mid", "precision", "large"])
def test_full_size_sample_matches_oracle(hb, oracle_lib, name):
    N, n, tau, B, sig, ks, form, sample = SIZES[name]
    wl = _wl()
    gc.collect()                 # indexes and tensors of earlier tests
    torch.cuda.empty_cache()
    free, total = torch.cuda.mem_get_info()
    need = N * n * 4 * 2.6 if form == "fp16" else N * n * 4 * 2.1
    if free < need:
        pytest.skip("needs %.0f GB of free device memory" % (need / 1e9))
    X = wl.random_walk(N, n, seed=0, device="cuda")
    if sig == "uniform":
        sig = wl.uniform_sigmas(B, 0.01, 1.0, seed=1)
    Q, _ = wl.queries(X, B, sig, seed=1)
    idx = hb.Index(X, tau, flags=hb.HK_BUILD_FP16 if form == "fp16" else 0)
    del X
    gc.collect()
    torch.cuda.empty_cache()
    flags = hb.HK_Q_BF16 if form == "fp16" else 0
    Qs = Q.cpu().numpy()[sample]
    for k in ks:
        ids, dist, st = idx.query(Q, k, flags=flags)
        assert st["queries"] == B
        oids, od2 = _oracle_stream(N, n, 0, Qs, k)
        np.testing.assert_array_equal(ids.cpu().numpy()[sample], oids)
        np.testing.assert_allclose(dist.cpu().numpy()[sample], np.sqrt(od2).astype(np.float32), rtol=1e-5)
    idx.close()
    del idx
    gc.collect()
    torch.cuda.empty_cache()
