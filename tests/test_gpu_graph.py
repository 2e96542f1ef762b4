"""Graph mode (HK_Q_GRAPH) and the configuration search (hk_tune): both must
leave every answer unchanged.  Graph replays are checked against ordinary
calls and the brute-force oracle, across batches of one shape, a change of
shape (a new capture) and an ordinary call in between."""
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
def setup(hb):
    from paper_2212_13297_gb300 import workload as wl
    X = wl.random_walk(60_000, 128, seed=31, device="cuda")
    idx = hb.Index(X, 500, flags=hb.HK_BUILD_FP16)
    batches = [wl.queries(X, 48, [0.1, 0.5, 1.0], seed=40 + i)[0] for i in range(4)]
    return X, idx, batches


@pytest.mark.parametrize("form", ["plain", "tc"])
def test_graph_replays_equal_ordinary_calls(hb, oracle_lib, setup, form):
    X, idx, batches = setup
    f = hb.HK_Q_BF16 if form == "tc" else 0
    k = 10
    for i, Q in enumerate(batches):
        ids_g, dist_g, st = idx.query(Q, k, flags=f | hb.HK_Q_GRAPH)
        ids_o, dist_o, _ = idx.query(Q, k, flags=f)
        np.testing.assert_array_equal(ids_g.cpu().numpy(), ids_o.cpu().numpy())
        np.testing.assert_array_equal(dist_g.cpu().numpy(), dist_o.cpu().numpy())
        assert st["kernel_launches"] > 0 and st["queries"] == Q.shape[0]
    oids, od2 = oracle.knn(X.cpu().numpy(), batches[-1].cpu().numpy(), k)
    np.testing.assert_array_equal(ids_g.cpu().numpy(), oids)
    np.testing.assert_allclose(dist_g.cpu().numpy(), np.sqrt(od2).astype(np.float32), rtol=1e-5)


def test_graph_shape_change_and_host_buffers(hb, setup):
    X, idx, batches = setup
    # another batch size and k: a new capture; then back to the first shape
    for Q, k in [(batches[0][:17].contiguous(), 3), (batches[1], 10), (batches[2][:17].contiguous(), 3)]:
        ids_g, dist_g, _ = idx.query(Q, k, flags=hb.HK_Q_GRAPH)
        ids_o, dist_o, _ = idx.query(Q, k)
        np.testing.assert_array_equal(ids_g.cpu().numpy(), ids_o.cpu().numpy())
        np.testing.assert_array_equal(dist_g.cpu().numpy(), dist_o.cpu().numpy())
    # host queries and host outputs through the graph path
    Qh = batches[3].cpu().numpy()
    ids_h, dist_h, _ = idx.query(Qh, 10, flags=hb.HK_Q_GRAPH)
    ids_h2, dist_h2, _ = idx.query(Qh, 10, flags=hb.HK_Q_GRAPH)
    ids_o, _, _ = idx.query(Qh, 10)
    np.testing.assert_array_equal(ids_h, ids_o)
    np.testing.assert_array_equal(ids_h2, ids_o)
    np.testing.assert_array_equal(dist_h, dist_h2)


def test_graph_duplicates_take_the_retry_path(hb, oracle_lib):
    """Near ties that overflow the lists still end exact when the pass comes
    from a graph (the retry runs after the replay)."""
    from paper_2212_13297_gb300 import workload as wl
    X = wl.random_walk(8000, 64, seed=5, device="cuda")
    X[1000:7000] = X[3]
    idx = hb.Index(X, 200)
    Q = torch.cat([X[[3]], X[[10]]]).contiguous()
    for _ in range(2):
        ids, dist, st = idx.query(Q, 10, flags=hb.HK_Q_GRAPH)
        oids, _ = oracle.knn(X.cpu().numpy(), Q.cpu().numpy(), 10)
        np.testing.assert_array_equal(ids.cpu().numpy(), oids)


def test_tune_picks_a_configuration_with_the_same_answers(hb, setup):
    X, idx, batches = setup
    Q = batches[0]
    r = idx.tune(Q, 10)
    assert r["tried"] >= 2 and r["ms_per_query"] > 0
    assert r["tensor_cores"] == (1 if r["flags"] & hb.HK_Q_BF16 else 0)
    kw = {key: r[key] for key in ("l_max", "eapca_th", "sax_th", "flags", "query_group", "series_tile")}
    ids_t, dist_t, _ = idx.query(batches[1], 10, **kw)
    ids_o, dist_o, _ = idx.query(batches[1], 10)
    np.testing.assert_array_equal(ids_t.cpu().numpy(), ids_o.cpu().numpy())
    np.testing.assert_array_equal(dist_t.cpu().numpy(), dist_o.cpu().numpy())
    # a plain index (no 16-bit copy) is tuned over the float32 form only
    plain = hb.Index(X, 500)
    r2 = plain.tune(Q, 5)
    assert r2["tensor_cores"] == 0 and r2["tried"] >= 1
    with pytest.raises(hb.HerculesError):
        idx.tune(Q, 10, keep_flags=hb.HK_Q_BF16)
