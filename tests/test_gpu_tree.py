"""The tree's internal-node synopses (Sec. 3.3) and pruning with them.

  * Every node the GPU build makes (leaves and internal nodes) has the
    oracle's position range and segmentation, and its synopsis equals the
    oracle's: the min / max of the segment means and stds over every series
    that traversed the node, which the paper's ProcessLeaf / VSplitSynopsis /
    HSplitSynopsis fold arrives at (tests/test_oracle_tree.py pins the fold
    against that definition).
  * HK_Q_TREE (best-first approximate search over the tree, subtrees pruned
    by their roots' LB_EAPCA) gives the brute-force answers, on the float32
    path and the tensor-core form, and evaluates fewer LB_EAPCA than the flat
    pass on easy queries; after hk_save / hk_load it still does.
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


@pytest.mark.parametrize("N,n,tau", [(2500, 64, 60), (2000, 16, 30), (1800, 96, 40)])
def test_every_node_synopsis_matches_oracle(hb, oracle_lib, N, n, tau):
    X = _wl().random_walk(N, n, seed=N + n, device="cuda")
    Xh = X.cpu().numpy()
    idx = hb.Index(X, tau)
    ex = idx.export()
    tr = idx.export_tree()
    T = tr["parent"].size
    L = idx.info()["leaves"]
    assert T == 2 * L - 1
    root = otree.build_tree(Xh, tau)
    onodes = otree.nodes_preorder(root)
    assert len(onodes) == T
    # the GPU node covering the same positions with the same segmentation
    pos = np.empty(N, np.int64)
    pos[ex["perm"]] = np.arange(N)
    by_range = {}
    for u in range(T):
        key = (int(tr["beg"][u]), int(tr["end"][u]), tuple(tr["seg_end"][u, :tr["nseg"][u]]))
        by_range.setdefault(key, []).append(u)
    internal = 0
    for nd in onodes:
        members = otree.subtree_members(nd)
        p = np.sort(pos[members])
        assert p[-1] - p[0] + 1 == len(members), "a node's series are not contiguous in leaf order"
        key = (int(p[0]), int(p[-1]) + 1, tuple(nd.seg_end))
        assert key in by_range, key
        u = by_range[key][-1]          # a chain of one-child ranges cannot occur: take the deepest
        np.testing.assert_array_equal(tr["env"][u, :len(nd.seg_end)], otree.node_synopsis(Xh, nd))
        if not nd.is_leaf:
            internal += 1
            assert u >= L and tr["left"][u] >= 0 and tr["right"][u] >= 0
            assert tr["parent"][tr["left"][u]] == u and tr["parent"][tr["right"][u]] == u
    assert internal == L - 1


@pytest.mark.parametrize("N,n,tau,nq,k,sig,fmt", [
    (30000, 64, 50, 24, 1, [0.01, 0.1], None),
    (30000, 64, 50, 24, 10, [0.5, 1.0], None),
    (20000, 256, 40, 40, 10, [0.01, 0.5, 1.0], "fp16"),
    (12000, 128, 30, 30, 100, [0.1, 1.0], "fp16"),
    (6000, 96, 20, 9, 5, [0.2], None),
])
def test_tree_mode_matches_bruteforce(hb, oracle_lib, N, n, tau, nq, k, sig, fmt):
    wl = _wl()
    X = wl.random_walk(N, n, seed=N + 3 * n, device="cuda")
    Q, _ = wl.queries(X, nq, sig, seed=k + 7)
    idx = hb.Index(X, tau, flags=hb.HK_BUILD_FP16 if fmt else 0)
    oids, od2 = oracle.knn(X.cpu().numpy(), Q.cpu().numpy(), k)
    flat_flags = hb.HK_Q_BF16 if fmt else 0
    _, _, st_flat = idx.query(Q, k, flags=flat_flags)
    ids, dist, st = idx.query(Q, k, flags=flat_flags | hb.HK_Q_TREE)
    np.testing.assert_array_equal(ids.cpu().numpy(), oids)
    np.testing.assert_allclose(dist.cpu().numpy(), np.sqrt(od2).astype(np.float32), rtol=1e-5)
    L = idx.info()["leaves"]
    assert st_flat["lb_evaluations"] == nq * L
    assert 0 < st["lb_evaluations"]
    if max(sig) <= 0.1:
        assert st["lb_evaluations"] < st_flat["lb_evaluations"] // 2, (st["lb_evaluations"], nq * L)


def test_tree_survives_save_load(hb, oracle_lib, tmp_path):
    wl = _wl()
    X = wl.random_walk(15000, 64, seed=91, device="cuda")
    Q, _ = wl.queries(X, 12, [0.05, 0.7], seed=92)
    idx = hb.Index(X, 40)
    path = str(tmp_path / "tree.hkx")
    idx.save(path)
    back = hb.Index.load(path)
    a, b = idx.export_tree(), back.export_tree()
    for key in a:
        np.testing.assert_array_equal(a[key], b[key])
    ids, dist, _ = back.query(Q, 7, flags=hb.HK_Q_TREE)
    oids, od2 = oracle.knn(X.cpu().numpy(), Q.cpu().numpy(), 7)
    np.testing.assert_array_equal(ids.cpu().numpy(), oids)
