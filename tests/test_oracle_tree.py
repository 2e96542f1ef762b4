"""Pins for the oracle tree (Sec. 3.2 node structure and splits; Algorithm
InsertSeriesToNode, Sec. 3.3).

The split policy is a reading (the paper defers it to DSTree), so the tree's
shape is not pinned by the paper beyond its worked example; what is pinned:
the worked threshold, the half-open routing rule, the structural invariants
the paper states (every series in exactly one leaf, leaves within capacity,
synopses enclosing their series, children segmentation after H/V splits),
and the policy's arithmetic on hand-built nodes.
"""
import os

import numpy as np
import pytest

import oracle
from oracle import tree as otree

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "split_example.txt")


def _golden():
    vals = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.split()
        vals[k] = float(v)
    return vals


def _series_with_segment_means(means, n=16):
    """Rows whose first segment (of 4) has the given mean, rest 0."""
    X = np.zeros((len(means), n), np.float32)
    l = n // 4
    for i, m in enumerate(means):
        X[i, :l] = m
    return X


def test_worked_split_example(oracle_lib):
    g = _golden()
    X = _series_with_segment_means([g["mu_min"], -0.2, -0.1, -0.08, 0.0, 0.05, g["mu_max"]])
    # evaluate the H-split on the mean of segment 0 directly
    mu, _ = oracle.seg_stats_rows(X, np.arange(len(X)), 0, 4)
    thr = (float(mu.min()) + float(mu.max())) * 0.5
    assert thr == pytest.approx(g["threshold"], abs=1e-7)
    p = otree.Policy("H", 0, -1, 0, 0, 4, thr)
    right = p.side(X, np.arange(len(X)))
    assert list(right) == [False, False, False, False, True, True, True]
    # half-open: a series exactly on the threshold goes right.  0.10 is not a
    # float32, so use a range whose midpoint is: [-0.25, 0.125] -> -0.0625.
    X2 = _series_with_segment_means([-0.25, 0.125, -0.0625, -0.0625 - 2**-20])
    mu2, _ = oracle.seg_stats_rows(X2, np.arange(2), 0, 4)
    thr2 = (float(mu2.min()) + float(mu2.max())) * 0.5
    assert thr2 == -0.0625
    p2 = otree.Policy("H", 0, -1, 0, 0, 4, thr2)
    assert list(p2.side(X2, np.arange(4))) == [False, True, True, False]


def test_policy_picks_the_informative_segment(oracle_lib):
    # Two clusters differ only in segment 2's mean; every other segment is
    # noise-free.  Every split except those on segment 2 (or its halves)
    # leaves both children as wide as the parent, so the policy must split
    # segment 2, and the H-split (listed first) wins the tie with the
    # V-splits of equal score.
    n = 32
    X = np.zeros((10, n), np.float32)
    X[5:, 16:24] = 3.0
    p = otree.best_split(X, list(range(10)), otree.root_segmentation(n))
    assert (p.kind, p.seg, p.stat) == ("H", 2, 0)
    assert p.threshold == 1.5
    assert list(p.side(X, np.arange(10))) == [False] * 5 + [True] * 5


def test_policy_prefers_v_split_when_halves_differ(oracle_lib):
    # Segment 0 of every series has the same mean and std, but its two
    # halves differ between the clusters: only a V-split can separate them.
    n = 16
    X = np.zeros((8, n), np.float32)
    X[:4, 0:2] = 1.0
    X[:4, 2:4] = -1.0
    X[4:, 0:2] = -1.0
    X[4:, 2:4] = 1.0
    p = otree.best_split(X, list(range(8)), otree.root_segmentation(n))
    assert p.kind == "V" and p.seg == 0 and p.stat == 0
    assert otree.child_segmentation([4, 8, 12, 16], "V", 0) == [2, 4, 8, 12, 16]
    assert sorted(p.side(X, np.arange(8)).tolist()) == [False] * 4 + [True] * 4


def test_unsplittable_node_stays_leaf(oracle_lib):
    X = np.tile(np.linspace(-1, 1, 16, dtype=np.float32), (30, 1))
    assert otree.best_split(X, list(range(30)), [4, 8, 12, 16]) is None
    root = otree.build_tree(X, 10)
    assert root.is_leaf and root.unsplittable and len(root.members) == 30


def _check_tree(X, root, tau):
    leaves = otree.leaves_inorder(root)
    seen = np.concatenate([np.asarray(l.members, np.int64) for l in leaves])
    assert sorted(seen.tolist()) == list(range(X.shape[0]))     # a partition
    for leaf in leaves:
        assert len(leaf.members) <= tau or leaf.unsplittable
        assert leaf.members == sorted(leaf.members)
        assert leaf.seg_end[-1] == X.shape[1]
        assert all(a < b for a, b in zip(leaf.seg_end, leaf.seg_end[1:]))
        env = otree.leaf_synopsis(X, leaf)
        a = 0
        for j, b in enumerate(leaf.seg_end):
            mu, sd = oracle.seg_stats_rows(X, leaf.members, a, b)
            assert env[j, 0] <= mu.min() and mu.max() <= env[j, 1]
            assert env[j, 2] <= sd.min() and sd.max() <= env[j, 3]
            a = b
    return leaves


def _route(root, X, i):
    node = root
    while not node.is_leaf:
        mu, sd = oracle.seg_stats(X[i], node.policy.a, node.policy.b)
        v = mu if node.policy.stat == 0 else sd
        node = node.left if v < node.policy.threshold else node.right
    return node


@pytest.mark.parametrize("N,n,tau", [(400, 16, 20), (600, 64, 50), (300, 96, 25)])
def test_tree_invariants(oracle_lib, N, n, tau):
    rng = np.random.default_rng(N)
    X = np.cumsum(rng.standard_normal((N, n)), axis=1)
    X = ((X - X.mean(1, keepdims=True)) / X.std(1, keepdims=True)).astype(np.float32)
    root = otree.build_tree(X, tau)
    leaves = _check_tree(X, root, tau)
    assert len(leaves) >= N // tau
    # routing any series again lands it in the leaf that holds it
    where = {}
    for li, leaf in enumerate(leaves):
        for m in leaf.members:
            where[m] = li
    for i in range(0, N, 7):
        assert leaves.index(_route(root, X, i)) == where[i]
    # children segmentation: H keeps it, V adds exactly one cut point
    stack = [root]
    while stack:
        node = stack.pop()
        if node.is_leaf:
            continue
        extra = len(node.left.seg_end) - len(node.seg_end)
        assert extra == (1 if node.policy.kind == "V" else 0)
        assert set(node.seg_end) <= set(node.left.seg_end)
        assert node.left.seg_end == node.right.seg_end
        stack += [node.left, node.right]


def test_single_leaf_when_capacity_not_exceeded(oracle_lib):
    X = np.random.default_rng(0).standard_normal((50, 32)).astype(np.float32)
    root = otree.build_tree(X, 50)
    assert root.is_leaf and root.members == list(range(50))
    root = otree.build_tree(X, 49)
    assert not root.is_leaf


def test_eval_cap_uses_first_members(oracle_lib):
    # With eval_cap = 4 the policy sees only series 0..3, which differ in
    # segment 1 only; series 4.. differ in segment 3 and must not steer it.
    n = 16
    X = np.zeros((12, n), np.float32)
    X[2:4, 4:8] = 1.0
    X[4:, 12:16] = np.linspace(-5, 5, 8, dtype=np.float32)[:, None]
    root = otree.build_tree(X, 3, eval_cap=4)
    assert root.policy.seg == 1 and root.policy.threshold == 0.5
    root_full = otree.build_tree(X, 3, eval_cap=4096)
    assert root_full.policy.seg == 1      # at overflow only 4 series exist


# ---- internal-node synopses (Sec. 3.3: ProcessLeaf, VSplitSynopsis, HSplitSynopsis)

@pytest.mark.parametrize("N,n,tau,seed", [(600, 64, 20, 0), (400, 32, 8, 1), (300, 16, 5, 2)])
def test_folded_synopses_equal_their_definition(oracle_lib, N, n, tau, seed):
    from oracle import tree
    rng = np.random.default_rng(seed)
    X = np.cumsum(rng.standard_normal((N, n)), axis=1)
    X = ((X - X.mean(1, keepdims=True)) / X.std(1, keepdims=True)).astype(np.float32)
    root = tree.build_tree(X, tau)
    syn = tree.fold_synopses(X, root)
    nodes = tree.nodes_preorder(root)
    assert sum(1 for nd in nodes if not nd.is_leaf) >= 5
    for nd in nodes:
        np.testing.assert_array_equal(syn[id(nd)], tree.node_synopsis(X, nd))


def test_vsplit_fold_worked_example(oracle_lib):
    """A parent that split its first segment [0, 4) vertically, with one
    series in each child.  Over [0, 4) both series have mean 1 and std 1,
    while over the halves each has std 0 and means 0 / 2: the parent's
    synopsis of [0, 4) must come from the raw points (VSplitSynopsis), not
    from the children's halves, whose union (means [0, 2], stds [0, 0])
    would not even enclose the series."""
    from oracle import tree
    X = np.zeros((2, 16), np.float32)
    X[0, :4] = [0, 0, 2, 2]
    X[1, :4] = [2, 2, 0, 0]
    child_seg = [2, 4, 8, 12, 16]
    root = tree.Node([4, 8, 12, 16])
    root.policy = tree.Policy("V", 0, 0, 0, 0, 2, 1.0)
    root.left = tree.Node(list(child_seg), members=[0])
    root.right = tree.Node(list(child_seg), members=[1])
    expect = np.array([[1, 1, 1, 1], [0, 0, 0, 0], [0, 0, 0, 0], [0, 0, 0, 0]], np.float64)
    syn = tree.fold_synopses(X, root)
    np.testing.assert_array_equal(syn[id(root)], expect)
    np.testing.assert_array_equal(tree.node_synopsis(X, root), expect)
    np.testing.assert_array_equal(syn[id(root.left)][:2], [[0, 0, 0, 0], [2, 2, 0, 0]])


def test_node_lb_bounds_every_member(oracle_lib):
    """LB_EAPCA of a query to any node's synopsis is at most the distance to
    each series of the node's subtree: pruning a whole subtree on its root's
    bound is exact (Sec. 3.4)."""
    import oracle
    from oracle import tree
    rng = np.random.default_rng(5)
    X = np.cumsum(rng.standard_normal((300, 32)), axis=1)
    X = ((X - X.mean(1, keepdims=True)) / X.std(1, keepdims=True)).astype(np.float32)
    Q = X[rng.integers(0, 300, 6)] + rng.standard_normal((6, 32)).astype(np.float32)
    root = tree.build_tree(X, 10)
    for nd in tree.nodes_preorder(root):
        env = tree.node_synopsis(X, nd)
        for q in Q:
            lb = oracle.lb_eapca(q, nd.seg_end, env)
            for i in tree.subtree_members(nd):
                assert lb <= oracle.dist2(q, X[i]) * (1 + 1e-12)
