"""Oracle Hercules tree: sequential insertion (Sec. 3.2, Sec. 3.3).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Parity unpinned for the split policy: the paper leaves getBestSplitPolicy to
DSTree, so which split a node takes is this project's reading (below); what
the paper fixes -- the threshold rule of its worked example, children that
partition their parent, synopses that enclose their members, inorder leaf
order -- is pinned by tests.  Exact answers do not depend on the policy: any
valid tree gives the same k nearest neighbours.

Series are inserted one at a time in id order, as Algorithm InsertSeriesToNode
does for a single insert worker: route to a leaf through the split policies of
the internal nodes, append, and split the leaf once it holds more than tau
series (Sec. 3.2: a leaf that exceeds its capacity tau becomes an internal node
with two leaf children).

Node split (Sec. 3.2).  A node with segmentation SG = (r_1..r_m) is split on
one of its segments SG_i = [r_{i-1}, r_i):
  * H-split: children keep SG; a series goes left when its mean (or std) over
    SG_i is in [v_min, (v_min+v_max)/2) and right otherwise, v_min/v_max taken
    over the node's series (the worked example in Sec. 3.2: mean range
    [-0.25, 0.10] gives the threshold -0.075).
  * V-split: SG_i is first cut in two, then an H-split is applied on one of the
    two halves; children have m+1 segments.

Readings where the paper is silent (it defers getBestSplitPolicy to DSTree):
  * root segmentation: 4 equal segments (n divisible by 4);
  * a V-split cuts [a, b) at floor((a+b)/2), only when b - a >= 2 and the
    node has fewer than MAX_SEGMENTS (64) segments;
  * candidates, enumerated in this order (earlier wins a tie): for each segment
    i ascending, for the mean then the std: the H-split on SG_i, the V-split
    on the left half, the V-split on the right half;
  * the threshold is (v_min + v_max) * 0.5, left is value < threshold;
  * a candidate that leaves a child empty is invalid;
  * the chosen candidate minimises n_l * E(N_l) + n_r * E(N_r), with
    E(child) = sum_j l_j * ((mu_max_j - mu_min_j)^2 + (sd_max_j - sd_min_j)^2)
    over the child's segmentation and the child's series (the mean of the two
    children's spreads weighted by size; the common factor 1/|N| is dropped);
  * a node with no valid candidate stays a leaf for good (it may exceed tau);
  * the policy is chosen from the node's first min(tau + 1, eval_cap) series
    in insertion (id) order, i.e. from the series it holds when it overflows,
    capped at eval_cap (default 4096) so the cost of a split stays bounded for
    large leaf capacities.  Routing then uses the chosen policy for all of
    the node's series.

Every quantity is binary64 with the operation order written here; the segment
statistics come from the oracle's C routine (two passes, sequential sums).
"""
from dataclasses import dataclass, field

import numpy as np

from . import seg_stats, seg_stats_rows

ROOT_SEGMENTS = 4
MAX_SEGMENTS = 64


def root_segmentation(n: int):
    assert n % ROOT_SEGMENTS == 0
    l = n // ROOT_SEGMENTS
    return [l * (i + 1) for i in range(ROOT_SEGMENTS)]


@dataclass
class Policy:
    kind: str          # 'H' or 'V'
    seg: int           # segment index i in the parent's segmentation
    half: int          # -1 for H, 0/1 for the half a V-split tests
    stat: int          # 0 = mean, 1 = std
    a: int             # tested range [a, b)
    b: int
    threshold: float

    def side(self, X, rows):
        """True where the series goes right (value >= threshold)."""
        mu, sd = seg_stats_rows(X, rows, self.a, self.b)
        v = mu if self.stat == 0 else sd
        return ~(v < self.threshold)


@dataclass
class Node:
    seg_end: list
    members: list = field(default_factory=list)
    policy: Policy | None = None
    left: "Node | None" = None
    right: "Node | None" = None
    unsplittable: bool = False

    @property
    def is_leaf(self):
        return self.policy is None


def candidates(seg_end):
    """(kind, seg, half, stat, a, b) in tie-break order."""
    out = []
    a = 0
    can_v = len(seg_end) < MAX_SEGMENTS
    for i, b in enumerate(seg_end):
        mid = (a + b) // 2
        for stat in (0, 1):
            out.append(("H", i, -1, stat, a, b))
            if b - a >= 2 and can_v:
                out.append(("V", i, 0, stat, a, mid))
                out.append(("V", i, 1, stat, mid, b))
        a = b
    return out


def child_segmentation(seg_end, kind, seg):
    if kind == "H":
        return list(seg_end)
    a = 0 if seg == 0 else seg_end[seg - 1]
    b = seg_end[seg]
    mid = (a + b) // 2
    return list(seg_end[:seg]) + [mid] + list(seg_end[seg:])


def spread(stats_by_range, child_seg, mask):
    """E(child) = sum_j l_j ((mu_max-mu_min)^2 + (sd_max-sd_min)^2) over the
    child's segments, for the series selected by mask."""
    e = 0.0
    a = 0
    for b in child_seg:
        mu, sd = stats_by_range[(a, b)]
        mu = mu[mask]
        sd = sd[mask]
        dm = float(mu.max()) - float(mu.min())
        ds = float(sd.max()) - float(sd.min())
        t = dm * dm + ds * ds
        e = e + float(b - a) * t
        a = b
    return e


def best_split(X, members, seg_end):
    """The policy the reading above picks for these members, or None."""
    rows = np.asarray(members, dtype=np.int64)
    cands = candidates(seg_end)
    ranges = set()
    a = 0
    for b in seg_end:
        ranges.add((a, b))
        mid = (a + b) // 2
        if b - a >= 2:
            ranges.add((a, mid))
            ranges.add((mid, b))
        a = b
    stats = {r: seg_stats_rows(X, rows, r[0], r[1]) for r in ranges}
    best = None
    best_score = None
    for kind, seg, half, stat, ca, cb in cands:
        v = stats[(ca, cb)][stat]
        thr = (float(v.min()) + float(v.max())) * 0.5
        left = v < thr
        nl = int(left.sum())
        nr = rows.size - nl
        if nl == 0 or nr == 0:
            continue
        cseg = child_segmentation(seg_end, kind, seg)
        el = spread(stats, cseg, left)
        er = spread(stats, cseg, ~left)
        score = float(nl) * el + float(nr) * er
        if best_score is None or score < best_score:
            best_score = score
            best = Policy(kind, seg, half, stat, ca, cb, thr)
    return best


def _route(node, X, i):
    while not node.is_leaf:
        p = node.policy
        mu, sd = seg_stats(X[i], p.a, p.b)
        v = mu if p.stat == 0 else sd
        node = node.left if v < p.threshold else node.right
    return node


EVAL_CAP = 4096


def _split(node, X, eval_cap):
    p = best_split(X, node.members[:eval_cap], node.seg_end)
    if p is None:
        node.unsplittable = True
        return
    cseg = child_segmentation(node.seg_end, p.kind, p.seg)
    node.policy = p
    node.left = Node(list(cseg))
    node.right = Node(list(cseg))
    rows = np.asarray(node.members, dtype=np.int64)
    right = p.side(X, rows)
    node.left.members = [int(r) for r, g in zip(rows, right) if not g]
    node.right.members = [int(r) for r, g in zip(rows, right) if g]
    node.members = []


def build_tree(X, tau: int, eval_cap: int = EVAL_CAP):
    """Insert X's rows in id order; return the root Node."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    N, n = X.shape
    root = Node(root_segmentation(n))
    for i in range(N):
        leaf = _route(root, X, i)
        leaf.members.append(i)
        if len(leaf.members) > tau and not leaf.unsplittable:
            _split(leaf, X, eval_cap)
    return root


def leaves_inorder(root):
    out = []
    stack = [root]
    while stack:
        node = stack.pop()
        if node.is_leaf:
            out.append(node)
        else:
            stack.append(node.right)
            stack.append(node.left)
    return out


def leaf_synopsis(X, leaf):
    """Synopsis Z of a leaf (Sec. 3.2): per segment (mu_min, mu_max, sd_min,
    sd_max) over its series, as an [m, 4] binary64 array."""
    rows = np.asarray(leaf.members, dtype=np.int64)
    env = np.empty((len(leaf.seg_end), 4), dtype=np.float64)
    a = 0
    for j, b in enumerate(leaf.seg_end):
        mu, sd = seg_stats_rows(X, rows, a, b)
        env[j] = (mu.min(), mu.max(), sd.min(), sd.max())
        a = b
    return env


def nodes_preorder(root):
    """Every node, parents before children, left subtree before right."""
    out = []
    stack = [root]
    while stack:
        node = stack.pop()
        out.append(node)
        if not node.is_leaf:
            stack.append(node.right)
            stack.append(node.left)
    return out


def subtree_members(node):
    """Ids of every series in the node's subtree (the series that traversed
    it), in inorder leaf order."""
    return [i for leaf in leaves_inorder(node) for i in leaf.members]


def node_synopsis(X, node):
    """Synopsis of any node by its definition (Sec. 3.3): for every segment of
    the node's own segmentation, the min / max of the mean and of the std over
    all series that traversed the node, as an [m, 4] binary64 array."""
    rows = np.asarray(subtree_members(node), dtype=np.int64)
    env = np.empty((len(node.seg_end), 4), dtype=np.float64)
    a = 0
    for j, b in enumerate(node.seg_end):
        mu, sd = seg_stats_rows(X, rows, a, b)
        env[j] = (mu.min(), mu.max(), sd.min(), sd.max())
        a = b
    return env


def fold_synopses(X, root):
    """Synopses of every node as the paper's post-processing of each leaf
    computes them (Sec. 3.3, Algorithms ProcessLeaf, VSplitSynopsis and
    HSplitSynopsis), leaf by leaf in inorder:
      * each leaf's own synopsis comes from its series (insertion keeps it);
      * VSplitSynopsis, per series of the leaf: every ancestor whose split
        was vertical updates the segment it split (its own segmentation's
        segment) with the series' mean and std over that segment;
      * HSplitSynopsis, once per leaf: walking up from the leaf, each parent
        updates every segment it did not split vertically with the min / max
        of the corresponding segment (same end points) of the child on the
        path.
    Returns {id(node): [m, 4] array}."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    parent = {}
    for node in nodes_preorder(root):
        if not node.is_leaf:
            parent[id(node.left)] = node
            parent[id(node.right)] = node
    syn = {}
    for node in nodes_preorder(root):
        m = len(node.seg_end)
        syn[id(node)] = np.tile(np.array([np.inf, -np.inf, np.inf, -np.inf]), (m, 1))

    def upd(z, mu, sd):
        z[0] = min(z[0], mu)
        z[1] = max(z[1], mu)
        z[2] = min(z[2], sd)
        z[3] = max(z[3], sd)

    for leaf in leaves_inorder(root):
        syn[id(leaf)] = leaf_synopsis(X, leaf)
        for i in leaf.members:                           # VSplitSynopsis
            node = parent.get(id(leaf))
            while node is not None:
                if node.policy.kind == "V":
                    j = node.policy.seg
                    a = 0 if j == 0 else node.seg_end[j - 1]
                    mu, sd = seg_stats(X[i], a, node.seg_end[j])
                    upd(syn[id(node)][j], mu, sd)
                node = parent.get(id(node))
        child = leaf                                     # HSplitSynopsis
        node = parent.get(id(leaf))
        while node is not None:
            vseg = node.policy.seg if node.policy.kind == "V" else -1
            cz = syn[id(child)]
            a = 0
            for j, b in enumerate(node.seg_end):
                if j != vseg:
                    jc = child.seg_end.index(b)          # the child's segment ending at b
                    ac = 0 if jc == 0 else child.seg_end[jc - 1]
                    assert ac == a, "child segment does not match the parent's"
                    z = syn[id(node)][j]
                    z[0] = min(z[0], cz[jc][0])
                    z[1] = max(z[1], cz[jc][1])
                    z[2] = min(z[2], cz[jc][2])
                    z[3] = max(z[3], cz[jc][3])
                a = b
            child = node
            node = parent.get(id(node))
    return syn
