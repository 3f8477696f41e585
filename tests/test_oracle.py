"""Pins for the CPU oracle (no GPU).

Each check ties the oracle to something other than itself: hand-worked
fixtures, an independent leaf-box enumeration, invariants of the method, the
paper's closed form for EU, and the paper's statement that its layouts do not
change predictions (Section III-A).
"""
import numpy as np
import pytest

import datagen
import oracle
from golden_io import load

FIXTURES = ["stump_split.txt", "chain_full.txt"]


# ------------------------------------------------------------ hand fixtures

@pytest.mark.parametrize("name", FIXTURES)
def test_oracle_matches_hand_fixture(name):
    forest, X, exp = load(name)
    r = oracle.predict(forest, X)
    np.testing.assert_array_equal(r["leaf"], exp["leaf"])
    np.testing.assert_array_equal(r["votes"], exp["votes"])
    np.testing.assert_array_equal(r["cls"], exp["cls"])
    assert r["visits"] == int(exp["visits"].sum())


@pytest.mark.parametrize("name", FIXTURES)
def test_oracle_fixture_one_row_at_a_time(name):
    forest, X, exp = load(name)
    for i in range(X.shape[0]):
        r = oracle.predict(forest, X[i:i + 1])
        assert r["visits"] == exp["visits"][i]
        np.testing.assert_array_equal(r["leaf"][0], exp["leaf"][i])


@pytest.mark.parametrize("name", FIXTURES)
@pytest.mark.parametrize("kind", [oracle.BF, oracle.DF, oracle.DFM, oracle.STAT])
def test_paper_layouts_match_hand_fixture(name, kind):
    forest, X, exp = load(name)
    L = oracle.Layout(forest, kind)
    p = L.predict(X)
    leaf = oracle.leaf_from_parent(forest, p["parent"], p["dir"])
    np.testing.assert_array_equal(leaf, exp["leaf"])


@pytest.mark.parametrize("name", FIXTURES)
@pytest.mark.parametrize("B,d", [(1, 0), (1, 2), (2, 0), (2, 1), (2, 5), (3, 0), (3, 3)])
def test_bin_layout_matches_hand_fixture(name, B, d):
    forest, X, exp = load(name)
    p = oracle.Layout(forest, oracle.BIN, B, d).predict(X)
    np.testing.assert_array_equal(oracle.leaf_from_parent(forest, p["parent"], p["dir"]), exp["leaf"])


def test_empty_input():
    forest, X, exp = load("chain_full.txt")
    r = oracle.predict(forest, X[:0])
    assert r["leaf"].shape == (0, 2) and r["visits"] == 0


# --------------------------------------------------- brute-force leaf boxes

def leaf_boxes(tree: dict, n_features: int):
    """For every leaf, the box of its root path: lo < x[f] <= hi per feature.

    Written independently of the walk: it enumerates paths top-down and keeps
    the bounds, then membership is tested on all leaves at once."""
    left, right, feat, thr = tree["left"], tree["right"], tree["feature"], tree["threshold"]
    out = []
    stack = [(0, np.full(n_features, -np.inf, np.float64), np.full(n_features, np.inf, np.float64))]
    while stack:
        v, lo, hi = stack.pop()
        if left[v] < 0:
            out.append((v, lo, hi))
            continue
        f, t = feat[v], float(thr[v])
        hl = hi.copy(); hl[f] = min(hl[f], t)
        lr = lo.copy(); lr[f] = max(lr[f], t)
        stack.append((int(left[v]), lo, hl))
        stack.append((int(right[v]), lr, hi))
    ids = np.array([o[0] for o in out])
    los = np.stack([o[1] for o in out])
    his = np.stack([o[2] for o in out])
    return ids, los, his


def brute_force_leaves(forest, X):
    n, T = X.shape[0], forest.n_trees
    out = np.empty((n, T), np.int32)
    Xd = X.astype(np.float64)
    for t in range(T):
        ids, lo, hi = leaf_boxes(forest.tree(t), forest.n_features)
        above = (Xd[:, None, :] > lo[None]) | np.isneginf(lo)[None]  # an open -inf bound admits -inf
        inside = np.all(above & (Xd[:, None, :] <= hi[None]), axis=2)
        cnt = inside.sum(axis=1)
        assert np.all(cnt == 1), "every observation must fall in exactly one leaf box"
        out[:, t] = ids[np.argmax(inside, axis=1)]
    return out


def test_leaf_boxes_tiny_workload(tiny_forest, tiny_rows):
    X, _ = tiny_rows
    r = oracle.predict(tiny_forest, X)
    np.testing.assert_array_equal(r["leaf"], brute_force_leaves(tiny_forest, X))


@pytest.mark.parametrize("name", FIXTURES)
def test_leaf_boxes_fixture(name):
    forest, X, exp = load(name)
    finite = np.all(np.isfinite(X) | np.isinf(X), axis=1)  # NaN rows have no box
    np.testing.assert_array_equal(brute_force_leaves(forest, X[finite]), exp["leaf"][finite])


# ------------------------------------------------------------- invariants

def test_votes_and_class_invariants(tiny_forest, tiny_rows):
    X, _ = tiny_rows
    r = oracle.predict(tiny_forest, X)
    T, C = tiny_forest.n_trees, tiny_forest.n_classes
    assert np.all(r["votes"].sum(axis=1) == T)
    cls_of_leaf = tiny_forest.leaf_class[tiny_forest.node_begin[:-1][None, :] + r["leaf"]]
    assert np.all(cls_of_leaf >= 0)
    counts = np.stack([(cls_of_leaf == c).sum(axis=1) for c in range(C)], axis=1)
    np.testing.assert_array_equal(r["votes"], counts)
    # argmax with the lowest index on ties: the first maximal entry
    np.testing.assert_array_equal(r["cls"], np.argmax(r["votes"], axis=1))
    # every leaf reached is a leaf
    assert np.all(tiny_forest.left[tiny_forest.node_begin[:-1][None, :] + r["leaf"]] == -1)


def test_thread_count_does_not_change_results(tiny_forest, tiny_rows):
    X, _ = tiny_rows
    a = oracle.predict(tiny_forest, X, threads=1)
    b = oracle.predict(tiny_forest, X, threads=4)
    for k in ("leaf", "votes", "cls"):
        np.testing.assert_array_equal(a[k], b[k])
    assert a["visits"] == b["visits"]


def test_outputs_are_optional(tiny_forest, tiny_rows):
    X, _ = tiny_rows
    full = oracle.predict(tiny_forest, X[:100])
    only = oracle.predict(tiny_forest, X[:100], leaves=False, votes=False)
    np.testing.assert_array_equal(full["cls"], only["cls"])
    assert only["visits"] == full["visits"]


# ------------------------------------------------------- layout invariance

@pytest.mark.parametrize("kind", [oracle.BF, oracle.DF, oracle.DFM, oracle.STAT])
def test_paper_layouts_preserve_predictions(tiny_forest, tiny_rows, kind):
    X, _ = tiny_rows
    ref = oracle.predict(tiny_forest, X)
    p = oracle.Layout(tiny_forest, kind).predict(X)
    np.testing.assert_array_equal(oracle.leaf_from_parent(tiny_forest, p["parent"], p["dir"]), ref["leaf"])
    cls = tiny_forest.leaf_class[tiny_forest.node_begin[:-1][None, :] + ref["leaf"]]
    np.testing.assert_array_equal(p["cls"], cls)


@pytest.mark.parametrize("B", [1, 2, 5, 16, 32])
@pytest.mark.parametrize("d", [0, 1, 3, 8])
def test_bin_layout_preserves_predictions(tiny_forest, tiny_rows, B, d):
    X, _ = tiny_rows
    ref = oracle.predict(tiny_forest, X[:2000])
    p = oracle.Layout(tiny_forest, oracle.BIN, B, d).predict(X[:2000])
    np.testing.assert_array_equal(oracle.leaf_from_parent(tiny_forest, p["parent"], p["dir"]), ref["leaf"])


# ------------------------------------------------- layout structural rules

def _children(forest, t, v):
    b = int(forest.node_begin[t])
    return int(forest.left[b + v]), int(forest.right[b + v])


def _is_leaf(forest, t, v):
    return forest.left[int(forest.node_begin[t]) + v] < 0


@pytest.mark.parametrize("name", ["tiny"] + FIXTURES)
def test_stat_layout_rules(name, tiny_forest):
    forest = tiny_forest if name == "tiny" else load(name)[0]
    a = oracle.Layout(forest, oracle.STAT).arrays()
    C = forest.n_classes
    pos = 0
    for t in range(forest.n_trees):
        n_int = int((forest.tree(t)["left"] >= 0).sum())
        span = n_int + C  # internal nodes, then the tree's class nodes
        seg = slice(pos, pos + span)
        # class nodes close the tree's array (Section III-A, DF-)
        assert np.all(a["feature"][pos + n_int: pos + span] == -1)
        assert np.all(a["feature"][pos: pos + n_int] >= 0)
        np.testing.assert_array_equal(a["cls"][pos + n_int: pos + span], np.arange(C))
        for k in range(pos, pos + n_int):
            v = a["orig"][k]
            l, r = _children(forest, t, v)
            c0, c1 = a["child0"][k], a["child1"][k]
            li, ri = not _is_leaf(forest, t, l), not _is_leaf(forest, t, r)
            b = int(forest.node_begin[t])
            if li and ri:
                hot = 1 if forest.cardinality[b + r] > forest.cardinality[b + l] else 0
            elif li or ri:
                hot = 1 if ri else 0  # the internal child is adjacent
            else:
                hot = None
            if hot is not None:
                assert (c1 if hot else c0) == k + 1, "hot child must follow its parent"
            for c, ch in ((c0, l), (c1, r)):
                if _is_leaf(forest, t, ch):
                    assert a["feature"][c] == -1 and a["cls"][c] == forest.leaf_class[b + ch]
                else:
                    assert a["orig"][c] == ch
        assert a["root"][t] == pos or (n_int == 0)
        pos += span
        del seg


def test_bin_depth0_roots_contiguous(tiny_forest):
    """Fig. 2 caption: interleaved depth zero places all roots of a bin together."""
    B = 8
    a = oracle.Layout(tiny_forest, oracle.BIN, B, 0).arrays()
    for t0 in range(0, tiny_forest.n_trees, B):
        roots = a["root"][t0:t0 + B]
        np.testing.assert_array_equal(roots, roots[0] + np.arange(len(roots)))


@pytest.mark.parametrize("d", [1, 2, 3])
def test_bin_interleaved_levels(tiny_forest, d):
    """Section III-A: levels 0..d of the bin's trees are interleaved level by
    level; level k of the block holds the trees' internal nodes of depth k."""
    B = 4
    f = tiny_forest
    a = oracle.Layout(f, oracle.BIN, B, d).arrays()
    for t0 in range(0, f.n_trees, B):
        trees = range(t0, min(t0 + B, f.n_trees))
        expect = []
        for level in range(d + 1):
            for t in trees:
                frontier = [0]
                for _ in range(level):
                    frontier = [c for v in frontier if not _is_leaf(f, t, v) for c in _children(f, t, v)]
                expect += [(t, v) for v in frontier if not _is_leaf(f, t, v)]
        start = a["root"][t0]
        got = list(zip(a["tree"][start:start + len(expect)], a["orig"][start:start + len(expect)]))
        assert got == expect


# ------------------------------------------------------------ closed forms

def test_eu_closed_form():
    """Section III-A: EU_Stat = 1 + b(1 + b(1 + b)); a line can be used at most
    four times (b = 1); BF-like use is 1 (b = 0); the unordered DF case b = 0.5
    gives 1.875 by the formula (the text prints 1.85)."""
    assert oracle.eu_stat(0.0) == 1.0
    assert oracle.eu_stat(1.0) == 4.0
    assert oracle.eu_stat(0.5) == 1.875


def test_forest_stats_fixture():
    forest, _, _ = load("chain_full.txt")
    s = oracle.forest_stats(forest)
    assert s["mean_internal"] == (4 + 7) / 2
    assert s["max_depth"] == 4
    # biases by hand: chain 6/10, 3/4, 2/3, 1/2; full 8/16, 4/8, 3/4, 2/4, 5/8, 3/5, 2/3
    b = [6 / 10, 3 / 4, 2 / 3, 1 / 2, 8 / 16, 4 / 8, 3 / 4, 2 / 4, 5 / 8, 3 / 5, 2 / 3]
    assert abs(s["mean_bias"] - sum(b) / len(b)) < 1e-12
