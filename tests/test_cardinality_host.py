"""Statistics from observations, host side (Section III-A: the cardinalities
behind the Stat ordering may be measured on observations after training).

fp_cardinality_from_leaf_counts (the library's post-order sum) is pinned to
the trainer's own node cardinalities: counting each training row's leaf with
its bootstrap multiplicity (the oracle's walk) and summing upwards must give
back exactly the in-bag counts the trainer recorded at every node while it
grew the tree.  The binding's infer_cardinality only marshals."""
import ast
import inspect

import numpy as np
import pytest

import datagen
import oracle
import paper_1806_07300_gb300 as fp


def _bootstrap_leaf_counts(forest, name):
    X, _ = datagen.rows(name, 0)
    leaf = oracle.predict(forest, X, votes=False, classes=False)["leaf"]
    seed = datagen.RECIPES[name]["seed"]
    cnt = np.zeros(forest.n_nodes, np.int64)
    for t in range(forest.n_trees):
        w = datagen.bootstrap_weights(seed, t, X.shape[0])
        np.add.at(cnt, int(forest.node_begin[t]) + leaf[:, t], w)
    return cnt


def test_sums_reproduce_training_cardinalities(tiny_forest):
    cnt = _bootstrap_leaf_counts(tiny_forest, "tiny")
    leaves = np.asarray(tiny_forest.left) < 0
    # only the leaves' entries are read: garbage in the internal ones changes nothing
    cnt[~leaves] = -12345
    card = fp.fp_cardinality_from_leaf_counts(tiny_forest, cnt)
    np.testing.assert_array_equal(card, tiny_forest.cardinality)


def test_sums_in_place_and_unreached_nodes():
    """out_card may alias leaf_count; a node that no path reaches gets 0."""
    import ctypes
    f = datagen.Forest(2, 2, np.array([0, 6], np.int64),
                       np.array([1, -1, 3, -1, -1, -1], np.int32), np.array([2, -1, 4, -1, -1, -1], np.int32),
                       np.array([0, 0, 1, 0, 0, 0], np.int32), np.array([0.5, 0, 1.5, 0, 0, 0], np.float32),
                       np.array([0, 1, 0, 0, 1, 1], np.int32), np.zeros(6, np.int64))
    keep = []
    desc = fp.make_desc(f, keep)
    buf = np.array([99, 3, 99, 4, 5, 77], np.int64)  # node 5 is unreachable
    rc = fp.lib().fp_cardinality_from_leaf_counts(ctypes.byref(desc), buf.ctypes.data, buf.ctypes.data)
    assert rc == fp.FP_OK
    np.testing.assert_array_equal(buf, [12, 3, 9, 4, 5, 0])


def test_malformed_forest_rejected(tiny_forest):
    left = np.array(tiny_forest.left, copy=True)
    v = int(np.nonzero(left >= 0)[0][3])
    left[v] = v  # a node that is its own child
    bad = datagen.Forest(tiny_forest.n_features, tiny_forest.n_classes, tiny_forest.node_begin, left,
                         tiny_forest.right, tiny_forest.feature, tiny_forest.threshold, tiny_forest.leaf_class,
                         tiny_forest.cardinality)
    with pytest.raises(fp.FPError) as e:
        fp.fp_cardinality_from_leaf_counts(bad, np.zeros(bad.n_nodes, np.int64))
    assert e.value.code == fp.FP_EINVAL


def test_binding_only_marshals():
    """infer_cardinality forwards to fp_infer_cardinality: no loop over trees
    or nodes, no arithmetic on counts in Python."""
    for fn in (fp.infer_cardinality, fp.fp_cardinality_from_leaf_counts):
        tree = ast.parse(inspect.getsource(fn).lstrip())
        loops = [n for n in ast.walk(tree) if isinstance(n, (ast.For, ast.While, ast.comprehension))]
        assert not loops, f"{fn.__name__} loops in Python"
    assert "fp_infer_cardinality" in inspect.getsource(fp.infer_cardinality)
