"""Checks of the seeded input generators and the CART trainer (no GPU).

The trainer produces the forests the method takes as input; these tests pin
its rules (bootstrap, cardinalities, purity, exact Gini optimality, threshold
placement) against brute force written independently here.
"""
from fractions import Fraction

import numpy as np
import pytest

import datagen
import oracle

MASK = (1 << 64) - 1


def _rotl(x, k):
    return ((x << k) | (x >> (64 - k))) & MASK


def _xoshiro256ss(state, n):
    s = list(state)
    out = []
    for _ in range(n):
        out.append((_rotl((s[1] * 5) & MASK, 7) * 9) & MASK)
        t = (s[1] << 17) & MASK
        s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3]
        s[2] ^= t
        s[3] = _rotl(s[3], 45)
    return out


def test_xoshiro_definition():
    # first two outputs from state {1,2,3,4}, worked by hand from the
    # published definition: rotl(2*5, 7)*9 = 11520, then s[1] becomes 0.
    state = np.array([1, 2, 3, 4], np.uint64)
    out = np.empty(16, np.uint64)
    datagen.lib().dg_xoshiro_from_state(state.ctypes.data, 16, out.ctypes.data)
    assert int(out[0]) == 11520 and int(out[1]) == 0
    assert [int(v) for v in out] == _xoshiro256ss([1, 2, 3, 4], 16)


def test_streams_are_independent_and_deterministic():
    L = datagen.lib()
    a = {L.dg_stream_first(7, p, i) for p in range(4) for i in range(50)}
    assert len(a) == 200
    assert L.dg_stream_first(7, 2, 3) == L.dg_stream_first(7, 2, 3)


def test_rows_deterministic_and_prefix_stable():
    X1, y1 = datagen.gen_logistic(3, 70000, 1)
    X2, y2 = datagen.gen_logistic(3, 1000, 1)
    np.testing.assert_array_equal(X1[:1000], X2)
    np.testing.assert_array_equal(y1[:1000], y2)
    X3, _ = datagen.gen_logistic(3, 1000, 0)
    assert not np.array_equal(X2, X3)


def test_image_rows_shape():
    X, y = datagen.gen_image(2, 2000, 1)
    assert X.shape == (2000, 784) and X.dtype == np.float32
    zero = (X == 0).mean()
    assert 0.75 < zero < 0.85, zero
    assert X.min() >= 0.0 and X.max() <= 1.0
    np.testing.assert_array_equal(np.bincount(y, minlength=10), np.full(10, 200))


def test_bootstrap_cardinalities(tiny_forest):
    """Leaf cardinalities sum to the bootstrap size; each internal node's is the
    sum of its children's; every in-bag row reaches a leaf whose weighted class
    counts reproduce that leaf's cardinality and majority class."""
    X, y = datagen.rows("tiny", 0)
    r = oracle.predict(tiny_forest, X)
    seed = datagen.RECIPES["tiny"]["seed"]
    C = tiny_forest.n_classes
    for t in range(tiny_forest.n_trees):
        tr = tiny_forest.tree(t)
        leaves = tr["left"] < 0
        assert tr["cardinality"][leaves].sum() == X.shape[0]
        internal = np.nonzero(~leaves)[0]
        np.testing.assert_array_equal(tr["cardinality"][internal],
                                      tr["cardinality"][tr["left"][internal]] + tr["cardinality"][tr["right"][internal]])
        w = datagen.bootstrap_weights(seed, t, X.shape[0])
        counts = np.zeros((len(tr["left"]), C), np.int64)
        np.add.at(counts, (r["leaf"][:, t], y), w)
        np.testing.assert_array_equal(counts.sum(axis=1)[leaves], tr["cardinality"][leaves])
        lv = np.nonzero(leaves)[0]
        np.testing.assert_array_equal(np.argmax(counts[lv], axis=1), tr["leaf_class"][lv])
        # grown to purity: an impure leaf only holds rows that no feature separates
        for v in lv[(counts[lv] > 0).sum(axis=1) > 1]:
            rows = np.nonzero((r["leaf"][:, t] == v) & (w > 0))[0]
            assert np.all(X[rows] == X[rows[0]])


def _gini_score(counts_l, counts_r):
    wl, wr = sum(counts_l), sum(counts_r)
    return Fraction(sum(c * c for c in counts_l), wl) + Fraction(sum(c * c for c in counts_r), wr)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_splits_are_gini_optimal(seed):
    """With mtry = d every feature is searched: each chosen split must reach the
    largest exact Gini score over all features and candidate thresholds, with
    its threshold at the float midpoint of two consecutive distinct values and
    the smallest such candidate on its feature."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n, d, C = 40, 3, 3
    X = rng.integers(0, 6, size=(n, d)).astype(np.float32) * np.float32(0.5)
    y = rng.integers(0, C, size=n).astype(np.int32)
    F = datagen.train_forest(X, y, C, n_trees=4, mtry=d, seed=seed)
    r = oracle.predict(F, X)
    for t in range(F.n_trees):
        tr = F.tree(t)
        w = datagen.bootstrap_weights(seed, t, n)
        # rows reaching each node, by replaying the split rule from the root
        reach = {0: np.nonzero(w > 0)[0]}
        order = [0]
        while order:
            v = order.pop()
            idx = reach[v]
            if tr["left"][v] < 0:
                continue
            f, thr = tr["feature"][v], tr["threshold"][v]
            reach[tr["left"][v]] = idx[X[idx, f] <= thr]
            reach[tr["right"][v]] = idx[X[idx, f] > thr]
            order += [tr["left"][v], tr["right"][v]]
            best = None
            cands = {}
            for g in range(d):
                vals = np.unique(X[idx, g])
                for a, b in zip(vals[:-1], vals[1:]):
                    m = idx[X[idx, g] <= a]
                    o = idx[X[idx, g] > a]
                    cl = [int(w[m][y[m] == c].sum()) for c in range(C)]
                    cr = [int(w[o][y[o] == c].sum()) for c in range(C)]
                    s = _gini_score(cl, cr)
                    cands.setdefault(g, []).append((s, a, b))
                    best = s if best is None or s > best else best
            assert best is not None
            chosen = [c for c in cands[f] if X[idx, f][X[idx, f] <= thr].max() == c[1]]
            assert len(chosen) == 1
            s, a, b = chosen[0]
            assert s == best, "chosen split must reach the best Gini score"
            mid = np.float32((np.float64(a) + np.float64(b)) / 2)
            assert thr == (mid if a <= mid < b else a)
            same = [c for c in cands[f] if c[0] == best]
            assert same[0][1] == a, "ties on a feature go to the smaller threshold"
        assert r["leaf"].shape[1] == F.n_trees


def test_trainer_deterministic_across_threads():
    X, y = datagen.rows("tiny", 0)
    a = datagen.train_forest(X, y, 4, 8, 4, seed=11, threads=1)
    b = datagen.train_forest(X, y, 4, 8, 4, seed=11, threads=5)
    for k in ("node_begin", "left", "right", "feature", "threshold", "leaf_class", "cardinality"):
        np.testing.assert_array_equal(getattr(a, k), getattr(b, k))


def test_tiny_forest_accuracy(tiny_forest, tiny_rows):
    X, y = tiny_rows
    r = oracle.predict(tiny_forest, X, leaves=False, votes=False)
    assert (r["cls"] == y).mean() > 0.9
