"""The trainer's feature draws pinned by an independent re-implementation.

The forest every benchmark consumes comes from the CART trainer in
datagen.c (bootstrap, mtry features per node by a partial Fisher-Yates
shuffle continued until a feature splits, exact Gini, ties to the feature
drawn first, then to the smaller threshold).  Here the same rules are written
again in plain Python from their published definitions -- SplitMix64 seeding
xoshiro256** (Blackman and Vigna), Lemire's multiply-shift bounded integer,
Fisher-Yates -- with Gini scores as exact fractions, and whole forests are
compared node by node on small inputs built to exercise mtry < d:
constant columns (a node's first draws often cannot split, so further
features of the same permutation are drawn) and duplicated columns (two
features score exactly the same, so the one drawn first must win)."""
from fractions import Fraction

import numpy as np
import pytest

import datagen

M64 = (1 << 64) - 1
PURPOSE_TREE = 3


def _splitmix_next(x):
    x = (x + 0x9E3779B97F4A7C15) & M64
    z = x
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return x, z ^ (z >> 31)


def _mix(z):
    return _splitmix_next(z)[1]


def _rotl(x, k):
    return ((x << k) | (x >> (64 - k))) & M64


class Rng:
    """One stream per (seed, purpose, index): the three are mixed with
    SplitMix64 into a key, whose next four SplitMix64 outputs seed
    xoshiro256**."""

    def __init__(self, seed, purpose, index):
        k = _mix(seed)
        k = _mix(k ^ _mix((purpose * 0xD1B54A32D192ED03 + 1) & M64))
        k = _mix(k ^ _mix((index * 0x8CB92BA72F3D8DD7 + 7) & M64))
        self.s = []
        for _ in range(4):
            k, out = _splitmix_next(k)
            self.s.append(out)

    def next(self):
        s = self.s
        result = (_rotl((s[1] * 5) & M64, 7) * 9) & M64
        t = (s[1] << 17) & M64
        s[2] ^= s[0]
        s[3] ^= s[1]
        s[1] ^= s[2]
        s[0] ^= s[3]
        s[2] ^= t
        s[3] = _rotl(s[3], 45)
        return result

    def bounded(self, n):  # integer in [0, n): the high 64 bits of next() * n
        return (self.next() * n) >> 64


def _best_split(X, y, w, idx, f, C):
    """Best threshold of feature f over the node's samples: the largest
    S_L/W_L + S_R/W_R (S = sum of squared weighted class counts), the smallest
    threshold on ties; the threshold is the float32 midpoint of the two
    values around it (the lower value if rounding reaches the upper)."""
    vals = sorted(set(float(v) for v in X[idx, f]))
    if len(vals) < 2:
        return None
    best = None
    for a, b in zip(vals[:-1], vals[1:]):
        left = [i for i in idx if X[i, f] <= a]
        right = [i for i in idx if X[i, f] > a]
        cl = [sum(int(w[i]) for i in left if y[i] == c) for c in range(C)]
        cr = [sum(int(w[i]) for i in right if y[i] == c) for c in range(C)]
        s = Fraction(sum(c * c for c in cl), sum(cl)) + Fraction(sum(c * c for c in cr), sum(cr))
        if best is None or s > best[0]:
            t = np.float32(np.float64(np.float32(a)) + (np.float64(np.float32(b)) - np.float64(np.float32(a))) * 0.5)
            if not (np.float32(a) <= t < np.float32(b)):
                t = np.float32(a)
            best = (s, t)
    return best


def train_reference(X, y, C, n_trees, mtry, seed, stats=None):
    """The forest as lists of nodes in pre-order; ``stats`` (a dict) counts
    nodes that drew more than mtry features and nodes where a later draw
    scored exactly as well as the best so far (a tie the first draw wins)."""
    n, d = X.shape
    trees = []
    stats = {} if stats is None else stats
    stats.setdefault("continued", 0)
    stats.setdefault("feature_ties", 0)
    for ti in range(n_trees):
        rng = Rng(seed, PURPOSE_TREE, ti)
        w = np.zeros(n, np.int64)
        for _ in range(n):
            w[rng.bounded(n)] += 1
        nodes = []  # (left, right, feature, threshold, leaf_class, cardinality), pre-order

        def grow(idx):
            me = len(nodes)
            nodes.append(None)
            cnt = [sum(int(w[i]) for i in idx if y[i] == c) for c in range(C)]
            maj = max(range(C), key=lambda c: (cnt[c], -c))  # the first largest count
            leaf = (-1, -1, -1, np.float32(0.0), maj, sum(cnt))
            if sum(1 for c in cnt if c > 0) <= 1:
                nodes[me] = leaf
                return me
            perm = list(range(d))
            bf = None
            for i in range(d):  # partial Fisher-Yates, continued until a drawn feature splits
                j = i + rng.bounded(d - i)
                perm[i], perm[j] = perm[j], perm[i]
                f = perm[i]
                r = _best_split(X, y, w, idx, f, C)
                if r is not None and bf is not None and r[0] == bf[1]:
                    stats["feature_ties"] += 1
                if r is not None and (bf is None or r[0] > bf[1]):  # ties: the feature drawn first
                    bf = (f, r[0], r[1])
                if i + 1 >= mtry and bf is not None:
                    stats["continued"] += i + 1 > mtry
                    break
            if bf is None:
                nodes[me] = leaf
                return me
            f, _, t = bf
            li = grow([i for i in idx if X[i, f] <= t])
            ri = grow([i for i in idx if X[i, f] > t])
            nodes[me] = (li, ri, f, t, -1, sum(cnt))
            return me

        grow([i for i in range(n) if w[i] > 0])
        trees.append(nodes)
    return trees


def _inputs(seed, n, d_live, n_const, n_dup, C):
    rng = np.random.Generator(np.random.PCG64(seed))
    live = rng.integers(0, 5, size=(n, d_live)).astype(np.float32) * np.float32(0.25)
    cols = [live, np.zeros((n, n_const), np.float32), live[:, :n_dup]]
    X = np.ascontiguousarray(np.concatenate(cols, axis=1))
    X = X[:, np.random.Generator(np.random.PCG64(seed + 100)).permutation(X.shape[1])]
    y = rng.integers(0, C, size=n).astype(np.int32)
    return np.ascontiguousarray(X), y


def _compare(F, ref):
    assert F.n_trees == len(ref)
    for t, nodes in enumerate(ref):
        tr = F.tree(t)
        assert len(tr["left"]) == len(nodes), f"tree {t}: node count"
        for v, (l, r, f, thr, cls, card) in enumerate(nodes):
            assert (tr["left"][v], tr["right"][v], tr["feature"][v]) == (l, r, f), f"tree {t} node {v}"
            assert tr["cardinality"][v] == card, f"tree {t} node {v}: cardinality"
            if l >= 0:
                assert tr["threshold"][v] == thr, f"tree {t} node {v}: threshold"
            else:
                assert tr["leaf_class"][v] == cls, f"tree {t} node {v}: leaf class"


@pytest.mark.parametrize("seed,mtry", [(3, 1), (4, 2), (5, 3)])
def test_draws_with_constant_and_duplicate_columns(seed, mtry):
    """mtry < d with 3 constant and 2 duplicated columns among 7: continued
    draws and exact ties between features both occur in these trees."""
    X, y = _inputs(seed, n=48, d_live=2, n_const=3, n_dup=2, C=3)
    F = datagen.train_forest(X, y, 3, n_trees=3, mtry=mtry, seed=seed, threads=1)
    _compare(F, train_reference(X, y, 3, 3, mtry, seed))


def test_reference_exercises_continued_draws_and_ties():
    """The fixtures really take both paths: across the compared forests some
    nodes draw more than mtry features, and at some nodes a later-drawn
    feature scores exactly as well as the one drawn first."""
    stats = {}
    for seed, mtry in [(3, 1), (4, 2), (5, 3)]:
        X, y = _inputs(seed, n=48, d_live=2, n_const=3, n_dup=2, C=3)
        train_reference(X, y, 3, 3, mtry, seed, stats)
    assert stats["continued"] > 0 and stats["feature_ties"] > 0, stats
