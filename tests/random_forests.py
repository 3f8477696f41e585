"""Seeded random forests with adversarial thresholds, for packer and kernel
fuzzing (not trained: the packing and the compare must be exact for any
forest a caller hands over).

Tree shapes are random (each node splits with a probability that falls with
its depth); thresholds mix ordinary values with subnormals, signed zeros,
huge magnitudes, infinities and NaN, so that the order keys, the key prefixes
and the remap of three-level super-nodes meet every corner of the float
line; cardinalities are leaf counts summed upwards (consistent, so the
Stat ordering is exercised).  Rows take values from the same mixture, the
forest's own thresholds and their float neighbours."""
from __future__ import annotations

import numpy as np

import datagen

_SPECIAL = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1e-45, -1e-45, 1.17549435e-38, -1.17549435e-38,
                     3.4028235e38, -3.4028235e38], dtype=np.float32)


def values(rng, n: int, kind: str) -> np.ndarray:
    """n float32 values: 'mixed' (every scale and sign, some specials),
    'positive' (tiny to one, as image pixels), 'narrow' (near 1000)."""
    if kind == "positive":
        return (rng.random(n) ** rng.uniform(1, 8, n)).astype(np.float32)
    if kind == "narrow":
        return (1000.0 + rng.normal(0, 1e-3, n)).astype(np.float32)
    mag = 10.0 ** rng.uniform(-40, 38, n)
    v = (np.where(rng.random(n) < 0.5, -1.0, 1.0) * mag).astype(np.float32)
    sp = rng.random(n) < 0.1
    v[sp] = _SPECIAL[rng.integers(0, _SPECIAL.size, int(sp.sum()))]
    return v


def forest(seed: int, n_trees: int = 12, n_features: int = 9, n_classes: int = 5, max_depth: int = 9,
           kind: str = "mixed", nan_thresholds: bool = True) -> datagen.Forest:
    rng = np.random.default_rng(seed)
    begin = [0]
    L, R, Fe, Th, Cl, Ca = [], [], [], [], [], []
    for _ in range(n_trees):
        left, right, feat, thr, cls = [], [], [], [], []

        def grow(depth):
            me = len(left)
            left.append(-1), right.append(-1), feat.append(0), thr.append(0.0), cls.append(0)
            if depth < max_depth and rng.random() < 0.92 - 0.08 * depth:
                feat[me] = int(rng.integers(0, n_features))
                t = values(rng, 1, kind)[0]
                if not nan_thresholds and np.isnan(t):
                    t = np.float32(0.5)
                thr[me] = t
                left[me] = grow(depth + 1)
                right[me] = grow(depth + 1)
            else:
                cls[me] = int(rng.integers(0, n_classes))
            return me

        grow(0)
        m = len(left)
        card = np.zeros(m, np.int64)
        for v in range(m - 1, -1, -1):  # children come after their parent (pre-order)
            card[v] = int(rng.integers(1, 50)) if left[v] < 0 else card[left[v]] + card[right[v]]
        L += left; R += right; Fe += feat; Th += thr; Cl += cls; Ca += list(card)
        begin.append(begin[-1] + m)
    return datagen.Forest(n_features, n_classes, np.array(begin, np.int64), np.array(L, np.int32),
                          np.array(R, np.int32), np.array(Fe, np.int32), np.array(Th, np.float32),
                          np.array(Cl, np.int32), np.array(Ca, np.int64))


def rows(f: datagen.Forest, n: int, seed: int, kind: str = "mixed") -> np.ndarray:
    """Rows whose values come from the mixture, the forest's thresholds of
    that feature, and those thresholds' float neighbours."""
    rng = np.random.default_rng(seed)
    X = values(rng, n * f.n_features, kind).reshape(n, f.n_features)
    internal = f.left >= 0
    for j in range(f.n_features):
        thr = f.threshold[internal & (f.feature == j)]
        thr = thr[~np.isnan(thr)]
        if thr.size == 0:
            continue
        pick = rng.random(n) < 0.6
        v = thr[rng.integers(0, thr.size, int(pick.sum()))]
        step = rng.integers(-1, 2, v.size)
        with np.errstate(over="ignore"):  # the neighbours of the largest finite thresholds are infinite
            v = np.where(step > 0, np.nextafter(v, np.float32(np.inf)),
                         np.where(step < 0, np.nextafter(v, np.float32(-np.inf)), v)).astype(np.float32)
        X[pick, j] = v
    return np.ascontiguousarray(X)
