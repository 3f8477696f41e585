"""Seeded observations that sit on the forest's own thresholds.

Every feature value is, with probability 1/2, a threshold that the forest
uses on that feature, moved by one float step up or down in a third of those
cases each; some values are replaced by -0.0, +0.0, +inf, -inf and NaN.
Such rows make the comparison x <= t meet equality and near-equality at
many nodes, and so hit the three-level super-nodes' key-prefix ties.  This
module only draws inputs; it holds none of the method's arithmetic."""
import numpy as np


def rows_on_thresholds(forest, X: np.ndarray, seed: int, specials: bool = True) -> np.ndarray:
    rng = np.random.default_rng(seed)
    X = np.array(X, dtype=np.float32, copy=True)
    n, F = X.shape
    internal = forest.left >= 0
    for f in range(F):
        thr = forest.threshold[internal & (forest.feature == f)]
        if thr.size == 0:
            continue
        pick = rng.random(n) < 0.5
        v = thr[rng.integers(0, thr.size, size=int(pick.sum()))].astype(np.float32)
        step = rng.integers(-1, 2, size=v.size)
        v = np.where(step > 0, np.nextafter(v, np.float32(np.inf)),
                     np.where(step < 0, np.nextafter(v, np.float32(-np.inf)), v)).astype(np.float32)
        X[pick, f] = v
    if specials:
        sp = np.array([-0.0, 0.0, np.inf, -np.inf, np.nan], dtype=np.float32)
        m = rng.random(X.shape) < 0.02
        X[m] = sp[rng.integers(0, sp.size, size=int(m.sum()))]
    return X
