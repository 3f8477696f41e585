"""Pins of the oracle for forests with real leaf values (regression and
boosted trees) and of the trainers that make them.

The oracle's value path is the plain definition: the leaf walk of every
tree, then bias + scale * the fp64 sum of the reached leaves' values.  It is
checked against a hand-worked fixture, exact algebraic properties, an
independent per-tree walk, and the float32 error bound the GPU parity tests
use; the trainers are checked against the definitions of a leaf value (mean
target in a leaf; learning rate times the mean residual for boosting) and
against a brute-force best split."""
from fractions import Fraction

import numpy as np
import pytest

import datagen
import oracle
from golden_io import load_values


@pytest.fixture(scope="module")
def small_regress():
    X, y = datagen.gen_regression(11, 3000, 0, 1.0, 1.0)
    F = datagen.train_regression(X, y, 8, mtry=9, min_leaf=3, seed=11, threads=4)
    return F, X, y


@pytest.fixture(scope="module")
def small_boosted():
    X, y = datagen.gen_regression(12, 2000, 0, 1.0, 1.0)
    F = datagen.train_regression(X, y, 20, mtry=28, max_depth=3, eta=0.1, seed=12)
    return F, X, y


def test_values_fixture_worked_by_hand():
    F, X, exp = load_values("values_small.txt")
    r = oracle.predict_values(F, X)
    np.testing.assert_array_equal(r["leaf"], exp["leaf"])
    np.testing.assert_array_equal(r["sum"], exp["sum"])
    np.testing.assert_array_equal(r["out"], exp["out"])


def test_unit_leaf_values_count_trees(small_regress):
    F, X, _ = small_regress
    ones = datagen.Forest(F.n_features, 1, F.node_begin, F.left, F.right, F.feature, F.threshold, F.leaf_class,
                          F.cardinality, leaf_value=np.where(F.left < 0, 1.0, 0.0), value_scale=1.0,
                          value_bias=0.0)
    r = oracle.predict_values(ones, X[:500])
    np.testing.assert_array_equal(r["sum"], np.full(500, float(F.n_trees)))


def test_linearity_in_the_leaf_values(small_regress):
    F, X, _ = small_regress
    F2 = datagen.Forest(F.n_features, 1, F.node_begin, F.left, F.right, F.feature, F.threshold, F.leaf_class,
                        F.cardinality, leaf_value=F.leaf_value * np.float32(2.0), value_scale=F.value_scale,
                        value_bias=F.value_bias)
    a = oracle.predict_values(F, X[:500])
    b = oracle.predict_values(F2, X[:500])
    np.testing.assert_array_equal(b["sum"], 2.0 * a["sum"])


def test_independent_per_tree_walk(small_boosted):
    F, X, _ = small_boosted
    r = oracle.predict_values(F, X[:40])
    for i in range(40):
        total = 0.0
        for t in range(F.n_trees):
            tr = F.tree(t)
            v = 0
            while tr["left"][v] >= 0:
                v = int(tr["left"][v]) if X[i, tr["feature"][v]] <= tr["threshold"][v] else int(tr["right"][v])
            total += float(F.leaf_value[F.node_begin[t] + v])
        assert r["sum"][i] == total
        assert r["out"][i] == F.value_bias + F.value_scale * total


def test_tolerance_covers_float32_sums_in_any_order(small_regress):
    """The bound the GPU parity tests use holds for float32 evaluations that
    add the leaf values in shuffled orders (a plain float32 loop)."""
    F, X, _ = small_regress
    r = oracle.predict_values(F, X[:200])
    vals = F.leaf_value[F.node_begin[:-1][None, :] + r["leaf"]]
    tol = oracle.value_tolerance(F, r["abs"])
    rng = np.random.Generator(np.random.PCG64(5))
    for i in range(200):
        for _ in range(3):
            s = np.float32(0.0)
            for v in vals[i][rng.permutation(F.n_trees)]:
                s = np.float32(s + v)
            out = np.float32(np.float32(F.value_bias) + np.float32(F.value_scale) * s)
            assert abs(float(out) - r["out"][i]) <= tol[i]


def test_forest_leaf_value_is_mean_in_bag_target(small_regress):
    F, X, y = small_regress
    leaves = oracle.predict(F, X, votes=False, classes=False)["leaf"]
    for t in range(F.n_trees):
        w = datagen.bootstrap_weights(11, t, X.shape[0]).astype(np.float64)
        lf = leaves[:, t]
        for leaf in np.unique(lf[w > 0])[:200]:
            m = (lf == leaf) & (w > 0)
            mean = np.sum(w[m] * y[m]) / np.sum(w[m])
            got = F.leaf_value[F.node_begin[t] + leaf]
            np.testing.assert_allclose(got, np.float32(mean), rtol=2.0 ** -22, atol=1e-30)
            assert int(np.sum(w[m])) == F.cardinality[F.node_begin[t] + leaf]


def test_boosting_leaf_value_is_scaled_mean_residual(small_boosted):
    F, X, y = small_boosted
    base = 0.0
    for v in y.tolist():  # F_0 = mean(y), summed in row order as the trainer does
        base += v
    assert F.value_scale == 1.0 and F.value_bias == base / len(y)
    leaves = oracle.predict(F, X, votes=False, classes=False)["leaf"]
    score = np.full(X.shape[0], F.value_bias)
    mse = [np.mean((y - score) ** 2)]
    for t in range(F.n_trees):
        resid = y - score
        lf = leaves[:, t]
        for leaf in np.unique(lf):
            m = lf == leaf
            got = F.leaf_value[F.node_begin[t] + leaf]
            np.testing.assert_allclose(got, np.float32(0.1 * resid[m].mean()), rtol=2.0 ** -22, atol=1e-30)
        score = score + F.leaf_value[F.node_begin[t] + lf].astype(np.float64)
        mse.append(np.mean((y - score) ** 2))
    assert all(b <= a for a, b in zip(mse, mse[1:])), "squared loss never rises"
    assert F.tree_depth.max() <= 3


def test_regression_root_split_is_the_best_split():
    """Stumps on small integer targets: the root split maximises
    S_L^2/W_L + S_R^2/W_R over every feature and threshold (exact fractions)."""
    rng = np.random.Generator(np.random.PCG64(9))
    for trial in range(5):
        n, d = 40, 3
        X = rng.integers(0, 8, size=(n, d)).astype(np.float32)
        y = rng.integers(-5, 6, size=n).astype(np.float64)
        F = datagen.train_regression(X, y, 1, mtry=d, max_depth=1, eta=0.1, seed=trial)
        tr = F.tree(0)
        assert tr["left"][0] >= 0
        best = None
        for f in range(d):
            for t in np.unique(X[:, f])[:-1]:
                L = X[:, f] <= t
                if L.all() or not L.any():
                    continue
                sl, sr = Fraction(int(y[L].sum())), Fraction(int(y[~L].sum()))
                sc = sl * sl / int(L.sum()) + sr * sr / int((~L).sum())
                best = sc if best is None else max(best, sc)
        f, t = int(tr["feature"][0]), tr["threshold"][0]
        L = X[:, f] <= t
        got = Fraction(int(y[L].sum())) ** 2 / int(L.sum()) + Fraction(int(y[~L].sum())) ** 2 / int((~L).sum())
        assert got == best
