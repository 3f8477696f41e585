"""Seeded synthetic inputs: observation matrices and trained forests.

The paper's method starts from a trained forest (Section III) and classifies
observations with it.  Neither the paper's datasets (MNIST, Higgs, Allstate,
Table I) nor its trained forests are available, so this module generates
stand-ins with the shapes of Table I and trains CART forests on them
(Section IV-C: Gini, grown to maximum depth).  It holds none of the packing or
classification arithmetic; the oracle and the GPU library both consume it.

Workloads (each a dict made by :func:`workload`):

* ``tiny``: 4-class mixture of unit Gaussians, means U[-2,2]^16; 2,000 training
  rows, 16 trees, mtry 4; test rows from the same mixture; seed 0.
* ``image``: 784 features in [0,1] with ~80 % exact zeros, 10 balanced
  classes; 60,000 training rows, 128 trees, mtry 28; seed 2 (MNIST stand-in).
* ``hbm``: 28 features (21 normal, 7 log-normal), 2 classes from a noisy
  logistic model with pairwise terms; 500,000 training rows, 256 trees, mtry 5;
  seed 3 (Allstate/Higgs stand-in; forest far larger than L2).
* ``batched``: 8 Gaussian-mixture forests of varied tree, feature and class
  counts; seed 4.
* ``wide``: 64-tree, 50-class, 100-feature mixture forest for serving; seed 5.
* ``regress``: regression forest with real leaf values (the forest variants
  the paper names beside classification): the ``hbm`` features with a real
  target (the logistic model's score plus Gaussian noise); 200,000 training
  rows, 128 trees, mtry 9, leaves of at least 5; seed 6.
* ``boosted``: gradient-boosted shallow trees (squared loss, depth <= 6,
  learning rate 0.1) on the same kind of rows; 30,000 training rows, 256
  rounds; seed 7.
"""
from __future__ import annotations

import ctypes
import hashlib
import json
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "datagen.c")
_LIB_PATH = os.path.join(_HERE, "libfpdata.so")
_lib = None
_lock = threading.Lock()

REPO_ROOT = os.path.dirname(_HERE)
CACHE_DIR = os.environ.get("FP_CACHE_DIR", os.path.join(REPO_ROOT, ".fpcache"))

# Label-noise scale of the logistic workload; chosen so that trees grown to
# purity on 500,000 rows hold about 10^5 internal nodes (Table I, Allstate).
HBM_LOGIT_SCALE = 0.25


def build(force: bool = False) -> str:
    """Compile datagen.c into libfpdata.so (plain gcc, no fast-math)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-pthread", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            i32, i64, u64, u32, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double
            P = ctypes.c_void_p
            L.dg_gen_mixture.argtypes = [u64, i32, i32, dbl, dbl, i64, u32, P, P, ctypes.c_int]
            L.dg_gen_mixture.restype = ctypes.c_int
            L.dg_gen_image.argtypes = [u64, i64, u32, P, P, ctypes.c_int]
            L.dg_gen_image.restype = ctypes.c_int
            L.dg_gen_logistic.argtypes = [u64, i64, u32, dbl, P, P, ctypes.c_int]
            L.dg_gen_logistic.restype = ctypes.c_int
            L.dg_train.argtypes = [P, P, i64, i32, i32, i32, i32, u64, ctypes.c_int]
            L.dg_train.restype = P
            L.dg_forest_total_nodes.argtypes = [P]
            L.dg_forest_total_nodes.restype = i64
            L.dg_forest_n_trees.argtypes = [P]
            L.dg_forest_n_trees.restype = i32
            L.dg_forest_export.argtypes = [P] * 9
            L.dg_forest_export.restype = None
            L.dg_forest_free.argtypes = [P]
            L.dg_forest_free.restype = None
            L.dg_bootstrap_weights.argtypes = [u64, i32, i64, P]
            L.dg_bootstrap_weights.restype = None
            L.dg_stream_first.argtypes = [u64, u64, u64]
            L.dg_stream_first.restype = u64
            L.dg_xoshiro_from_state.argtypes = [P, ctypes.c_int, P]
            L.dg_xoshiro_from_state.restype = None
            L.dg_gen_regression.argtypes = [u64, i64, u32, dbl, dbl, P, P, ctypes.c_int]
            L.dg_gen_regression.restype = ctypes.c_int
            L.dg_train_regression.argtypes = [P, P, i64, i32, i32, i32, i32, i64, dbl, u64, P, ctypes.c_int]
            L.dg_train_regression.restype = P
            L.dg_forest_export_values.argtypes = [P, P]
            L.dg_forest_export_values.restype = None
            _lib = L
    return _lib


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def n_threads() -> int:
    return max(1, min(64, os.cpu_count() or 1))


# ----------------------------------------------------------------- rows

def gen_mixture(seed: int, n_classes: int, n_features: int, n: int, split: int,
                lo: float = -2.0, hi: float = 2.0):
    X = np.empty((n, n_features), dtype=np.float32)
    y = np.empty(n, dtype=np.int32)
    rc = lib().dg_gen_mixture(seed, n_classes, n_features, lo, hi, n, split, _ptr(X), _ptr(y), n_threads())
    if rc != 0:
        raise RuntimeError(f"dg_gen_mixture failed: {rc}")
    return X, y


def gen_image(seed: int, n: int, split: int):
    X = np.empty((n, 784), dtype=np.float32)
    y = np.empty(n, dtype=np.int32)
    rc = lib().dg_gen_image(seed, n, split, _ptr(X), _ptr(y), n_threads())
    if rc != 0:
        raise RuntimeError(f"dg_gen_image failed: {rc}")
    return X, y


def gen_logistic(seed: int, n: int, split: int, scale: float = HBM_LOGIT_SCALE):
    X = np.empty((n, 28), dtype=np.float32)
    y = np.empty(n, dtype=np.int32)
    rc = lib().dg_gen_logistic(seed, n, split, scale, _ptr(X), _ptr(y), n_threads())
    if rc != 0:
        raise RuntimeError(f"dg_gen_logistic failed: {rc}")
    return X, y


def gen_regression(seed: int, n: int, split: int, scale: float = 1.0, noise: float = 1.0):
    X = np.empty((n, 28), dtype=np.float32)
    y = np.empty(n, dtype=np.float64)
    rc = lib().dg_gen_regression(seed, n, split, scale, noise, _ptr(X), _ptr(y), n_threads())
    if rc != 0:
        raise RuntimeError(f"dg_gen_regression failed: {rc}")
    return X, y


# --------------------------------------------------------------- forests

class Forest:
    """A trained forest as flat arrays (node ids are tree-local, pre-order).

    ``left[i] == -1`` marks a leaf; ``leaf_class`` is set on leaves only.
    ``cardinality`` is the in-bag training count (with bootstrap multiplicity)
    reaching each node.  Forests with real leaf values (regression, boosting)
    also carry ``leaf_value`` (float32 per node, 0 on internal nodes) and
    predict ``value_bias + value_scale * sum over trees of the leaf value``.
    """

    def __init__(self, n_features, n_classes, node_begin, left, right, feature, threshold,
                 leaf_class, cardinality, tree_depth=None, leaf_value=None, value_scale=1.0, value_bias=0.0):
        self.n_features = int(n_features)
        self.n_classes = int(n_classes)
        self.node_begin = np.ascontiguousarray(node_begin, dtype=np.int64)
        self.left = np.ascontiguousarray(left, dtype=np.int32)
        self.right = np.ascontiguousarray(right, dtype=np.int32)
        self.feature = np.ascontiguousarray(feature, dtype=np.int32)
        self.threshold = np.ascontiguousarray(threshold, dtype=np.float32)
        self.leaf_class = np.ascontiguousarray(leaf_class, dtype=np.int32)
        self.cardinality = np.ascontiguousarray(cardinality, dtype=np.int64)
        if tree_depth is None:
            tree_depth = np.zeros(self.n_trees, dtype=np.int32)
        self.tree_depth = np.ascontiguousarray(tree_depth, dtype=np.int32)
        self.leaf_value = None if leaf_value is None else np.ascontiguousarray(leaf_value, dtype=np.float32)
        self.value_scale = float(value_scale)
        self.value_bias = float(value_bias)

    @property
    def n_trees(self) -> int:
        return len(self.node_begin) - 1

    @property
    def n_nodes(self) -> int:
        return int(self.node_begin[-1])

    def tree(self, t: int) -> dict:
        a, b = int(self.node_begin[t]), int(self.node_begin[t + 1])
        return dict(left=self.left[a:b], right=self.right[a:b], feature=self.feature[a:b],
                    threshold=self.threshold[a:b], leaf_class=self.leaf_class[a:b],
                    cardinality=self.cardinality[a:b])

    def internal_nodes_per_tree(self) -> np.ndarray:
        per = np.add.reduceat((self.left >= 0).astype(np.int64), self.node_begin[:-1]) \
            if self.n_nodes else np.zeros(self.n_trees, np.int64)
        return per

    _FIELDS = ("node_begin", "left", "right", "feature", "threshold", "leaf_class", "cardinality", "tree_depth")

    def save(self, path: str) -> None:
        os.makedirs(path, exist_ok=True)
        for k in self._FIELDS:
            np.save(os.path.join(path, k + ".npy"), getattr(self, k))
        if self.leaf_value is not None:
            np.save(os.path.join(path, "leaf_value.npy"), self.leaf_value)
        with open(os.path.join(path, "meta.json"), "w") as f:
            json.dump({"n_features": self.n_features, "n_classes": self.n_classes,
                       "value_scale": self.value_scale, "value_bias": self.value_bias}, f)

    @classmethod
    def load(cls, path: str) -> "Forest":
        with open(os.path.join(path, "meta.json")) as f:
            meta = json.load(f)
        arrs = {k: np.load(os.path.join(path, k + ".npy")) for k in cls._FIELDS}
        lv = os.path.join(path, "leaf_value.npy")
        if os.path.exists(lv):
            arrs["leaf_value"] = np.load(lv)
        return cls(meta["n_features"], meta["n_classes"], value_scale=meta.get("value_scale", 1.0),
                   value_bias=meta.get("value_bias", 0.0), **arrs)


def train_forest(X: np.ndarray, y: np.ndarray, n_classes: int, n_trees: int, mtry: int | None = None,
                 seed: int = 0, threads: int | None = None) -> Forest:
    """Train a CART random forest grown to purity (see datagen.c for every rule)."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.int32)
    n, d = X.shape
    if mtry is None:
        mtry = max(1, int(math.isqrt(d)))
    L = lib()
    h = L.dg_train(_ptr(X), _ptr(y), n, d, n_classes, n_trees, mtry, seed, threads or n_threads())
    if not h:
        raise RuntimeError("dg_train failed (bad arguments or out of memory)")
    try:
        T = L.dg_forest_n_trees(h)
        m = L.dg_forest_total_nodes(h)
        node_begin = np.empty(T + 1, np.int64)
        left = np.empty(m, np.int32)
        right = np.empty(m, np.int32)
        feature = np.empty(m, np.int32)
        threshold = np.empty(m, np.float32)
        leaf_class = np.empty(m, np.int32)
        card = np.empty(m, np.int64)
        depth = np.empty(T, np.int32)
        L.dg_forest_export(h, _ptr(node_begin), _ptr(left), _ptr(right), _ptr(feature), _ptr(threshold),
                           _ptr(leaf_class), _ptr(card), _ptr(depth))
    finally:
        L.dg_forest_free(h)
    return Forest(d, n_classes, node_begin, left, right, feature, threshold, leaf_class, card, depth)


def train_regression(X: np.ndarray, y: np.ndarray, n_trees: int, mtry: int | None = None, max_depth: int = 0,
                     min_leaf: int = 1, eta: float = 0.0, seed: int = 0, threads: int | None = None) -> Forest:
    """A regression forest (eta == 0: bootstrap, mean of the trees) or a
    boosted ensemble (eta > 0: F_0 + sum of the trees); see datagen.c."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.float64)
    n, d = X.shape
    if mtry is None:
        mtry = max(1, d // 3)
    L = lib()
    base = ctypes.c_double(0.0)
    h = L.dg_train_regression(_ptr(X), _ptr(y), n, d, n_trees, mtry, max_depth, min_leaf, eta, seed,
                              ctypes.addressof(base), threads or n_threads())
    if not h:
        raise RuntimeError("dg_train_regression failed (bad arguments or out of memory)")
    try:
        T = L.dg_forest_n_trees(h)
        m = L.dg_forest_total_nodes(h)
        node_begin = np.empty(T + 1, np.int64)
        left = np.empty(m, np.int32)
        right = np.empty(m, np.int32)
        feature = np.empty(m, np.int32)
        threshold = np.empty(m, np.float32)
        leaf_class = np.empty(m, np.int32)
        card = np.empty(m, np.int64)
        depth = np.empty(T, np.int32)
        value = np.empty(m, np.float32)
        L.dg_forest_export(h, _ptr(node_begin), _ptr(left), _ptr(right), _ptr(feature), _ptr(threshold),
                           _ptr(leaf_class), _ptr(card), _ptr(depth))
        L.dg_forest_export_values(h, _ptr(value))
    finally:
        L.dg_forest_free(h)
    scale = 1.0 / T if eta == 0.0 else 1.0
    return Forest(d, 1, node_begin, left, right, feature, threshold, leaf_class, card, depth,
                  leaf_value=value, value_scale=scale, value_bias=base.value)


def bootstrap_weights(seed: int, tree: int, n: int) -> np.ndarray:
    w = np.empty(n, np.int64)
    lib().dg_bootstrap_weights(seed, tree, n, _ptr(w))
    return w


# ------------------------------------------------------------- workloads

# Batched workload: 8 forests (tree count, features, classes); training rows
# log-spaced over 20k..200k.
BATCHED_SPECS = [(32, 8, 2), (64, 12, 3), (96, 20, 5), (128, 32, 8),
                 (192, 50, 12), (256, 80, 20), (384, 128, 32), (512, 200, 50)]


def _batched_train_rows(k: int) -> int:
    return int(round(20000 * (10.0 ** (k / 7.0))))


RECIPES = {
    "tiny": dict(kind="mixture", seed=0, C=4, d=16, n_train=2000, n_test=10000, T=16, mtry=4),
    "image": dict(kind="image", seed=2, C=10, d=784, n_train=60000, n_test=1000000, T=128, mtry=28),
    "hbm": dict(kind="logistic", seed=3, C=2, d=28, n_train=500000, n_test=4000000, T=256, mtry=5,
                scale=HBM_LOGIT_SCALE),
    "wide": dict(kind="mixture", seed=5, C=50, d=100, n_train=50000, n_test=100000, T=64, mtry=10),
    "regress": dict(kind="regression", seed=6, C=1, d=28, n_train=200000, n_test=4000000, T=128, mtry=9,
                    max_depth=0, min_leaf=5, eta=0.0, noise=1.0),
    "boosted": dict(kind="regression", seed=7, C=1, d=28, n_train=30000, n_test=4000000, T=256, mtry=28,
                    max_depth=6, min_leaf=1, eta=0.1, noise=1.0),
}
for _k, (_T, _d, _C) in enumerate(BATCHED_SPECS):
    RECIPES[f"batched{_k}"] = dict(kind="mixture", seed=400 + _k, C=_C, d=_d, n_train=_batched_train_rows(_k),
                                   n_test=100000, T=_T, mtry=max(1, math.isqrt(_d)))

_RECIPE_VERSION = 1


def _recipe_key(name: str, recipe: dict) -> str:
    blob = json.dumps({"v": _RECIPE_VERSION, "name": name, **recipe}, sort_keys=True).encode()
    return f"{name}-{hashlib.sha1(blob).hexdigest()[:12]}"


def rows(name: str, split: int, n: int | None = None):
    """Observation rows of a workload; split 0 = training, 1 = test."""
    r = RECIPES[name]
    if n is None:
        n = r["n_train"] if split == 0 else r["n_test"]
    if r["kind"] == "mixture":
        return gen_mixture(r["seed"], r["C"], r["d"], n, split)
    if r["kind"] == "image":
        return gen_image(r["seed"], n, split)
    if r["kind"] == "logistic":
        return gen_logistic(r["seed"], n, split, r["scale"])
    if r["kind"] == "regression":
        return gen_regression(r["seed"], n, split, 1.0, r["noise"])
    raise KeyError(r["kind"])


def forest(name: str, use_cache: bool = True) -> Forest:
    """The trained forest of a workload, cached on disk under FP_CACHE_DIR."""
    r = RECIPES[name]
    path = os.path.join(CACHE_DIR, _recipe_key(name, r))
    if use_cache and os.path.exists(os.path.join(path, "meta.json")):
        return Forest.load(path)
    X, y = rows(name, 0)
    if r["kind"] == "regression":
        F = train_regression(X, y, r["T"], r["mtry"], max_depth=r["max_depth"], min_leaf=r["min_leaf"],
                             eta=r["eta"], seed=r["seed"])
    else:
        F = train_forest(X, y, r["C"], r["T"], r["mtry"], seed=r["seed"])
    if use_cache:
        tmp = path + f".tmp{os.getpid()}"
        F.save(tmp)
        try:
            os.replace(tmp, path)
        except OSError:
            pass
    return F


def test_rows(name: str, n: int | None = None):
    return rows(name, 1, n)


def batch_sizes(seed: int = 4, k: int = 8, lo: int = 1, hi: int = 100000) -> list[int]:
    """Per-forest batch sizes of the batched workload: round(exp(U[ln lo, ln hi]))."""
    rng = np.random.Generator(np.random.PCG64(seed))
    u = rng.uniform(math.log(lo), math.log(hi), size=k)
    return [int(min(hi, max(lo, round(math.exp(v))))) for v in u]
