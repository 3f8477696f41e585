"""The CPU oracle -- TEST INFRASTRUCTURE ONLY.

A plain, slow, obviously correct C implementation of forest classification
(Section III of the paper) and of the paper's own layouts (Section III-A:
BF, DF, DF-, Stat, Bin; Section III-B: Bin+ round-robin evaluation), and the
plain definition of forests with real leaf values (regression and boosted
trees, the other forest variants the paper names): the leaf walk above, then
bias + scale * the fp64 sum of the reached leaves' values.  Only the
tests, the smoke check and the benchmark's CPU-baseline leg may use it; the
GPU library never imports it and shares no code with it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()

BF, DF, DFM, STAT, BIN = 0, 1, 2, 3, 4
LAYOUT_NAMES = {BF: "BF", DF: "DF", DFM: "DF-", STAT: "Stat", BIN: "Bin"}


def build(force: bool = False) -> str:
    """Compile oracle.c (gcc, OpenMP, IEEE comparisons: no fast-math)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
            L.or_predict.argtypes = [i32, i32, i32, P, P, P, P, P, P, P, i64, i32, P, P, P, P]
            L.or_predict.restype = ctypes.c_int
            L.or_layout_build.argtypes = [i32, i32, i32, P, P, P, P, P, P, P, i32, i32]
            L.or_layout_build.restype = P
            L.or_layout_free.argtypes = [P]
            L.or_layout_free.restype = None
            L.or_layout_n_nodes.argtypes = [P]
            L.or_layout_n_nodes.restype = i64
            L.or_layout_export.argtypes = [P] * 9
            L.or_layout_export.restype = None
            L.or_layout_predict.argtypes = [P, i32, P, i64, i32, P, P, P]
            L.or_layout_predict.restype = ctypes.c_int
            L.or_eu_stat.argtypes = [ctypes.c_double]
            L.or_eu_stat.restype = ctypes.c_double
            L.or_forest_stats.argtypes = [i32, P, P, P, P, P]
            L.or_forest_stats.restype = None
            _lib = L
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"], "oracle inputs must be C-contiguous"
    return a.ctypes.data


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def predict(forest, X: np.ndarray, leaves: bool = True, votes: bool = True, classes: bool = True,
            threads: int = 1):
    """Plain pointer-per-tree classification.

    Returns dict(leaf [n][T] int32, votes [n][C] uint32, cls [n] int32, visits int).
    """
    X = np.ascontiguousarray(X, dtype=np.float32)
    n = X.shape[0]
    if X.ndim != 2 or X.shape[1] != forest.n_features:
        raise ValueError("X must be [n][n_features]")
    T, C = forest.n_trees, forest.n_classes
    out_leaf = np.empty((n, T), np.int32) if leaves else None
    out_votes = np.empty((n, C), np.uint32) if votes else None
    out_cls = np.empty(n, np.int32) if classes else None
    visits = ctypes.c_int64(0)
    rc = lib().or_predict(T, forest.n_features, C, _p(forest.node_begin), _p(forest.left), _p(forest.right),
                          _p(forest.feature), _p(forest.threshold), _p(forest.leaf_class), _p(X), n, threads,
                          _p(out_leaf), _p(out_votes), _p(out_cls), ctypes.byref(visits))
    if rc != 0:
        raise RuntimeError(f"or_predict failed: {rc}")
    return dict(leaf=out_leaf, votes=out_votes, cls=out_cls, visits=int(visits.value))


def predict_values(forest, X: np.ndarray, threads: int = 1):
    """Forests with leaf values: out = bias + scale * sum over trees of the
    value of the leaf reached (every term exact in fp64, summed in fp64).

    Returns dict(leaf [n][T], sum [n] fp64, abs [n] fp64 = sum of |value|,
    out [n] fp64, visits int)."""
    if forest.leaf_value is None:
        raise ValueError("the forest has no leaf values")
    r = predict(forest, X, leaves=True, votes=False, classes=False, threads=threads)
    leaf = r["leaf"]
    vals = forest.leaf_value[forest.node_begin[:-1][None, :] + leaf].astype(np.float64)
    s = vals.sum(axis=1)
    return dict(leaf=leaf, sum=s, abs=np.abs(vals).sum(axis=1),
                out=forest.value_bias + forest.value_scale * s, visits=r["visits"])


def value_tolerance(forest, abs_sum: np.ndarray) -> np.ndarray:
    """Per-row bound on |float32 result - exact result| for a float32
    evaluation that adds the T leaf values in any order and then computes
    bias + scale * sum: recursive summation in any order is within
    (T-1) u / (1 - (T-1) u) * sum|v| of the exact sum (u = 2^-24, Higham,
    Accuracy and Stability of Numerical Algorithms, Sec. 4.2), and the
    final multiply-add adds at most two roundings; (T + 2) u covers both
    with a margin."""
    u = 2.0 ** -24
    T = forest.n_trees
    return (T + 2) * u * (abs(forest.value_bias) + abs(forest.value_scale) * abs_sum) * 1.01 + 1e-30


class Layout:
    """One of the paper's layouts (BF, DF, DF-, Stat, Bin) built by the oracle."""

    def __init__(self, forest, kind: int, bin_size: int = 0, depth: int = 0):
        self.forest = forest
        self.kind = kind
        self.bin_size = bin_size
        self.depth = depth
        f = forest
        self._h = lib().or_layout_build(kind, f.n_trees, f.n_classes, _p(f.node_begin), _p(f.left), _p(f.right),
                                        _p(f.feature), _p(f.threshold), _p(f.leaf_class), _p(f.cardinality),
                                        bin_size, depth)
        if not self._h:
            raise RuntimeError("or_layout_build failed")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().or_layout_free(h)
            self._h = None

    def arrays(self) -> dict:
        m = lib().or_layout_n_nodes(self._h)
        out = dict(feature=np.empty(m, np.int32), threshold=np.empty(m, np.float32), child0=np.empty(m, np.int32),
                   child1=np.empty(m, np.int32), cls=np.empty(m, np.int32), orig=np.empty(m, np.int32),
                   tree=np.empty(m, np.int32), root=np.empty(self.forest.n_trees, np.int32))
        lib().or_layout_export(self._h, *[_p(out[k]) for k in ("feature", "threshold", "child0", "child1", "cls",
                                                               "orig", "tree", "root")])
        return out

    def predict(self, X: np.ndarray, threads: int = 1):
        """Per (observation, tree): class, and the leaf as (last internal node, direction)."""
        X = np.ascontiguousarray(X, dtype=np.float32)
        n, T = X.shape[0], self.forest.n_trees
        cls = np.empty((n, T), np.int32)
        par = np.empty((n, T), np.int32)
        d = np.empty((n, T), np.int8)
        rc = lib().or_layout_predict(self._h, self.forest.n_features, _p(X), n, threads, _p(cls), _p(par), _p(d))
        if rc != 0:
            raise RuntimeError("or_layout_predict failed")
        return dict(cls=cls, parent=par, dir=d)


def leaf_from_parent(forest, parent: np.ndarray, direction: np.ndarray) -> np.ndarray:
    """Tree-local leaf ids from (last internal node, direction) pairs."""
    n, T = parent.shape
    out = np.empty((n, T), np.int32)
    for t in range(T):
        b = int(forest.node_begin[t])
        p = parent[:, t]
        leaf = np.where(direction[:, t] == 1, forest.right[b + np.maximum(p, 0)], forest.left[b + np.maximum(p, 0)])
        out[:, t] = np.where(p < 0, 0, leaf)
    return out


def eu_stat(bias: float) -> float:
    return lib().or_eu_stat(bias)


def forest_stats(forest) -> dict:
    out = np.zeros(3, np.float64)
    lib().or_forest_stats(forest.n_trees, _p(forest.node_begin), _p(forest.left), _p(forest.right),
                          _p(forest.cardinality), _p(out))
    return dict(mean_internal=float(out[0]), max_depth=int(out[1]), mean_bias=float(out[2]))
