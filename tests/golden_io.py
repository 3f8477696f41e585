"""Reader for the hand-written forest fixtures under tests/golden/."""
from __future__ import annotations

import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _f(tok: str) -> float:
    return float(tok)  # accepts inf, -inf, nan, -0.0


def load(name: str):
    """Returns (Forest, X, expected) where expected has leaf [n][T], votes [n][C],
    cls [n] and visits [n] (internal nodes evaluated per observation)."""
    import datagen
    path = os.path.join(GOLDEN, name)
    lines = [ln.split("#", 1)[0].strip() for ln in open(path)]
    lines = [ln for ln in lines if ln]
    it = iter(lines)
    head = next(it).split()
    assert head[0] == "forest"
    kv = dict(t.split("=") for t in head[1:])
    nf, nc = int(kv["n_features"]), int(kv["n_classes"])
    trees, rows = [], []
    cur = None
    for ln in it:
        if ln == "tree":
            cur = []
            continue
        if ln == "end":
            trees.append(cur)
            cur = None
            continue
        if ln == "rows":
            break
        tok = ln.split()
        cur.append((int(tok[0]), int(tok[1]), int(tok[2]), int(tok[3]), np.float32(_f(tok[4])), int(tok[5]),
                    int(tok[6]) if len(tok) > 6 else 1))
    for ln in it:
        x, rest = ln.split("|", 1)
        parts = [p.split() for p in rest.split("|")]
        rows.append(([np.float32(_f(t)) for t in x.split()], [int(t) for t in parts[0]],
                     [int(t) for t in parts[1]], int(parts[2][0]), int(parts[3][0])))
    node_begin = [0]
    L, R, Fe, Th, Cl, Ca = [], [], [], [], [], []
    for tr in trees:
        tr = sorted(tr)
        assert [r[0] for r in tr] == list(range(len(tr)))
        for (_, l, r, f, t, c, card) in tr:
            L.append(l); R.append(r); Fe.append(f); Th.append(t); Cl.append(c); Ca.append(card)
        node_begin.append(node_begin[-1] + len(tr))
    forest = datagen.Forest(nf, nc, node_begin, L, R, Fe, np.array(Th, np.float32), Cl, Ca)
    X = np.array([r[0] for r in rows], np.float32).reshape(len(rows), nf)
    expected = dict(leaf=np.array([r[1] for r in rows], np.int32), votes=np.array([r[2] for r in rows], np.uint32),
                    cls=np.array([r[3] for r in rows], np.int32), visits=np.array([r[4] for r in rows], np.int64))
    return forest, X, expected


def load_values(name: str):
    """Returns (Forest with leaf values, X, expected) for a value fixture;
    expected has leaf [n][T], sum [n] and out [n]."""
    import datagen
    path = os.path.join(GOLDEN, name)
    lines = [ln.split("#", 1)[0].strip() for ln in open(path)]
    lines = [ln for ln in lines if ln]
    it = iter(lines)
    head = next(it).split()
    assert head[0] == "forest"
    kv = dict(t.split("=") for t in head[1:])
    nf = int(kv["n_features"])
    trees, rows, cur = [], [], None
    for ln in it:
        if ln == "tree":
            cur = []
            continue
        if ln == "end":
            trees.append(cur)
            continue
        if ln == "rows":
            break
        tok = ln.split()
        cur.append((int(tok[0]), int(tok[1]), int(tok[2]), int(tok[3]), np.float32(_f(tok[4])),
                    np.float32(_f(tok[5]))))
    for ln in it:
        x, rest = ln.split("|", 1)
        parts = [p.split() for p in rest.split("|")]
        rows.append(([np.float32(_f(t)) for t in x.split()], [int(t) for t in parts[0]], _f(parts[1][0]),
                     _f(parts[2][0])))
    node_begin = [0]
    L, R, Fe, Th, V = [], [], [], [], []
    for tr in trees:
        tr = sorted(tr)
        assert [r[0] for r in tr] == list(range(len(tr)))
        for (_, l, r, f, t, v) in tr:
            L.append(l); R.append(r); Fe.append(f); Th.append(t); V.append(v)
        node_begin.append(node_begin[-1] + len(tr))
    L = np.array(L, np.int32)
    forest = datagen.Forest(nf, 1, node_begin, L, R, Fe, np.array(Th, np.float32), np.where(L < 0, 0, -1),
                            np.ones(len(L), np.int64), leaf_value=np.array(V, np.float32),
                            value_scale=float(kv["scale"]), value_bias=float(kv["bias"]))
    X = np.array([r[0] for r in rows], np.float32).reshape(len(rows), nf)
    expected = dict(leaf=np.array([r[1] for r in rows], np.int32), sum=np.array([r[2] for r in rows]),
                    out=np.array([r[3] for r in rows]))
    return forest, X, expected
