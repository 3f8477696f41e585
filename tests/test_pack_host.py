"""CPU tests of the C-ABI library: it loads, exports every declared symbol,
validates forests, and packs records that decode (on the host, by
packed_decode.py) to the oracle's leaves.  No kernel is launched."""
import ctypes
import os
import re

import numpy as np
import pytest

import datagen
import oracle
import paper_1806_07300_gb300 as fp
from golden_io import load
from packed_decode import Image, LEAF, thr_key

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))



# (deep_levels, deep_format): two-level super-nodes, three-level of format 1
# (full keys first) and of format 2 (remapped key prefixes in every slot)
DEEP_KINDS = [(2, 0), (3, 1), (3, 2)]

def declared_symbols():
    src = open(os.path.join(ROOT, "include", "forest_pack.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fp_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = fp.lib()
    decl = declared_symbols()
    assert decl, "no declarations found"
    for name in decl:
        assert hasattr(L, name), f"{name} is declared in include/forest_pack.h but not exported"
    assert sorted(fp.EXPORTS) == decl


def test_binding_has_no_cpu_path():
    """The binding forwards to the library only; it never imports the oracle."""
    src = open(os.path.join(ROOT, "paper_1806_07300_gb300", "__init__.py")).read()
    assert "oracle" not in src.replace("never imports the oracle", "")


@pytest.mark.parametrize("name", ["stump_split.txt", "chain_full.txt"])
@pytest.mark.parametrize("B,d,sel", [(1, 0, 3), (2, 0, 3), (2, 1, 3), (3, 2, 3), (1, 5, 3), (1, 0, 1), (2, 1, 1),
                                     (3, 4, 1), (1, 1, 2), (2, 3, 2)])
@pytest.mark.parametrize("dl,fmt", DEEP_KINDS)
def test_packed_records_decode_to_fixture_leaves(name, B, d, sel, dl, fmt):
    forest, X, exp = load(name)
    pk = fp.fp_pack_forest(forest, bin_size=B, interleave_depth=d, head_select=sel, deep_levels=dl, deep_format=fmt)
    leaf, cls = Image(pk.image()).walk(X)
    np.testing.assert_array_equal(leaf, exp["leaf"])


@pytest.mark.parametrize("B,d,sel", [(16, 4, 3), (5, 0, 3), (1, 2, 3), (7, 7, 3), (16, 4, 1), (3, 0, 1), (1, 9, 1),
                                     (1, 11, 1), (3, 1, 2), (4, 9, 2), (1, 11, 2), (16, 5, 2)])
@pytest.mark.parametrize("dl,fmt", DEEP_KINDS)
def test_packed_records_decode_to_oracle_leaves(tiny_forest, tiny_rows, B, d, sel, dl, fmt):
    X, _ = tiny_rows
    ref = oracle.predict(tiny_forest, X[:3000])
    pk = fp.fp_pack_forest(tiny_forest, bin_size=B, interleave_depth=d, head_select=sel, deep_levels=dl,
                           deep_format=fmt)
    assert pk.info()["deep_levels"] == dl and pk.info()["deep_format"] == fmt
    leaf, cls = Image(pk.image()).walk(X[:3000])
    np.testing.assert_array_equal(leaf, ref["leaf"])
    np.testing.assert_array_equal(cls, tiny_forest.leaf_class[tiny_forest.node_begin[:-1][None, :] + ref["leaf"]])


def _head_nodes(forest, t, im):
    """Node ids of tree t's head, in rank order, recovered by walking the block."""
    B = im.h["bin_size"]
    b, k = t // B, t % B
    thr, meta, exits, par = im.head(b)
    tr = forest.tree(t)
    if tr["left"][0] < 0:
        return [], {}
    rank_node = {0: 0}
    exit_node = {}
    nr = int(im.bins[b]["nranks"])
    for r in range(meta.shape[0]):
        if r not in rank_node:
            continue
        v = rank_node[r]
        m = int(meta[r, k])
        assert m >> 22 == tr["feature"][v] and thr[r, k] == im.word(tr["threshold"][v])
        for c, tgt in ((int(tr["left"][v]), m & 2047), (int(tr["right"][v]), (m >> 11) & 2047)):
            if tgt < nr:
                assert tr["left"][c] >= 0, "a head target is an internal node"
                rank_node[tgt] = c
            else:
                exit_node[tgt - nr] = c
    ranks = sorted(rank_node)
    assert ranks == list(range(len(ranks))), "head ranks are dense"
    return [rank_node[r] for r in ranks], exit_node


def _super_roots(forest, t, im, exit_node):
    """Global super-node index -> the tree-local node it is rooted at."""
    b, k = t // im.h["bin_size"], t % im.h["bin_size"]
    _, _, exits, _ = im.head(b)
    tr = forest.tree(t)
    roots = {}
    stack = [(int(exits[e, k]), v) for e, v in exit_node.items() if not int(exits[e, k]) & LEAF]
    while stack:
        i, v = stack.pop()
        roots[i] = v
        l, r = int(tr["left"][v]), int(tr["right"][v])
        ex = [l, l] if tr["left"][l] < 0 else [int(tr["left"][l]), int(tr["right"][l])]
        ex += [r, r] if tr["left"][r] < 0 else [int(tr["left"][r]), int(tr["right"][r])]
        for q in range(4):
            ref = int(im.sw[i, 4 + q])
            if not ref & LEAF:
                stack.append((ref, ex[q]))
    return roots


@pytest.mark.parametrize("d", [0, 2, 5])
def test_head_is_top_cardinality_and_stat_ranked(tiny_forest, d):
    """A tree's head holds its 2^(d+1)-1 internal nodes of highest training
    cardinality (ties: shallower first), the most popular paths of
    Section III-A; within the head the first child visited sits at the next
    rank and is the child of larger cardinality (Stat)."""
    f = tiny_forest
    im = Image(fp.fp_pack_forest(f, bin_size=3, interleave_depth=d, head_select=3).image())
    K = 2 ** (d + 1) - 1
    for t in range(f.n_trees):
        tr = f.tree(t)
        head, _ = _head_nodes(f, t, im)
        depth = {0: 0}
        for v in range(len(tr["left"])):
            if tr["left"][v] >= 0:
                depth[int(tr["left"][v])] = depth[v] + 1
                depth[int(tr["right"][v])] = depth[v] + 1
        internal = [v for v in range(len(tr["left"])) if tr["left"][v] >= 0]
        want = sorted(internal, key=lambda v: (-int(tr["cardinality"][v]), depth[v], v))[:K]
        assert sorted(head) == sorted(want)
        for i, v in enumerate(head[:-1]):
            l, r = int(tr["left"][v]), int(tr["right"][v])
            if head[i + 1] in (l, r):  # depth-first: the first child visited is the more popular one
                other = r if head[i + 1] == l else l
                if other in head:
                    assert tr["cardinality"][head[i + 1]] >= tr["cardinality"][other]


@pytest.mark.parametrize("d", [0, 3, 6])
def test_head_select_levels(tiny_forest, d):
    """Level heads (the Bin layout's interleaved levels 0..d): slot s of tree k
    holds the node at breadth-first position s (children 2s+1, 2s+2); below a
    leaf the slots are dummies and every exit names that leaf; exit e is the
    node at level d+1, position e."""
    f = tiny_forest
    im = Image(fp.fp_pack_forest(f, bin_size=5, interleave_depth=d, head_select=1).image())
    S = 2 ** (d + 1) - 1
    for t in range(f.n_trees):
        tr = f.tree(t)
        thr, meta, exits, par = im.head(t // 5)
        k = t % 5
        assert thr.shape[0] == S and exits.shape[0] == S + 1
        slot = {0: 0}  # slot -> node (a leaf marks a dummy slot)
        for s in range(S):
            v = slot[s]
            leaf = tr["left"][v] < 0
            if not leaf:
                assert meta[s, k] >> 22 == tr["feature"][v] and thr[s, k] == im.word(tr["threshold"][v])
                assert meta[s, k] & ((1 << 22) - 1) == 0
            kids = (v, v) if leaf else (int(tr["left"][v]), int(tr["right"][v]))
            for q, c in enumerate(kids):
                slot[2 * s + 1 + q] = c
        for e in range(S + 1):
            v = slot[S + e]
            ref = int(exits[e, k])
            if tr["left"][v] < 0:
                assert ref == LEAF | int(tr["leaf_class"][v]) and par[e, k] == v
            else:
                assert not ref & LEAF and par[e, k] == -1
                # the first word of either kind of super-node is its root's full key
                assert im.sw[ref, 0] == im.word(tr["threshold"][v]), "the exit roots the super-node of its node"


def test_stat_order_in_super_nodes(tiny_forest):
    """Below the head each super-node is followed by its most frequently
    reached child super-node (Section III-A, Stat), and every internal node
    lies in the head or in exactly one super-node."""
    f = tiny_forest
    pk = fp.fp_pack_forest(f, bin_size=4, interleave_depth=2, head_select=3, deep_levels=2)
    im = Image(pk.image())
    total = 0
    for t in range(f.n_trees):
        tr = f.tree(t)
        head, exit_node = _head_nodes(f, t, im)
        roots = _super_roots(f, t, im, exit_node)
        base = int(im.tree_base[t])
        end = int(im.tree_base[t + 1]) if t + 1 < f.n_trees else im.sw.shape[0]
        assert sorted(roots) == list(range(base, end)), "a tree's super-nodes are one contiguous region"
        for i, v in roots.items():
            kids = sorted({int(im.sw[i, 4 + q]) for q in range(4)} - {c for c in
                          (int(im.sw[i, 4 + q]) for q in range(4)) if c & LEAF})
            if kids:
                card = {c: int(tr["cardinality"][roots[c]]) for c in kids}
                assert i + 1 in kids and card[i + 1] == max(card.values()), "hottest child super-node follows"
        covered = set(head)
        for v in roots.values():
            covered.add(v)
            for c in (int(tr["left"][v]), int(tr["right"][v])):
                if tr["left"][c] >= 0:
                    covered.add(c)
        total += len(covered)
    assert total == pk.info()["n_internal"]


def test_head_interleaving_roots_contiguous(tiny_forest):
    """Fig. 2 caption: the roots of a bin's trees sit side by side (rank 0),
    then the trees' next nodes, rank by rank."""
    f = tiny_forest
    im = Image(fp.fp_pack_forest(f, bin_size=8, interleave_depth=0, head_select=3).image())
    for b in range(im.h["n_bins"]):
        thr, meta, exits, par = im.head(b)
        assert meta.shape[0] == 1  # d = 0: one node (the root) per tree
        first = int(im.bins[b]["first_tree"])
        for k in range(int(im.bins[b]["width"])):
            root = int(f.node_begin[first + k])
            assert meta[0, k] >> 22 == f.feature[root]
            assert thr[0, k] == im.word(f.threshold[root])


def test_pack_info_sizes(tiny_forest):
    pk = fp.fp_pack_forest(tiny_forest, bin_size=16, interleave_depth=2)
    info = pk.info()
    assert info["n_internal"] == int((tiny_forest.left >= 0).sum())
    assert info["deep_bytes"] == 32 * info["n_super"]
    assert info["n_bins"] == 1 and info["passes"] == 1
    assert info["bin_buffers"] == 3
    assert fp.fp_pack_forest(tiny_forest, bin_buffers=2).info()["bin_buffers"] == 2
    # 16 features and 4 classes take 4 + 2 * 2 bits: three levels by default
    assert info["deep_levels"] == 3
    assert fp.fp_pack_forest(tiny_forest, deep_levels=2).info()["deep_levels"] == 2


def test_passes_split_by_budget(tiny_forest):
    pk = fp.fp_pack_forest(tiny_forest, bin_size=2, interleave_depth=1, pass_bytes=2048)
    info = pk.info()
    assert info["passes"] > 1
    im = Image(pk.image())
    pb = im.passes
    assert pb[0]["bin_begin"] == 0 and pb[-1]["bin_end"] == info["n_bins"]
    assert np.all(pb["bin_begin"][1:] == pb["bin_end"][:-1])


def _bad_forest(**changes):
    forest, _, _ = load("chain_full.txt")
    for k, v in changes.items():
        arr = getattr(forest, k).copy()
        for idx, val in v:
            arr[idx] = val
        setattr(forest, k, arr)
    return forest


@pytest.mark.parametrize("changes", [
    dict(left=[(0, 5)], right=[(0, 5)]),          # both children the same node
    dict(left=[(2, 0)]),                          # cycle back to the root
    dict(leaf_class=[(1, 9)]),                    # class out of range
    dict(feature=[(0, 3)]),                       # feature out of range
    dict(right=[(1, 3)]),                         # leaf with a right child
    dict(left=[(4, 99)]),                         # child id out of range
])
def test_malformed_forests_rejected(changes):
    forest = _bad_forest(**changes)
    with pytest.raises(fp.FPError) as ei:
        fp.fp_pack_forest(forest)
    assert ei.value.code == fp.FP_EINVAL


def test_unsupported_sizes_rejected():
    forest, _, _ = load("stump_split.txt")
    forest.n_features = 2000
    with pytest.raises(fp.FPError) as ei:
        fp.fp_pack_forest(forest)
    assert ei.value.code == fp.FP_EUNSUPPORTED


@pytest.mark.parametrize("kw", [dict(bin_size=-1), dict(interleave_depth=12), dict(interleave_depth=12, head_select=1),
                                dict(obs_tile=33), dict(warps_per_cta=40),
                                dict(bin_buffers=1), dict(bin_buffers=4), dict(head_select=2, interleave_depth=8),
                                dict(head_select=4), dict(head_select=3, interleave_depth=10),
                                dict(deep_levels=1), dict(deep_levels=4)])
def test_bad_params_rejected(tiny_forest, kw):
    with pytest.raises(fp.FPError) as ei:
        fp.fp_pack_forest(tiny_forest, **kw)
    assert ei.value.code == fp.FP_EINVAL


def test_null_arguments_rejected():
    L = fp.lib()
    assert L.fp_pack_forest(None, None, None) == fp.FP_EINVAL
    assert "NULL" in fp.fp_last_error() or "out" in fp.fp_last_error()
    assert L.fp_upload(None, None, None) == fp.FP_EINVAL
    assert L.fp_predict(None, None, 0, None, None, None) == fp.FP_EINVAL
    L.fp_release(None)
    L.fp_release_packed(None)
    L.fp_plain_release(None)
    # host-buffer calls and the serving runtime check their arguments before any CUDA call
    assert L.fp_predict_host(None, None, 0, None, None, 0, None) == fp.FP_EINVAL
    assert L.fp_predict_values_host(None, None, 0, 1.0, 0.0, None, 0, None) == fp.FP_EINVAL
    out = ctypes.c_void_p()
    assert L.fp_server_create(0, 0, 1024, 0, 0, 0.0, ctypes.byref(out)) == fp.FP_EINVAL   # no slot
    assert L.fp_server_create(0, 2, 0, 0, 0, 0.0, ctypes.byref(out)) == fp.FP_EINVAL     # no rows
    assert L.fp_server_create(0, 2, 1024, -1, 0, 0.0, ctypes.byref(out)) == fp.FP_EINVAL  # negative margin
    assert L.fp_server_create(0, 2, 1024, 0, 0, 0.0, None) == fp.FP_EINVAL
    assert L.fp_server_add_forest(None, None, None) == fp.FP_EINVAL
    assert L.fp_server_start(None) == fp.FP_EINVAL
    assert L.fp_server_submit(None, 0, None, 1, None, None, ctypes.byref(out)) == fp.FP_EINVAL
    assert L.fp_request_wait(None, 0.0) == fp.FP_EINVAL
    assert L.fp_request_latency(None) == -1.0
    assert L.fp_server_stop(None) == fp.FP_EINVAL
    assert L.fp_server_stats(None, None, None) == fp.FP_EINVAL
    assert L.fp_server_set_free_bytes(None, 0) == fp.FP_EINVAL
    L.fp_request_release(None)
    L.fp_server_release(None)


@pytest.mark.parametrize("B,d,sel", [(4, 3, 1), (1, 0, 3), (3, 6, 3), (2, 9, 1), (3, 9, 0)])
@pytest.mark.parametrize("dl,fmt", DEEP_KINDS)
def test_value_forest_records_decode_to_oracle(B, d, sel, dl, fmt):
    """A forest with leaf values: every leaf reference names a value slot
    holding the leaf's value, and the walk reaches the oracle's leaves."""
    import datagen
    X, y = datagen.gen_regression(21, 2000, 0, 1.0, 1.0)
    F = datagen.train_regression(X, y, 6, mtry=9, min_leaf=3, seed=21, threads=4)
    Xt, _ = datagen.gen_regression(21, 1500, 1, 1.0, 1.0)
    ref = oracle.predict_values(F, Xt)
    im = Image(fp.fp_pack_forest(F, bin_size=B, interleave_depth=d, head_select=sel, deep_levels=dl,
                                 deep_format=fmt).image())
    n_leaves = int((F.left < 0).sum())
    assert im.h["values3_base"] == n_leaves
    assert im.h["n_values"] == n_leaves + (8 * im.h["n_super"] if dl == 3 else 0)
    leaf, slot = im.walk(Xt)
    np.testing.assert_array_equal(leaf, ref["leaf"])
    np.testing.assert_array_equal(im.values[slot], F.leaf_value[F.node_begin[:-1][None, :] + ref["leaf"]])


def _kind(forest, **kw):
    i = fp.fp_pack_forest(forest, **kw).info()
    return i["deep_levels"], i["deep_format"]


def test_deep_levels_follow_field_widths():
    """Three-level super-nodes of format 1 hold two features and two classes
    beside the last level's key prefix: by default when those fields take at
    most 16 bits, on request up to 24.  Format 2 holds one feature per slot
    (and the classes in the last level): by default when fb + 2 cb <= 20, on
    request up to 24.  Beyond both, two-level super-nodes."""
    forest, _, _ = load("stump_split.txt")
    assert _kind(forest) == (3, 1)
    assert _kind(forest, deep_format=2) == (3, 2)
    assert _kind(forest, deep_levels=2) == (2, 0)
    forest.n_features, forest.n_classes = 784, 10  # format 1: 28 bits; format 2: 10 + 8
    assert _kind(forest) == (3, 2)
    assert _kind(forest, deep_levels=3) == (3, 2)
    assert _kind(forest, deep_format=1) == (2, 0)  # format 1 asked for by default: does not fit
    with pytest.raises(fp.FPError) as ei:
        fp.fp_pack_forest(forest, deep_levels=3, deep_format=1)
    assert ei.value.code == fp.FP_EUNSUPPORTED
    forest.n_features, forest.n_classes = 100, 30  # format 1: 24 bits, on request; format 2: 7 + 10
    assert _kind(forest) == (3, 2)
    assert _kind(forest, deep_levels=3) == (3, 1)
    forest.n_features, forest.n_classes = 1000, 200  # format 2: 10 + 16 bits
    assert _kind(forest) == (2, 0)
    with pytest.raises(fp.FPError) as ei:
        fp.fp_pack_forest(forest, deep_levels=3)
    assert ei.value.code == fp.FP_EUNSUPPORTED


def test_value_forest_rejects_non_finite_values():
    import datagen
    X, y = datagen.gen_regression(22, 500, 0, 1.0, 1.0)
    F = datagen.train_regression(X, y, 2, mtry=9, min_leaf=3, seed=22, threads=2)
    F.leaf_value = F.leaf_value.copy()
    F.leaf_value[np.flatnonzero(F.left < 0)[3]] = np.inf
    with pytest.raises(fp.FPError) as ei:
        fp.fp_pack_forest(F)
    assert ei.value.code == fp.FP_EINVAL


@pytest.mark.parametrize("dl,fmt", DEEP_KINDS)
@pytest.mark.parametrize("sel", [1, 3])
def test_rows_on_thresholds_decode_to_oracle_leaves(tiny_forest, tiny_rows, dl, fmt, sel):
    """Observations equal to the forest's thresholds (or one float step off),
    and -0, infinities and NaN: the key compares give the oracle's leaves,
    and with three-level super-nodes the key-prefix ties are decided by the
    full keys (many of them occur here)."""
    from edge_rows import rows_on_thresholds
    X = rows_on_thresholds(tiny_forest, tiny_rows[0][:3000], seed=11)
    ref = oracle.predict(tiny_forest, X)
    im = Image(fp.fp_pack_forest(tiny_forest, bin_size=4, interleave_depth=2, head_select=sel,
                                 deep_levels=dl, deep_format=fmt).image())
    leaf, cls = im.walk(X)
    np.testing.assert_array_equal(leaf, ref["leaf"])
    if dl == 3:
        assert im.ties > 100


def test_key_order_matches_float_compare():
    """x <= t exactly when key(x) <= key(t), over values that stress the map:
    signed zeros, subnormals, infinities, neighbours of each other; a NaN x
    goes right of every threshold, and every x goes right of a NaN threshold."""
    from packed_decode import obs_key
    v = np.array([0.0, -0.0, 1e-45, -1e-45, 1.17549435e-38, -1.17549435e-38, 1.0, -1.0, 3.4028235e38,
                  -3.4028235e38, np.inf, -np.inf, 0.5, np.nextafter(np.float32(0.5), np.float32(1)),
                  np.nextafter(np.float32(0.5), np.float32(0))], dtype=np.float32)
    kx, kt = obs_key(v), thr_key(v)
    for i in range(v.size):
        for j in range(v.size):
            assert (kx[i] <= kt[j]) == bool(v[i] <= v[j]), (v[i], v[j])
    nan = np.array([np.nan, -np.nan], dtype=np.float32)
    assert np.all(obs_key(nan)[:, None] > kt[None, :])
    assert np.all(kx[:, None] > thr_key(nan)[None, :])


def test_three_level_super_nodes(tiny_forest):
    """Three-level super-nodes (format in fp_internal.h): seven slots holding
    the node, its children and grandchildren (a leaf carried down as
    dummies); full keys for the first two levels, features, key prefixes and
    exit classes in the last level's words, its full keys in the side table;
    leaf mask and leaf ids of the eight exits, and the children side by side
    in exit order; a super-node whose children have their own children
    expands the most frequently reached one first (Stat); every internal node
    lies in the head or in exactly one super-node."""
    f = tiny_forest
    pk = fp.fp_pack_forest(f, bin_size=4, interleave_depth=1, head_select=1, deep_levels=3)
    im = Image(pk.image())
    fb, cb = im.h["feature_bits"], im.h["class_bits"]
    assert (fb, cb) == (4, 2)
    covered = 0
    for t in range(f.n_trees):
        tr = f.tree(t)
        thr, meta, exits, par = im.head(t // 4)
        k = t % 4
        covered += sum(1 for s in range(thr.shape[0]) if meta[s, k] or thr[s, k])  # head slots that split
        stack = [(int(exits[e, k]), None) for e in range(exits.shape[0]) if not int(exits[e, k]) & LEAF]
        # recover each super-node's root: the head exit's node
        slot = {0: 0}
        for s in range(thr.shape[0]):
            v = slot[s]
            kids = (v, v) if tr["left"][v] < 0 else (int(tr["left"][v]), int(tr["right"][v]))
            slot[2 * s + 1], slot[2 * s + 2] = kids
        todo = [(int(exits[e, k]), slot[thr.shape[0] + e]) for e in range(exits.shape[0])
                if not int(exits[e, k]) & LEAF]
        seen = set()
        while todo:
            g, v = todo.pop()
            assert g not in seen
            seen.add(g)
            w = [int(x) for x in im.sw[g]]
            sl = [v]
            for i in range(3):
                u = sl[i]
                sl += [u, u] if tr["left"][u] < 0 else [int(tr["left"][u]), int(tr["right"][u])]
            ex = []
            for i in range(3, 7):
                u = sl[i]
                ex += [u, u] if tr["left"][u] < 0 else [int(tr["left"][u]), int(tr["right"][u])]
            sh = 2 * fb + 2 * cb
            fm = (1 << fb) - 1
            for i, u in enumerate(sl):
                leaf = tr["left"][u] < 0
                key = 0 if leaf else int(thr_key(tr["threshold"][u]))
                feat = 0 if leaf else int(tr["feature"][u])
                covered += not leaf
                if i < 3:
                    assert w[i] == key and (w[3 + i] >> fb) & fm == feat
                else:
                    assert im.deep_keys[g, i - 3] == key and w[i] >> sh == key >> sh and w[i] & fm == feat
            assert (w[6] >> fb) & fm == 0
            mask = w[7] >> 24
            first = g + (w[7] & 0xFFFFFF)
            rank = 0
            kids = []
            for e, c in enumerate(ex):
                if tr["left"][c] < 0:
                    assert (mask >> e) & 1 and im.deep_leaf[g, e] == c
                    assert (w[3 + e // 2] >> (2 * fb + cb * (e & 1))) & ((1 << cb) - 1) == tr["leaf_class"][c]
                else:
                    assert not (mask >> e) & 1 and im.deep_leaf[g, e] == -1
                    kids.append((first + rank, c))
                    rank += 1
            todo += kids
            # Stat: of the children that have children, the most visited one's block comes first
            firsts = [(int(im.sw[gc, 7]) & 0xFFFFFF and gc + (int(im.sw[gc, 7]) & 0xFFFFFF), c) for gc, c in kids]
            firsts = [(fs, c) for fs, c in firsts if fs]
            if len(firsts) > 1:
                hot = max(firsts, key=lambda z: (int(tr["cardinality"][z[1]]), -z[0]))
                assert hot[0] == min(fs for fs, _ in firsts)
    assert covered == pk.info()["n_internal"]


def test_short_key_prefixes_decode_to_oracle_leaves(tiny_forest, tiny_rows):
    """The tiny forest declared with 100 features: 7 feature bits twice and 2
    class bits twice leave a 14-bit key prefix in the last level of each
    three-level super-node, so many compares tie and the full keys decide."""
    from edge_rows import rows_on_thresholds
    f = datagen.Forest(100, tiny_forest.n_classes, tiny_forest.node_begin, tiny_forest.left, tiny_forest.right,
                       tiny_forest.feature, tiny_forest.threshold, tiny_forest.leaf_class, tiny_forest.cardinality)
    X = np.zeros((3000, 100), np.float32)
    X[:, :16] = rows_on_thresholds(tiny_forest, tiny_rows[0][:3000], seed=14)
    ref = oracle.predict(f, X)
    im = Image(fp.fp_pack_forest(f, bin_size=4, interleave_depth=2, head_select=1, deep_levels=3).image())
    assert im.h["feature_bits"] == 7
    leaf, _ = im.walk(X)
    np.testing.assert_array_equal(leaf, ref["leaf"])
    assert im.ties > 300


def _remap_of(im):
    return lambda k: int(im.remap(np.array([k], np.int64))[0])


@pytest.mark.parametrize("thresholds", [
    [0.25, 0.5, 0.75, 1e-20, 0.9999999],                  # one sign
    [-3.0, 2.5, 0.0, 1e-3, -1e-30],                       # both signs, a narrow range
    [-2.0, -1e-3, 1e-3, 2.0, 0.5, -0.5],                  # both signs: the run around zero collapsed
    [-1e30, 1e30, 0.0],
    [-3e38, -1e10, -1.0, -1e-10, 1e-10, 1.0, 1e10, 3e38],  # spread over the whole key range
    [np.inf, -np.inf, 1.0],                                # infinite thresholds
    [1.5],                                                 # one threshold, no run to collapse
    [1.0, np.nextafter(np.float32(1.0), np.float32(2.0))],  # adjacent keys
])
def test_key_remap_is_exact(thresholds):
    """Format 2 compares V(key(x)) with V(key(t)): for every value x (signed
    zeros, subnormals, infinities, NaN, values below, inside and above the
    thresholds' range, inside the collapsed run, each threshold's float
    neighbours) and every threshold t of the forest, V(key(x)) <= V(key(t))
    exactly when x <= t; every row value lies above the stored word of a NaN
    threshold or a dummy slot (0); the run collapsed is the widest one
    between adjacent threshold keys, and the shift is dropped exactly when
    the remaining range needs 32 bits."""
    from packed_decode import obs_key
    th = np.array(thresholds, np.float32)
    n = th.size
    # a chain: internal node i has leaf n + i on its left and node i + 1 (the
    # last one: leaf 2n) on its right
    left = np.array([n + i for i in range(n)] + [-1] * (n + 1), np.int32)
    right = np.array([i + 1 for i in range(n - 1)] + [2 * n] + [-1] * (n + 1), np.int32)
    f = datagen.Forest(2, 2, np.array([0, 2 * n + 1], np.int64), left, right, np.zeros(2 * n + 1, np.int32),
                       np.concatenate([th, np.zeros(n + 1, np.float32)]), np.zeros(2 * n + 1, np.int32),
                       np.zeros(2 * n + 1, np.int64))
    im = Image(fp.fp_pack_forest(f, deep_levels=3, deep_format=2, interleave_depth=0).image())
    assert im.fmt == 2
    keys = np.unique(thr_key(th).astype(np.int64))
    widest = int(np.diff(keys).max()) if keys.size > 1 else 0
    span = int(keys.max()) + 1 - int(keys.min()) - max(0, widest - 2)
    assert (im.h["key_flag"] == 0) == (span >= 1 << 31)
    assert im.h["key_gap_d"] == max(0, widest - 2)
    probes = [0.0, -0.0, 1e-45, -1e-45, 1e-38, -1e-38, 1.0, -1.0, 3.4e38, -3.4e38, np.inf, -np.inf, 0.5, 2.0,
              -5.0, 7e-21, 1e-4, -1e-4, 1e-2, -1e-2, 1e20, -1e20]
    for t in th:
        for step in (np.float32(np.inf), np.float32(-np.inf)):
            probes.append(np.nextafter(t, step))
        probes.append(t)
    x = np.array(probes, np.float32)
    vx = im.remap(obs_key(x).astype(np.int64))
    vt = im.word(th).astype(np.int64)
    for i in range(x.size):
        for j in range(th.size):
            assert (vx[i] <= vt[j]) == bool(x[i] <= th[j]), (x[i], th[j])
    nan = np.array([np.nan], np.float32)
    assert im.remap(obs_key(nan).astype(np.int64))[0] > vt.max()
    assert int(im.word(nan)[0]) == 0
    if im.h["key_flag"]:
        assert np.all(vx >= 0x80000000)  # never equal in the top bit to a dummy's 0


def test_three_level_format2_super_nodes(tiny_forest):
    """Format 2 (fp_internal.h): every slot word is the top bits of the
    slot's remapped key over its feature (32 - fb prefix bits in slots 0..2,
    32 - fb - 2 cb in slots 3..6, whose words also hold their exits' classes);
    the side table holds the seven full remapped keys and a zero; dummies are
    0; leaf mask, offsets and leaf ids as in format 1."""
    f = tiny_forest
    pk = fp.fp_pack_forest(f, bin_size=4, interleave_depth=1, head_select=1, deep_levels=3, deep_format=2)
    im = Image(pk.image())
    fb, cb = im.h["feature_bits"], im.h["class_bits"]
    assert (fb, cb) == (4, 2) and im.fmt == 2 and im.h["key_flag"] == 0x80000000
    fm = (1 << fb) - 1
    n_checked = 0
    for g in range(im.h["n_super"]):
        w = [int(x) for x in im.sw[g]]
        K = [int(x) for x in im.deep_keys[g]]
        assert K[7] == 0
        for i in range(7):
            low = fb if i < 3 else fb + 2 * cb
            assert w[i] >> low == K[i] >> low
            if K[i] == 0:  # a dummy slot: nothing but (possibly) exit classes
                assert w[i] & fm == 0 and w[i] >> low == 0
            else:
                assert K[i] >= 0x80000000
                n_checked += 1
    assert n_checked > 100
    # every stored full key is a remapped threshold of the forest
    allk = set(int(v) for v in im.word(f.threshold[f.left >= 0]))
    assert set(int(k) for k in im.deep_keys[:, :7].reshape(-1) if k) <= allk
