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
from packed_decode import Image, HOT_RIGHT, BOTH_LEAF, COLD_LEAF, PAYLOAD

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "forest_pack.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fp_[a-z_]+)\s*\(", src)))


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
@pytest.mark.parametrize("B,d", [(1, 0), (2, 0), (2, 1), (3, 2), (1, 5)])
def test_packed_records_decode_to_fixture_leaves(name, B, d):
    forest, X, exp = load(name)
    pk = fp.fp_pack_forest(forest, bin_size=B, interleave_depth=d)
    leaf, cls = Image(pk.image()).walk(X)
    np.testing.assert_array_equal(leaf, exp["leaf"])


@pytest.mark.parametrize("B,d", [(16, 4), (5, 0), (1, 2), (7, 7)])
def test_packed_records_decode_to_oracle_leaves(tiny_forest, tiny_rows, B, d):
    X, _ = tiny_rows
    ref = oracle.predict(tiny_forest, X[:3000])
    pk = fp.fp_pack_forest(tiny_forest, bin_size=B, interleave_depth=d)
    leaf, cls = Image(pk.image()).walk(X[:3000])
    np.testing.assert_array_equal(leaf, ref["leaf"])
    np.testing.assert_array_equal(cls, tiny_forest.leaf_class[tiny_forest.node_begin[:-1][None, :] + ref["leaf"]])


def test_stat_order_in_packed_records(tiny_forest):
    """Below the interleaved levels the hot child sits right after its parent
    (Section III-A, Stat): the record at index+1 is the hot child's."""
    f = tiny_forest
    pk = fp.fp_pack_forest(f, bin_size=4, interleave_depth=1)
    im = Image(pk.image())
    m = im.deep_meta
    for t in range(f.n_trees):
        tr = f.tree(t)
        a, b = int(im.tree_base[t]), (int(im.tree_base[t + 1]) if t + 1 < f.n_trees else len(m))
        for i in range(a, b):
            mm = int(m[i])
            if mm & BOTH_LEAF:
                continue
            hot_right = bool(mm & HOT_RIGHT)
            assert i + 1 < b
            nxt = int(m[i + 1])
            feat = mm >> 22
            # the hot child record must exist at i+1 and be internal
            assert (nxt >> 22) < f.n_features
            if not (mm & COLD_LEAF):
                assert (mm & PAYLOAD) > i - a, "the cold subtree follows the hot one"
            del feat, hot_right


def test_head_interleaving_roots_contiguous(tiny_forest):
    """Fig. 2 caption: depth 0 puts the roots of a bin's trees side by side."""
    f = tiny_forest
    pk = fp.fp_pack_forest(f, bin_size=8, interleave_depth=0)
    im = Image(pk.image())
    for b in range(im.h["n_bins"]):
        thr, meta, link, par = im.head(b)
        first = int(im.bins[b]["first_tree"])
        for k in range(meta.shape[1]):
            t = first + k
            root = int(f.node_begin[t])
            assert meta[0, k] == f.feature[root]
            assert thr[0, k] == f.threshold[root]


def test_pack_info_sizes(tiny_forest):
    pk = fp.fp_pack_forest(tiny_forest, bin_size=16, interleave_depth=2)
    info = pk.info()
    internal = int((tiny_forest.left >= 0).sum())
    # nodes at levels 0..2 live in the interleaved block; the rest are records
    im = Image(pk.image())
    in_head = sum(int(((im.head(b)[1] & 0x80000000) == 0).sum()) for b in range(im.h["n_bins"]))
    assert info["n_deep_records"] + in_head == internal
    assert info["deep_bytes"] == 8 * info["n_deep_records"]
    assert info["n_bins"] == 1 and info["passes"] == 1


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


@pytest.mark.parametrize("kw", [dict(bin_size=-1), dict(interleave_depth=12), dict(obs_tile=33),
                                dict(warps_per_cta=40)])
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
