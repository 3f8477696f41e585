"""Packed records of random forests with adversarial thresholds (signed
zeros, subnormals, huge magnitudes, infinities, NaN; Section III-A: a layout
must not change any prediction) decode, through the independent image
reader, to the oracle's leaves for every kind of super-node, head kind and a
few (B, d); the prefix compares they make are checked against the full keys
on the way."""
import numpy as np
import pytest

import oracle
import paper_1806_07300_gb300 as fp
import random_forests as rf
from packed_decode import Image

KINDS = [(2, 0), (3, 1), (3, 2)]


@pytest.mark.parametrize("seed,kind", [(1, "mixed"), (2, "mixed"), (3, "positive"), (4, "narrow"), (5, "mixed")])
@pytest.mark.parametrize("dl,fmt", KINDS)
@pytest.mark.parametrize("B,d,sel", [(4, 3, 2), (3, 2, 1), (2, 3, 3)])
def test_random_forest_records_decode_to_oracle_leaves(seed, kind, dl, fmt, B, d, sel):
    f = rf.forest(seed, kind=kind)
    X = rf.rows(f, 1500, seed + 100, kind)
    ref = oracle.predict(f, X)
    pk = fp.fp_pack_forest(f, bin_size=B, interleave_depth=d, head_select=sel, deep_levels=dl, deep_format=fmt)
    assert (pk.info()["deep_levels"], pk.info()["deep_format"]) == (dl, fmt)
    im = Image(pk.image())
    leaf, _ = im.walk(X)
    np.testing.assert_array_equal(leaf, ref["leaf"])


def test_random_forests_reach_the_corners():
    """The fixtures do what they are for: NaN and infinite thresholds exist,
    the 'mixed' forests' keys span more than 2^31 even after the widest empty
    run is collapsed (so format 2 falls back to the plain keys there), the
    'positive' and 'narrow' ones remap, and rows tie with prefixes."""
    f = rf.forest(1, kind="mixed")
    th = f.threshold[f.left >= 0]
    assert np.isnan(th).any() and np.isinf(th).any() and (th == 0).any()
    im = Image(fp.fp_pack_forest(f, deep_levels=3, deep_format=2, interleave_depth=1).image())
    assert im.h["key_flag"] == 0
    for seed, kind in ((3, "positive"), (4, "narrow")):
        g = rf.forest(seed, kind=kind)
        im = Image(fp.fp_pack_forest(g, deep_levels=3, deep_format=2, interleave_depth=1).image())
        assert im.h["key_flag"] == 0x80000000
        im.walk(rf.rows(g, 1500, seed + 100, kind))
        assert im.ties > 0
