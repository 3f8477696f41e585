"""Degenerate forests through every kind of super-node and head: every tree a
single leaf (no thresholds at all, so format 2's remap has nothing to
spread), one class (no class bits), a single stump, trees whose only split
is NaN or infinite.  The host decoder and the kernel must give the oracle's
leaves, votes and classes."""
import numpy as np
import pytest

import datagen
import oracle
import paper_1806_07300_gb300 as fp
from packed_decode import Image

KINDS = [(2, 0), (3, 1), (3, 2)]
HEADS = [(1, 2, 3), (2, 0, 1), (3, 1, 2)]  # (bin_size, interleave_depth, head_select)


def _forest(trees, n_features=3, n_classes=2):
    """trees: list of (left, right, feature, threshold, leaf_class) node lists."""
    nb, L, R, Fe, Th, Cl, Ca = [0], [], [], [], [], [], []
    for left, right, feat, thr, cls in trees:
        m = len(left)
        card = np.zeros(m, np.int64)
        for v in range(m - 1, -1, -1):
            card[v] = 7 if left[v] < 0 else card[left[v]] + card[right[v]]
        L += left; R += right; Fe += feat; Th += thr; Cl += cls; Ca += list(card)
        nb.append(nb[-1] + m)
    return datagen.Forest(n_features, n_classes, np.array(nb, np.int64), np.array(L, np.int32), np.array(R, np.int32),
                          np.array(Fe, np.int32), np.array(Th, np.float32), np.array(Cl, np.int32),
                          np.array(Ca, np.int64))


LEAF = lambda c: ([-1], [-1], [0], [0.0], [c])  # noqa: E731
STUMP = lambda f, t, a, b: ([1, -1, -1], [2, -1, -1], [f, 0, 0], [t, 0.0, 0.0], [0, a, b])  # noqa: E731

FORESTS = {
    "all_leaves": lambda: _forest([LEAF(0), LEAF(1), LEAF(1)]),
    "one_class": lambda: _forest([STUMP(0, 0.5, 0, 0), LEAF(0), STUMP(2, -1.0, 0, 0)], n_classes=1),
    "single_stump": lambda: _forest([STUMP(1, 0.25, 1, 0)]),
    "nan_and_inf_splits": lambda: _forest([STUMP(0, np.nan, 0, 1), STUMP(1, np.inf, 1, 0), STUMP(2, -np.inf, 0, 1),
                                           LEAF(1)]),
}


def _rows(n=777):
    rng = np.random.default_rng(3)
    X = rng.normal(size=(n, 3)).astype(np.float32)
    sp = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 0.25, 0.5, -1.0], np.float32)
    m = rng.random(X.shape) < 0.3
    X[m] = sp[rng.integers(0, sp.size, int(m.sum()))]
    return X


@pytest.mark.parametrize("name", sorted(FORESTS))
@pytest.mark.parametrize("dl,fmt", KINDS)
@pytest.mark.parametrize("B,d,sel", HEADS)
def test_degenerate_forest_records(name, dl, fmt, B, d, sel):
    f = FORESTS[name]()
    X = _rows()
    ref = oracle.predict(f, X)
    im = Image(fp.fp_pack_forest(f, bin_size=B, interleave_depth=d, head_select=sel, deep_levels=dl,
                                 deep_format=fmt).image())
    leaf, _ = im.walk(X)
    np.testing.assert_array_equal(leaf, ref["leaf"])


@pytest.mark.gpu
@pytest.mark.parametrize("name", sorted(FORESTS))
@pytest.mark.parametrize("dl,fmt", KINDS)
@pytest.mark.parametrize("B,d,sel", HEADS)
def test_degenerate_forest_on_gpu(name, dl, fmt, B, d, sel):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    f = FORESTS[name]()
    X = _rows()
    ref = oracle.predict(f, X)
    df = fp.fp_upload(fp.fp_pack_forest(f, bin_size=B, interleave_depth=d, head_select=sel, deep_levels=dl,
                                        deep_format=fmt))
    Xd = torch.from_numpy(X).cuda()
    votes, cls = df.predict(Xd)
    leaves = df.predict_leaves(Xd)
    torch.cuda.synchronize()
    assert df.sync_status() == fp.FP_OK
    np.testing.assert_array_equal(leaves.cpu().numpy(), ref["leaf"])
    np.testing.assert_array_equal(votes.cpu().numpy().astype(np.uint32), ref["votes"])
    np.testing.assert_array_equal(cls.cpu().numpy(), ref["cls"])
    df.release()
