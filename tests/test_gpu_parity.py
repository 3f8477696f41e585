"""GPU parity: the CUDA path against the CPU oracle, element by element.

Everything on this path is integer control flow plus FP32 compares, so the
bar is bit-exactness: per-tree leaf ids, vote counts and classes must equal
the oracle's on the same seeded inputs (tolerance 0)."""
import numpy as np
import pytest

import datagen
import oracle
import paper_1806_07300_gb300 as fp
from golden_io import load

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


# (deep_levels, deep_format): two-level super-nodes, three-level of format 1
# (full keys first) and of format 2 (remapped key prefixes in every slot)
DEEP_KINDS = [(2, 0), (3, 1), (3, 2)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _dev(X):
    return torch.from_numpy(np.ascontiguousarray(X)).cuda()


def _check_all(forest, X, ref=None, **params):
    if ref is None:
        ref = oracle.predict(forest, X, threads=oracle.default_threads())
    pk = fp.fp_pack_forest(forest, **params)
    df = fp.fp_upload(pk)
    Xd = _dev(X)
    votes, cls = df.predict(Xd)
    leaves = df.predict_leaves(Xd)
    torch.cuda.synchronize()
    assert df.sync_status() == fp.FP_OK
    np.testing.assert_array_equal(leaves.cpu().numpy(), ref["leaf"])
    np.testing.assert_array_equal(votes.cpu().numpy().astype(np.uint32), ref["votes"])
    np.testing.assert_array_equal(cls.cpu().numpy(), ref["cls"])
    # classes only (no votes buffer) and votes only
    _, c2 = df.predict(Xd, votes=False)
    v3, _ = df.predict(Xd, classes=False)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(c2.cpu().numpy(), ref["cls"])
    np.testing.assert_array_equal(v3.cpu().numpy().astype(np.uint32), ref["votes"])
    df.release()
    return ref


@pytest.mark.parametrize("name", ["stump_split.txt", "chain_full.txt"])
@pytest.mark.parametrize("B,d,sel", [(1, 0, 3), (2, 1, 3), (3, 3, 3), (1, 0, 1), (2, 3, 1), (1, 1, 2), (3, 3, 2),
                                     (3, 9, 0)])
@pytest.mark.parametrize("dl,fmt", DEEP_KINDS)
def test_hand_fixtures_on_gpu(name, B, d, sel, dl, fmt):
    """±inf, NaN, -0.0, a subnormal and thresholds equal to inputs; ranked
    heads (sel 3), level heads (sel 1) and paired level heads (sel 2); super-
    nodes of two and three levels (both formats)."""
    forest, X, exp = load(name)
    ref = dict(leaf=exp["leaf"], votes=exp["votes"], cls=exp["cls"])
    _check_all(forest, X, ref, bin_size=B, interleave_depth=d, head_select=sel, deep_levels=dl, deep_format=fmt)


@pytest.mark.parametrize("B,d,sel", [(16, 4, 3), (1, 0, 3), (5, 2, 3), (7, 6, 3), (4, 9, 3), (16, 4, 1), (1, 0, 1),
                                     (3, 8, 1), (1, 11, 1), (16, 5, 2), (4, 9, 2), (1, 11, 2), (2, 1, 2)])
@pytest.mark.parametrize("dl,fmt", DEEP_KINDS)
def test_tiny_workload(tiny_forest, tiny_rows, B, d, sel, dl, fmt):
    X, _ = tiny_rows
    _check_all(tiny_forest, X, bin_size=B, interleave_depth=d, head_select=sel, deep_levels=dl, deep_format=fmt)


@pytest.mark.parametrize("B,d,sel", [(4, 2, 1), (3, 1, 2), (2, 3, 3), (1, 0, 1)])
@pytest.mark.parametrize("dl,fmt", DEEP_KINDS)
def test_rows_on_thresholds(tiny_forest, tiny_rows, B, d, sel, dl, fmt):
    """Observations on the forest's thresholds (exactly, or one float step
    off) and -0, infinities and NaN: with three-level super-nodes many
    compares tie on the key prefix and are decided by the full keys (in
    format 2 every row on a threshold ties)."""
    from edge_rows import rows_on_thresholds
    X = rows_on_thresholds(tiny_forest, tiny_rows[0], seed=12)
    _check_all(tiny_forest, X, bin_size=B, interleave_depth=d, head_select=sel, deep_levels=dl, deep_format=fmt)


@pytest.mark.parametrize("rows_kind", ["sampled", "on_thresholds"])
def test_short_key_prefixes(tiny_forest, tiny_rows, rows_kind):
    """The tiny forest declared with 100 features: a 14-bit key prefix in the
    last level of each three-level super-node, so ties are common and the
    kernel decides them from the full keys."""
    from edge_rows import rows_on_thresholds
    f = datagen.Forest(100, tiny_forest.n_classes, tiny_forest.node_begin, tiny_forest.left, tiny_forest.right,
                       tiny_forest.feature, tiny_forest.threshold, tiny_forest.leaf_class, tiny_forest.cardinality)
    X = np.zeros((tiny_rows[0].shape[0], 100), np.float32)
    X[:, :16] = tiny_rows[0] if rows_kind == "sampled" else rows_on_thresholds(tiny_forest, tiny_rows[0], seed=15)
    for B, d, sel in [(4, 2, 1), (3, 1, 2), (2, 3, 3)]:
        _check_all(f, X, bin_size=B, interleave_depth=d, head_select=sel, deep_levels=3)
        _check_all(f, X, bin_size=B, interleave_depth=d, head_select=sel, deep_levels=3, deep_format=2)


@pytest.mark.parametrize("tile,warps", [(32, 1), (64, 3), (256, 8), (1024, 32)])
def test_tiny_tiles_and_ragged_tail(tiny_forest, tiny_rows, tile, warps):
    X, _ = tiny_rows
    _check_all(tiny_forest, X[:tile * 3 + 17], bin_size=4, interleave_depth=2, obs_tile=tile, warps_per_cta=warps)


@pytest.mark.parametrize("B,d,sel,nbuf", [(1, 9, 1, 2), (4, 5, 1, 2), (3, 7, 0, 2), (2, 3, 1, 3)])
def test_tiny_two_bin_buffers(tiny_forest, tiny_rows, B, d, sel, nbuf):
    """Bin blocks streamed through two (or three) shared-memory buffers."""
    X, _ = tiny_rows
    _check_all(tiny_forest, X, bin_size=B, interleave_depth=d, head_select=sel, bin_buffers=nbuf)
    _check_all(tiny_forest, X[:777], bin_size=B, interleave_depth=d, head_select=sel, bin_buffers=nbuf,
               pass_bytes=4096, obs_tile=64)


@pytest.mark.parametrize("pass_bytes", [1, 2048, 8192])
@pytest.mark.parametrize("sel", [3, 1, 2])
def test_tiny_multi_pass(tiny_forest, tiny_rows, pass_bytes, sel):
    """Several passes: global accumulation and last-pass argmax."""
    X, _ = tiny_rows
    pk = fp.fp_pack_forest(tiny_forest, bin_size=2, interleave_depth=1, pass_bytes=pass_bytes, head_select=sel)
    assert pk.info()["passes"] > 1
    _check_all(tiny_forest, X, bin_size=2, interleave_depth=1, pass_bytes=pass_bytes, obs_tile=128, head_select=sel)


def test_resident_forests_sharing_a_kernel(tiny_forest, tiny_rows):
    """Forests that run the same compiled kernel (same super-node kind, head
    kind and CTA size) but need different shared memory (1024-row and 64-row
    tiles) all stay usable, in every mode, whichever was uploaded or
    configured last."""
    X, _ = tiny_rows
    ref = oracle.predict(tiny_forest, X)
    Xd = _dev(X)
    big = fp.fp_upload(fp.fp_pack_forest(tiny_forest, bin_size=4, interleave_depth=3, obs_tile=1024))
    small = fp.fp_upload(fp.fp_pack_forest(tiny_forest, bin_size=4, interleave_depth=3, obs_tile=64))
    assert big.info["obs_tile"] > small.info["obs_tile"]

    def check(df):
        votes, cls = df.predict(Xd)
        leaves = df.predict_leaves(Xd)
        torch.cuda.synchronize()
        assert df.sync_status() == fp.FP_OK
        np.testing.assert_array_equal(votes.cpu().numpy().astype(np.uint32), ref["votes"])
        np.testing.assert_array_equal(cls.cpu().numpy(), ref["cls"])
        np.testing.assert_array_equal(leaves.cpu().numpy(), ref["leaf"])

    for df in (big, small, big):
        check(df)
    small.configure(obs_tile=32)
    check(big)
    big.configure(obs_tile=512)
    check(small)
    check(big)
    big.release()
    small.release()


@pytest.mark.parametrize("n", [0, 1, 2, 31, 33])
def test_small_and_empty_batches(tiny_forest, tiny_rows, n):
    X, _ = tiny_rows
    if n == 0:
        df = fp.fp_upload(fp.fp_pack_forest(tiny_forest))
        Xd = torch.empty((0, tiny_forest.n_features), dtype=torch.float32, device="cuda")
        v, c = df.predict(Xd)
        assert v.shape == (0, tiny_forest.n_classes) and c.shape == (0,)
        df.release()
        return
    _check_all(tiny_forest, X[:n])


def test_no_cardinality_keeps_left_first(tiny_forest, tiny_rows):
    X, _ = tiny_rows
    f = datagen.Forest(tiny_forest.n_features, tiny_forest.n_classes, tiny_forest.node_begin, tiny_forest.left,
                       tiny_forest.right, tiny_forest.feature, tiny_forest.threshold, tiny_forest.leaf_class,
                       tiny_forest.cardinality)
    f.cardinality = None
    ref = oracle.predict(tiny_forest, X)
    _check_all(f, X, ref)


@pytest.mark.parametrize("order", [fp.FP_PLAIN_OBS_FASTEST, fp.FP_PLAIN_TREE_FASTEST])
def test_plain_baseline(tiny_forest, tiny_rows, order):
    X, _ = tiny_rows
    ref = oracle.predict(tiny_forest, X)
    pf = fp.fp_plain_build(tiny_forest)
    v, c = pf.predict(_dev(X), order=order)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(v.cpu().numpy().astype(np.uint32), ref["votes"])
    np.testing.assert_array_equal(c.cpu().numpy(), ref["cls"])
    pf.release()


@pytest.mark.parametrize("name", ["stump_split.txt", "chain_full.txt"])
def test_plain_baseline_fixture(name):
    forest, X, exp = load(name)
    pf = fp.fp_plain_build(forest)
    v, c = pf.predict(_dev(X))
    torch.cuda.synchronize()
    np.testing.assert_array_equal(v.cpu().numpy().astype(np.uint32), exp["votes"])
    np.testing.assert_array_equal(c.cpu().numpy(), exp["cls"])


@pytest.mark.parametrize("kinds", [((0, 0),) * 4, ((2, 0),) * 4, ((3, 2),) * 4, ((3, 1), (2, 0), (3, 1), (2, 0)),
                                   ((3, 2), (2, 0), (3, 1), (3, 2))])
def test_batched_matches_single(tiny_forest, tiny_rows, kinds):
    """One launch over four forests: all with three-level super-nodes of
    format 1 (the default here) or of format 2, all with two-level ones, or
    mixes of the kinds."""
    X, _ = tiny_rows
    forests, Xs, refs = [], [], []
    for i, n in enumerate([1, 700, 33, 5000]):
        dl, fmt = kinds[i]
        forests.append(fp.fp_upload(fp.fp_pack_forest(tiny_forest, bin_size=1 + 3 * i, interleave_depth=i,
                                                      deep_levels=dl, deep_format=fmt)))
        Xs.append(_dev(X[i * 10: i * 10 + n]))
        refs.append(oracle.predict(tiny_forest, X[i * 10: i * 10 + n]))
    votes = [torch.empty((x.shape[0], tiny_forest.n_classes), dtype=torch.int32, device="cuda") for x in Xs]
    cls = [torch.empty((x.shape[0],), dtype=torch.int32, device="cuda") for x in Xs]
    fp.fp_predict_batched(forests, Xs, votes, cls)
    torch.cuda.synchronize()
    for v, c, r in zip(votes, cls, refs):
        np.testing.assert_array_equal(v.cpu().numpy().astype(np.uint32), r["votes"])
        np.testing.assert_array_equal(c.cpu().numpy(), r["cls"])


def test_image_workload_10k():
    """Image-shaped workload (784 features, 10 classes, 128 trees), 10,000
    rows: the default (three-level super-nodes of format 2) and two-level
    super-nodes."""
    forest = datagen.forest("image")
    X, _ = datagen.test_rows("image", 10000)
    ref = _check_all(forest, X)
    assert fp.fp_pack_forest(forest).info()["deep_format"] == 2
    _check_all(forest, X, ref, deep_levels=2)


def test_image_workload_params_grid():
    forest = datagen.forest("image")
    X, _ = datagen.test_rows("image", 3000)
    ref = oracle.predict(forest, X, threads=oracle.default_threads())
    # rows of 784 features leave little shared memory: tiles shrink to fit
    for B, d, sel, nb in [(128, 1, 3, 3), (16, 3, 3, 3), (8, 5, 3, 3), (1, 9, 3, 3), (16, 5, 1, 3), (1, 10, 1, 3),
                          (4, 7, 2, 3), (1, 11, 2, 2)]:
        _check_all(forest, X, ref, bin_size=B, interleave_depth=d, head_select=sel, bin_buffers=nb)
    # rows on the forest's thresholds, through its (two-level) super-nodes
    from edge_rows import rows_on_thresholds
    Xe = rows_on_thresholds(forest, X[:1000], seed=13)
    _check_all(forest, Xe, None, bin_size=16, interleave_depth=3, head_select=2)
