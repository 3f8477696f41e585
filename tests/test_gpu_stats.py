"""Statistics inferred from observations (Section III-A) and the layout
ablation: every layout variant -- DF order (no statistics), Stat with
training cardinalities, Stat with cardinalities counted on the device from
observations, heads chosen by level or by cardinality -- classifies exactly
like the oracle (layouts never change predictions)."""
import numpy as np
import pytest

import datagen
import oracle
import paper_1806_07300_gb300 as fp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _oracle_cardinality(forest, X):
    """Leaf counts from the oracle's leaves, summed into ancestors (written
    here independently of the library helper)."""
    r = oracle.predict(forest, X, votes=False, classes=False)
    card = np.zeros(forest.n_nodes, np.int64)
    for t in range(forest.n_trees):
        b = int(forest.node_begin[t])
        np.add.at(card, b + r["leaf"][:, t], 1)
        tr = forest.tree(t)
        # bottom-up by decreasing depth
        depth = {0: 0}
        order = [0]
        for v in order:
            if tr["left"][v] >= 0:
                for c in (int(tr["left"][v]), int(tr["right"][v])):
                    depth[c] = depth[v] + 1
                    order.append(c)
        for v in sorted(order, key=lambda v: -depth[v]):
            if tr["left"][v] >= 0:
                card[b + v] = card[b + tr["left"][v]] + card[b + tr["right"][v]]
    return card


def test_inferred_cardinality_matches_oracle_counts(tiny_forest, tiny_rows):
    X, _ = tiny_rows
    Xd = torch.from_numpy(X).cuda()
    card = fp.infer_cardinality(tiny_forest, Xd)
    np.testing.assert_array_equal(card, _oracle_cardinality(tiny_forest, X))
    roots = card[tiny_forest.node_begin[:-1]]
    assert np.all(roots == X.shape[0])


@pytest.mark.parametrize("name,n", [("tiny", 10000), ("image", 4000)])
def test_layout_ablation_preserves_predictions(name, n):
    forest = datagen.forest(name)
    X, _ = datagen.test_rows(name, n)
    Xd = torch.from_numpy(X).cuda()
    ref = oracle.predict(forest, X, threads=oracle.default_threads())
    inferred = datagen.Forest(forest.n_features, forest.n_classes, forest.node_begin, forest.left, forest.right,
                              forest.feature, forest.threshold, forest.leaf_class, fp.infer_cardinality(forest, Xd))
    no_stats = datagen.Forest(forest.n_features, forest.n_classes, forest.node_begin, forest.left, forest.right,
                              forest.feature, forest.threshold, forest.leaf_class, forest.cardinality)
    no_stats.cardinality = None
    variants = [(no_stats, dict(bin_size=1, interleave_depth=0)),            # DF order, roots only
                (forest, dict(bin_size=1, interleave_depth=0)),              # Stat
                (inferred, dict(bin_size=1, interleave_depth=0)),            # Stat from observations
                (forest, dict(bin_size=16, interleave_depth=4, head_select=1)),  # Bin, levels 0..4
                (forest, dict(bin_size=16, interleave_depth=4)),             # Bin, popular nodes
                (inferred, dict(bin_size=5, interleave_depth=6))]
    for f, params in variants:
        df = fp.fp_upload(fp.fp_pack_forest(f, **params))
        v, c = df.predict(Xd)
        leaves = df.predict_leaves(Xd)
        torch.cuda.synchronize()
        assert df.sync_status() == fp.FP_OK
        np.testing.assert_array_equal(c.cpu().numpy(), ref["cls"])
        np.testing.assert_array_equal(v.cpu().numpy().astype(np.uint32), ref["votes"])
        np.testing.assert_array_equal(leaves.cpu().numpy(), ref["leaf"])
        df.release()


def test_inferred_cardinality_chunked_and_empty(tiny_forest, tiny_rows):
    """The rows go through the device in chunks of any size with the same
    counts; no rows give zero everywhere."""
    X, _ = tiny_rows
    Xd = torch.from_numpy(X).cuda()
    whole = fp.infer_cardinality(tiny_forest, Xd)
    for chunk in (1, 777, 4096):
        np.testing.assert_array_equal(fp.infer_cardinality(tiny_forest, Xd, chunk_rows=chunk), whole)
    assert not fp.infer_cardinality(tiny_forest, Xd[:0]).any()
