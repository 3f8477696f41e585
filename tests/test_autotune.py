"""Autotuner: candidate generation (CPU) and a GPU run on the tiny workload."""
import numpy as np
import pytest

import datagen
import oracle
import paper_1806_07300_gb300 as fp
from paper_1806_07300_gb300 import autotune as at


def test_block_bytes_formula():
    # stride = B | 1; K = 2^(d+1)-1 head nodes of 8 B and K+1 exits of 4 B per tree slot
    assert at.block_bytes(1, 0) == 1 * 1 * 8 + 1 * 2 * 4
    assert at.block_bytes(2, 1) == 3 * 3 * 8 + 3 * 4 * 4
    assert at.block_bytes(16, 3) == 17 * 15 * 8 + 17 * 16 * 4
    # paired level heads: (4^2 - 1)/3 = 5 records of 16 bytes and 16 exits per tree slot
    assert at.block_bytes(16, 3, 2) == 17 * 5 * 16 + 17 * 16 * 4


def test_candidate_layouts_pack(tiny_forest):
    cands = at.candidate_layouts(tiny_forest.n_trees)
    assert 2 <= len(cands) <= 17
    assert {c[2] for c in cands} == {1, 2, 3}
    assert [c[3] for c in cands if len(c) > 3] == [2]  # one two-level candidate beside the defaults
    assert len(at.candidate_layouts(tiny_forest.n_trees, max_layouts=5)) <= 5
    for c in cands:
        B, d, sel = c[:3]
        assert 1 <= B <= tiny_forest.n_trees and 0 <= d <= (9 if sel == 3 else 11)
        assert at.block_bytes(B, d, sel) <= 48 * 1024 or d == 0
        assert sel != 2 or d % 2 == 1
        fp.fp_pack_forest(tiny_forest, **dict(zip(at.LAYOUT_KEYS, c)))


def test_candidate_launches():
    for tile, warps, refill, nbuf in at.candidate_launches(480):
        assert tile % 32 == 0 and 32 <= tile <= 480
        assert warps in (16, 32) and refill in (8, 16) and nbuf in (2, 3)


def test_forest_key_changes_with_forest(tiny_forest):
    k1 = at.forest_key(tiny_forest)
    f2 = datagen.Forest(tiny_forest.n_features, tiny_forest.n_classes, tiny_forest.node_begin, tiny_forest.left,
                        tiny_forest.right, tiny_forest.feature, tiny_forest.threshold + np.float32(1.0),
                        tiny_forest.leaf_class, tiny_forest.cardinality)
    assert at.forest_key(f2) != k1
    assert at.forest_key(tiny_forest) == k1


@pytest.mark.gpu
def test_autotune_tiny_on_gpu(tiny_forest, tiny_rows, tmp_path, monkeypatch):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    monkeypatch.setenv("FP_CACHE_DIR", str(tmp_path))
    X, _ = tiny_rows
    Xd = torch.from_numpy(X).cuda()
    best = at.autotune(tiny_forest, Xd, layouts=[(1, 3), (16, 4, 1), (4, 6, 3), (2, 7, 2)],
                       launches=[(256, 16, 16), (128, 32, 32, 2)])
    assert best["ms"] > 0 and len(best["table"]) == 8
    again = at.autotune(tiny_forest, Xd, layouts=[(1, 0)])  # served from the cache
    assert all(again[k] == best[k] for k in at.LAYOUT_KEYS)
    df, _ = at.upload_tuned(tiny_forest, Xd)
    v, c = df.predict(Xd)
    torch.cuda.synchronize()
    ref = oracle.predict(tiny_forest, X)
    np.testing.assert_array_equal(c.cpu().numpy(), ref["cls"])
    np.testing.assert_array_equal(v.cpu().numpy().astype(np.uint32), ref["votes"])


@pytest.mark.gpu
def test_autotune_batched_on_gpu(tiny_forest, tiny_rows):
    """One layout for a shared batched launch, chosen by timing the launch."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    X, _ = tiny_rows
    Xh = [X[:3000], X[3000:3007], X[4000:9000]]
    Xs = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in Xh]
    dfs, best = at.autotune_batched([tiny_forest] * 3, Xs, layouts=[(3, 9, 2), (8, 4, 1), (2, 5, 3)],
                                    launches=[(0, 32, 16, 3), (256, 16, 8, 2)], reps=2)
    assert best["ms"] > 0 and len(best["table"]) == 6
    cls = [torch.empty((x.shape[0],), dtype=torch.int32, device="cuda") for x in Xs]
    fp.fp_predict_batched(dfs, Xs, None, cls)
    torch.cuda.synchronize()
    for x, c in zip(Xh, cls):
        np.testing.assert_array_equal(c.cpu().numpy(), oracle.predict(tiny_forest, x)["cls"])
