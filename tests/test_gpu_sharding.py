"""Tree-bin sharding on the device: shards packed with fp_pack_forest_trees
classify the same rows with fp_predict, their votes are added, and
fp_votes_argmax gives the whole forest's classes -- checked against the
oracle.  The ranks are emulated one after another on one GPU (their launches
do not wait on each other; the sum stands for the all-reduce), and a
ShardedForest without a process group is the whole forest."""
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


@pytest.mark.parametrize("name,n,world,bin_size,fmt", [("tiny", 10000, 2, 2, 0), ("tiny", 10000, 3, 1, 0),
                                                       ("wide", 20000, 3, 4, 0), ("hbm", 30000, 4, 4, 0),
                                                       ("tiny", 10000, 3, 2, 2), ("hbm", 30000, 3, 4, 2)])
def test_shards_sum_to_the_whole_forest(name, n, world, bin_size, fmt):
    """fmt 2: three-level super-nodes of format 2 forced, so every shard
    remaps its keys onto its own trees' thresholds (the wide forest takes
    format 2 by default)."""
    forest = datagen.forest(name)
    X, _ = datagen.test_rows(name, n)
    Xd = torch.from_numpy(X).cuda()
    total = torch.zeros((n, forest.n_classes), dtype=torch.int32, device="cuda")
    trees = 0
    for k in range(world):
        b, e = fp.fp_shard_trees(forest, bin_size, world, k)
        if e == b:
            continue
        df = fp.fp_upload(fp.fp_pack_forest_trees(forest, b, e, bin_size=bin_size, deep_format=fmt))
        votes = torch.empty((n, forest.n_classes), dtype=torch.int32, device="cuda")
        fp.fp_predict(df, Xd, votes, None)
        total += votes
        trees += e - b
        torch.cuda.synchronize()
        assert df.sync_status() == fp.FP_OK
        df.release()
    assert trees == forest.n_trees
    cls = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    fp.fp_votes_argmax(total, cls)
    torch.cuda.synchronize()
    ref = oracle.predict(forest, X, leaves=False, threads=oracle.default_threads())
    np.testing.assert_array_equal(total.cpu().numpy().astype(np.uint32), ref["votes"])
    np.testing.assert_array_equal(cls.cpu().numpy(), ref["cls"])


def test_argmax_ties_and_edges():
    """Lowest class on ties, one class, no rows."""
    v = torch.tensor([[3, 3, 1], [0, 0, 0], [1, 5, 5], [2, 1, 7]], dtype=torch.int32, device="cuda")
    c = torch.empty(4, dtype=torch.int32, device="cuda")
    fp.fp_votes_argmax(v, c)
    one = torch.zeros(5, dtype=torch.int32, device="cuda")
    fp.fp_votes_argmax(torch.ones((5, 1), dtype=torch.int32, device="cuda"), one)
    fp.fp_votes_argmax(torch.empty((0, 3), dtype=torch.int32, device="cuda"), torch.empty(0, dtype=torch.int32,
                                                                                          device="cuda"))
    torch.cuda.synchronize()
    assert c.cpu().tolist() == [0, 0, 1, 2] and one.cpu().tolist() == [0] * 5


def test_sharded_forest_without_a_group_is_the_whole_forest():
    from paper_1806_07300_gb300.sharding import ShardedForest
    forest = datagen.forest("tiny")
    X, _ = datagen.test_rows("tiny", 5000)
    sf = ShardedForest(forest, bin_size=4)
    assert (sf.tree_begin, sf.tree_end) == (0, forest.n_trees)
    votes, cls = sf.predict(torch.from_numpy(X).cuda())
    torch.cuda.synchronize()
    ref = oracle.predict(forest, X, leaves=False)
    np.testing.assert_array_equal(votes.cpu().numpy().astype(np.uint32), ref["votes"])
    np.testing.assert_array_equal(cls.cpu().numpy(), ref["cls"])
    sf.release()
