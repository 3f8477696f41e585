"""Tree-bin sharding on the host (Section III binds bins of trees to
processes): the split covers every tree exactly once in whole bins and
balances expected work, and two gloo ranks that each classify with their own
packed shard (decoded on the CPU by the independent image reader) and sum
their votes with an all-reduce get the oracle's votes and classes for the
whole forest.  The device path (fp_predict per shard, NCCL, fp_votes_argmax)
needs one GPU per rank; its arithmetic is checked on one GPU by
tests/test_gpu_sharding.py."""
import os
import socket

import numpy as np
import pytest

import datagen
import oracle
import paper_1806_07300_gb300 as fp
from packed_decode import Image

torch = pytest.importorskip("torch")


def _work(forest):
    """Expected internal visits per observation, per tree (from cardinalities)."""
    out = []
    for t in range(forest.n_trees):
        tr = forest.tree(t)
        out.append(tr["cardinality"][tr["left"] >= 0].sum() / tr["cardinality"][0])
    return np.array(out)


@pytest.mark.parametrize("n_shards,bin_size", [(1, 3), (2, 2), (3, 4), (5, 1), (7, 3), (40, 1)])
def test_split_covers_every_tree_in_whole_bins(tiny_forest, n_shards, bin_size):
    T = tiny_forest.n_trees
    ranges = [fp.fp_shard_trees(tiny_forest, bin_size, n_shards, k) for k in range(n_shards)]
    covered = []
    for b, e in ranges:
        assert b <= e and (b % bin_size == 0 or b == T) and (e % bin_size == 0 or e == T)
        covered.extend(range(b, e))
    assert covered == list(range(T))  # contiguous, disjoint, complete
    work = _work(tiny_forest)
    loads = [work[b:e].sum() for b, e in ranges]
    bins = [work[i: i + bin_size].sum() for i in range(0, T, bin_size)]
    if n_shards <= len(bins):  # each shard within one bin of the even share
        assert max(loads) <= work.sum() / n_shards + max(bins) + 1e-9


def test_split_without_cardinalities_counts_nodes(tiny_forest):
    f = datagen.Forest(tiny_forest.n_features, tiny_forest.n_classes, tiny_forest.node_begin, tiny_forest.left,
                       tiny_forest.right, tiny_forest.feature, tiny_forest.threshold, tiny_forest.leaf_class,
                       np.zeros(tiny_forest.n_nodes, np.int64))
    f.cardinality = None
    b, e = fp.fp_shard_trees(f, 1, 2, 0)
    nb = f.node_begin
    internal = np.array([(f.left[nb[t]: nb[t + 1]] >= 0).sum() for t in range(f.n_trees)])
    assert abs(internal[:e].sum() - internal.sum() / 2) <= internal.max()
    with pytest.raises(fp.FPError):
        fp.fp_shard_trees(f, 1, 2, 2)
    with pytest.raises(fp.FPError):
        fp.fp_pack_forest_trees(f, 3, 3)


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1806_07300_gb300.sharding import ShardedForest
    forest = datagen.forest("tiny")
    X, _ = datagen.test_rows("tiny", 3000)
    sf = ShardedForest(forest, bin_size=2, upload=False, interleave_depth=3)
    votes = np.zeros((X.shape[0], forest.n_classes), np.int32)
    if sf.packed is not None:
        _, cls = Image(sf.packed.image()).walk(X)  # this rank's trees only
        for c in range(forest.n_classes):
            votes[:, c] = (cls == c).sum(axis=1)
    t = torch.from_numpy(votes)
    sf.reduce_votes(t)
    q.put((rank, sf.tree_begin, sf.tree_end, t.numpy()))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_sum_to_the_whole_forest(world):
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    forest = datagen.forest("tiny")
    X, _ = datagen.test_rows("tiny", 3000)
    ref = oracle.predict(forest, X, leaves=False)
    spans = sorted((b, e) for _, b, e, _ in got)
    assert spans[0][0] == 0 and spans[-1][1] == forest.n_trees
    assert all(spans[i][1] == spans[i + 1][0] for i in range(world - 1))
    for _, _, _, votes in got:  # every rank holds the whole forest's votes
        np.testing.assert_array_equal(votes.astype(np.uint32), ref["votes"])
        np.testing.assert_array_equal(np.argmax(votes, axis=1), ref["cls"])
