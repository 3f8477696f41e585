"""Tree-bin sharding over the ranks of a process group.

The paper binds the bins of a forest to processes (Section III) and spreads
them over machines (Section IV-E).  Here every rank of a torch.distributed
group keeps the bins of its own shard resident on its GPU: fp_shard_trees
chooses whole bins so that each rank's expected work is about the same, and
fp_pack_forest_trees packs them.  Every rank classifies the same rows with
its shard (fp_predict, votes only), the per-class votes are summed over the
ranks with one all-reduce (NCCL for device tensors, gloo for host tensors),
and fp_votes_argmax turns the sums into classes on the device.  Every tree
belongs to exactly one shard, so the summed votes and the classes are the
whole forest's.  With one rank, or without an initialised process group, the
shard is the whole forest and no collective runs.

This module only plans and marshals: packing, classification and the argmax
run in the library, the sum in the collective library.
"""
from __future__ import annotations

from . import fp_pack_forest_trees, fp_predict, fp_shard_trees, fp_upload, fp_votes_argmax


class ShardedForest:
    """One rank's shard of a forest split by bins.

    forest       the whole forest (every rank passes the same one)
    group        torch.distributed process group (None: the default group, if
                 initialised)
    bin_size     trees per bin; shards are whole bins
    upload       False keeps only the packed host image (for host-side use)
    pack_params  further fp_pack_forest parameters for the shard
    """

    def __init__(self, forest, group=None, bin_size: int = 3, upload: bool = True, **pack_params):
        import torch.distributed as dist
        self.dist = dist if (dist.is_available() and dist.is_initialized()) else None
        self.group = group
        self.world = self.dist.get_world_size(group) if self.dist else 1
        self.rank = self.dist.get_rank(group) if self.dist else 0
        self.n_classes = forest.n_classes
        self.n_features = forest.n_features
        self.tree_begin, self.tree_end = fp_shard_trees(forest, bin_size, self.world, self.rank)
        self.packed = None
        self.df = None
        if self.tree_end > self.tree_begin:
            self.packed = fp_pack_forest_trees(forest, self.tree_begin, self.tree_end, bin_size=bin_size,
                                               **pack_params)
            if upload:
                self.df = fp_upload(self.packed)

    @property
    def n_trees(self) -> int:
        return self.tree_end - self.tree_begin

    def local_votes(self, X, stream=None):
        """Votes of this rank's trees for the rows X (CUDA float32 [n][F])."""
        import torch
        votes = torch.zeros((X.shape[0], self.n_classes), dtype=torch.int32, device=X.device)
        if self.df is not None and X.shape[0] > 0:
            fp_predict(self.df, X, votes, None, stream)
        return votes

    def reduce_votes(self, votes):
        """Sum a [n][n_classes] vote tensor over the ranks, in place."""
        if self.world > 1:
            self.dist.all_reduce(votes, op=self.dist.ReduceOp.SUM, group=self.group)
        return votes

    def predict(self, X, stream=None):
        """(votes, classes) of the whole forest for the rows X, on every rank."""
        import torch
        ctx = torch.cuda.stream(stream) if stream is not None else _null()
        with ctx:
            votes = self.reduce_votes(self.local_votes(X))
            classes = torch.empty((X.shape[0],), dtype=torch.int32, device=X.device)
            fp_votes_argmax(votes, classes)
        return votes, classes

    def release(self) -> None:
        if self.df is not None:
            self.df.release()
            self.df = None
        if self.packed is not None:
            self.packed.release()
            self.packed = None


class _null:
    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False
