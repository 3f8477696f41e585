"""GPU parity at the format's limits: the largest feature and class counts
(1024 features, 512 classes), row indices whose products pass 2^31 elements,
and batched calls over more forests than one launch holds."""
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


def random_forest(seed: int, n_trees: int, n_features: int, n_classes: int, depth: int) -> datagen.Forest:
    """Random complete-ish trees (no training): split features and thresholds
    drawn uniformly, each node a leaf with probability 0.1 below level 2."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nb, L, R, Fe, Th, Cl = [0], [], [], [], [], []
    for _ in range(n_trees):
        left, right, feat, thr, cls = [], [], [], [], []

        def node(level):
            i = len(left)
            left.append(-1); right.append(-1); feat.append(-1); thr.append(0.0); cls.append(-1)
            if level == depth or (level > 2 and rng.random() < 0.1):
                cls[i] = int(rng.integers(n_classes))
                return i
            feat[i] = int(rng.integers(n_features))
            thr[i] = float(np.float32(rng.normal()))
            left[i] = node(level + 1)
            right[i] = node(level + 1)
            return i

        node(0)
        L += left; R += right; Fe += feat; Th += thr; Cl += cls
        nb.append(nb[-1] + len(left))
    L = np.array(L, np.int32)
    return datagen.Forest(n_features, n_classes, nb, L, R, Fe, np.array(Th, np.float32), Cl,
                          np.ones(len(L), np.int64))


def test_max_features_and_classes():
    F = random_forest(5, 24, 1024, 512, 9)
    X = np.random.Generator(np.random.PCG64(6)).normal(size=(1500, 1024)).astype(np.float32)
    ref = oracle.predict(F, X, threads=oracle.default_threads())
    # 32-row tiles of 4 KB rows and 512 vote counters per row fill most of
    # shared memory: layouts whose bin blocks still fit
    for params in (dict(bin_size=1, interleave_depth=5), dict(bin_size=4, interleave_depth=4, head_select=3),
                   dict(bin_size=2, interleave_depth=7, bin_buffers=2)):
        df = fp.fp_upload(fp.fp_pack_forest(F, **params))
        Xd = torch.from_numpy(X).cuda()
        votes, cls = df.predict(Xd)
        leaves = df.predict_leaves(Xd)
        torch.cuda.synchronize()
        assert df.sync_status() == fp.FP_OK
        np.testing.assert_array_equal(leaves.cpu().numpy(), ref["leaf"])
        np.testing.assert_array_equal(votes.cpu().numpy().astype(np.uint32), ref["votes"])
        np.testing.assert_array_equal(cls.cpu().numpy(), ref["cls"])
        df.release()


def test_indices_past_two_to_the_31():
    """140 M rows of 16 features: row offsets (n * F = 2.24e9) and vote
    offsets pass 2^31; the last tile's rows and a seeded sample match the
    oracle."""
    F = datagen.forest("tiny")
    n = 140_000_000
    X, _ = datagen.test_rows("tiny", n)
    df = fp.fp_upload(fp.fp_pack_forest(F))
    Xd = torch.from_numpy(X).cuda()
    votes, cls = df.predict(Xd)
    torch.cuda.synchronize()
    assert df.sync_status() == fp.FP_OK
    rng = np.random.Generator(np.random.PCG64(8))
    idx = np.unique(np.concatenate([rng.choice(n, 4000, replace=False), np.arange(n - 3000, n)]))
    ref = oracle.predict(F, X[idx], threads=oracle.default_threads())
    np.testing.assert_array_equal(cls[torch.from_numpy(idx).cuda()].cpu().numpy(), ref["cls"])
    np.testing.assert_array_equal(votes[torch.from_numpy(idx).cuda()].cpu().numpy().astype(np.uint32), ref["votes"])
    df.release()


def test_batched_more_forests_than_one_launch(tiny_forest, tiny_rows):
    """40 (forest, batch) pairs: split into launches of at most 32."""
    X, _ = tiny_rows
    layouts = [dict(bin_size=1 + k % 5, interleave_depth=k % 8, head_select=[0, 1, 3][k % 3]) for k in range(40)]
    forests = [fp.fp_upload(fp.fp_pack_forest(tiny_forest, **p)) for p in layouts]
    Xh = [X[(k * 97) % 5000:][: 1 + (k * 131) % 900] for k in range(40)]
    Xs = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in Xh]
    cls = [torch.empty((x.shape[0],), dtype=torch.int32, device="cuda") for x in Xh]
    fp.fp_predict_batched(forests, Xs, None, cls)
    torch.cuda.synchronize()
    for x, c in zip(Xh, cls):
        np.testing.assert_array_equal(c.cpu().numpy(), oracle.predict(tiny_forest, x)["cls"])
