"""GPU parity on random forests with adversarial thresholds (signed zeros,
subnormals, huge magnitudes, infinities, NaN) and rows on those thresholds
and their float neighbours: leaf ids, votes and classes of fp_predict and
fp_predict_leaves equal the oracle's for every kind of super-node and head,
alone and in one batched launch that mixes the kinds."""
import numpy as np
import pytest

import oracle
import paper_1806_07300_gb300 as fp
import random_forests as rf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KINDS = [(2, 0), (3, 1), (3, 2)]
CASES = [(1, "mixed"), (2, "mixed"), (3, "positive"), (4, "narrow")]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


@pytest.mark.parametrize("seed,kind", CASES)
@pytest.mark.parametrize("dl,fmt", KINDS)
@pytest.mark.parametrize("B,d,sel", [(4, 3, 2), (3, 2, 1), (2, 3, 3)])
def test_random_forest_on_gpu(seed, kind, dl, fmt, B, d, sel):
    f = rf.forest(seed, kind=kind)
    X = rf.rows(f, 6000, seed + 100, kind)
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


def test_random_forests_batched_mixed_kinds():
    """Six random forests, each with its own kind of super-node and remap,
    in one persistent launch."""
    specs = [(1, "mixed", 3, 2), (3, "positive", 3, 2), (4, "narrow", 3, 1), (2, "mixed", 2, 0),
             (5, "positive", 3, 1), (6, "narrow", 3, 2)]
    dfs, Xs, refs = [], [], []
    for i, (seed, kind, dl, fmt) in enumerate(specs):
        f = rf.forest(seed, kind=kind)
        X = rf.rows(f, 500 + 997 * i, seed + 200, kind)
        refs.append(oracle.predict(f, X))
        dfs.append(fp.fp_upload(fp.fp_pack_forest(f, bin_size=3, interleave_depth=3, head_select=2, deep_levels=dl,
                                                  deep_format=fmt)))
        Xs.append(torch.from_numpy(X).cuda())
    votes = [torch.empty((x.shape[0], 5), dtype=torch.int32, device="cuda") for x in Xs]
    cls = [torch.empty((x.shape[0],), dtype=torch.int32, device="cuda") for x in Xs]
    fp.fp_predict_batched(dfs, Xs, votes, cls)
    torch.cuda.synchronize()
    for d, v, c, r in zip(dfs, votes, cls, refs):
        assert d.sync_status() == fp.FP_OK
        np.testing.assert_array_equal(v.cpu().numpy().astype(np.uint32), r["votes"])
        np.testing.assert_array_equal(c.cpu().numpy(), r["cls"])
        d.release()
