"""Many resident forests at once, as a serving process holds them: every kind
of super-node and head, tiles and CTA sizes that differ (so forests share
compiled kernels with different shared-memory needs), classification,
parity leaves and leaf values in a shuffled order, launch parameters
changed between rounds, and forests launched side by side on two streams.
Every output equals the oracle's (values within the float32 bound)."""
import numpy as np
import pytest

import datagen
import oracle
import paper_1806_07300_gb300 as fp
import random_forests as rf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _specs(tiny_forest):
    out = []
    for i, (dl, fmt, sel, d) in enumerate([(3, 1, 2, 3), (3, 2, 2, 3), (2, 0, 1, 2), (3, 1, 3, 4), (3, 2, 1, 4)]):
        out.append(("tiny", tiny_forest, dict(bin_size=2 + i, interleave_depth=d, head_select=sel, deep_levels=dl,
                                              deep_format=fmt)))
    for seed, kind, fmt in [(11, "mixed", 2), (12, "positive", 2), (13, "narrow", 1)]:
        out.append((f"random{seed}", rf.forest(seed, kind=kind), dict(bin_size=3, interleave_depth=3, deep_format=fmt)))
    Xr, yr = datagen.gen_regression(43, 3000, 0, 1.0, 1.0)
    out.append(("regression", datagen.train_regression(Xr, yr, 6, mtry=9, min_leaf=3, seed=43), dict(bin_size=2)))
    return out


def _rows(name, f, tiny_rows):
    if name == "tiny":
        return np.ascontiguousarray(tiny_rows[0][:4099])
    if name == "regression":
        return datagen.gen_regression(43, 3001, 1, 1.0, 1.0)[0]
    return rf.rows(f, 3001, 7, "mixed" if name == "random11" else ("positive" if name == "random12" else "narrow"))


LAUNCHES = [(1024, 32, 32, 3), (64, 32, 16, 2), (256, 16, 8, 3), (128, 24, 24, 2), (32, 8, 4, 3)]


def test_many_resident_forests(tiny_forest, tiny_rows):
    rng = np.random.default_rng(5)
    res = []
    for k, (name, f, params) in enumerate(_specs(tiny_forest)):
        df = fp.fp_upload(fp.fp_pack_forest(f, **params))
        tile, warps, refill, nbuf = LAUNCHES[k % len(LAUNCHES)]
        df.configure(obs_tile=tile, warps_per_cta=warps, refill_lanes=refill, bin_buffers=nbuf)
        X = _rows(name, f, tiny_rows)
        values = getattr(f, "leaf_value", None) is not None
        ref = oracle.predict_values(f, X) if values else oracle.predict(f, X)
        res.append((name, f, df, torch.from_numpy(X).cuda(), ref, values))

    def check(item, stream=None):
        name, f, df, Xd, ref, values = item
        if values:
            out = df.predict_values(Xd, stream=stream)
            leaves = df.predict_leaves(Xd, stream=stream)

            def verify_values():
                np.testing.assert_array_equal(leaves.cpu().numpy(), ref["leaf"], err_msg=name)
                err = np.abs(out.cpu().numpy().astype(np.float64) - ref["out"])
                assert np.all(err <= oracle.value_tolerance(f, ref["abs"])), name
            return verify_values
        votes, cls = df.predict(Xd, stream=stream)
        leaves = df.predict_leaves(Xd, stream=stream)
        return lambda: (np.testing.assert_array_equal(votes.cpu().numpy().astype(np.uint32), ref["votes"], err_msg=name),
                        np.testing.assert_array_equal(cls.cpu().numpy(), ref["cls"], err_msg=name),
                        np.testing.assert_array_equal(leaves.cpu().numpy(), ref["leaf"], err_msg=name))

    for rnd in range(3):
        for i in rng.permutation(len(res)):
            verify = check(res[i])
            torch.cuda.synchronize()
            verify()
        # side by side on two streams, then new launch parameters for some forests
        s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
        pending = []
        for j, i in enumerate(rng.permutation(len(res))):
            s = s1 if j % 2 else s2
            with torch.cuda.stream(s):
                pending.append(check(res[i], stream=s))
        torch.cuda.synchronize()
        for verify in pending:
            verify()
        for i in rng.choice(len(res), 4, replace=False):
            tile, warps, refill, nbuf = LAUNCHES[int(rng.integers(len(LAUNCHES)))]
            res[i][2].configure(obs_tile=tile, warps_per_cta=warps, refill_lanes=refill, bin_buffers=nbuf)
    for item in res:
        assert item[2].sync_status() == fp.FP_OK
        item[2].release()
