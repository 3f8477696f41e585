"""GPU parity for forests with real leaf values (regression and boosted trees).

The leaf each observation reaches in each tree must equal the oracle's (bit
for bit); the output bias + scale * sum of leaf values is computed in
float32 with additions in no fixed order, so it must lie within the bound
oracle.value_tolerance derives from the arithmetic: (T + 2) * 2^-24 *
(|bias| + |scale| * sum |value|) per row.  The hand-worked fixture, whose
values are short binary fractions, must match exactly."""
import numpy as np
import pytest

import datagen
import oracle
import paper_1806_07300_gb300 as fp
from golden_io import load_values

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


@pytest.fixture(scope="module")
def small_regress():
    X, y = datagen.gen_regression(31, 20000, 0, 1.0, 1.0)
    F = datagen.train_regression(X, y, 24, mtry=9, min_leaf=3, seed=31)
    Xt, _ = datagen.gen_regression(31, 9000, 1, 1.0, 1.0)
    return F, Xt, oracle.predict_values(F, Xt, threads=oracle.default_threads())


def _check(F, X, ref, exact=False, **params):
    df = fp.fp_upload(fp.fp_pack_forest(F, **params))
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    out = df.predict_values(Xd)
    leaves = df.predict_leaves(Xd)
    torch.cuda.synchronize()
    assert df.sync_status() == fp.FP_OK
    np.testing.assert_array_equal(leaves.cpu().numpy(), ref["leaf"])
    got = out.cpu().numpy().astype(np.float64)
    if exact:
        np.testing.assert_array_equal(got, ref["out"])
    err = np.abs(got - ref["out"])
    tol = oracle.value_tolerance(F, ref["abs"])
    assert np.all(err <= tol), f"max error {err.max()} over bound at row {int(np.argmax(err - tol))}"
    df.release()
    return got


@pytest.mark.parametrize("B,d,sel", [(1, 0, 3), (2, 1, 1), (3, 3, 3), (1, 2, 1), (3, 9, 0)])
@pytest.mark.parametrize("dl,fmt", [(2, 0), (3, 1), (3, 2)])
def test_values_fixture_on_gpu(B, d, sel, dl, fmt):
    F, X, exp = load_values("values_small.txt")
    ref = oracle.predict_values(F, X)
    _check(F, X, ref, exact=True, bin_size=B, interleave_depth=d, head_select=sel, deep_levels=dl, deep_format=fmt)


@pytest.mark.parametrize("params", [dict(bin_size=4, interleave_depth=9, head_select=1),
                                    dict(bin_size=8, interleave_depth=5, head_select=1, bin_buffers=2),
                                    dict(bin_size=3, interleave_depth=8, head_select=3),
                                    dict(bin_size=4, interleave_depth=9, head_select=2, bin_buffers=2),
                                    dict(bin_size=2, interleave_depth=4, head_select=1, pass_bytes=65536),
                                    dict(bin_size=1, interleave_depth=6, head_select=3, pass_bytes=1,
                                         obs_tile=128),
                                    dict(bin_size=4, interleave_depth=9, head_select=2, deep_levels=2),
                                    dict(bin_size=2, interleave_depth=4, head_select=1, pass_bytes=65536,
                                         deep_levels=2),
                                    dict(bin_size=4, interleave_depth=9, head_select=2, deep_format=2),
                                    dict(bin_size=2, interleave_depth=4, head_select=1, pass_bytes=65536,
                                         deep_format=2)])
def test_regression_forest_layouts(small_regress, params):
    F, X, ref = small_regress
    if "pass_bytes" in params:
        assert fp.fp_pack_forest(F, **params).info()["passes"] > 1
    _check(F, X, ref, **params)


def test_scale_and_bias_arguments(small_regress):
    F, X, ref = small_regress
    df = fp.fp_upload(fp.fp_pack_forest(F, bin_size=4, interleave_depth=6, head_select=1))
    Xd = torch.from_numpy(X).cuda()
    out = df.predict_values(Xd, scale=1.0, bias=0.0)  # the plain sum
    torch.cuda.synchronize()
    tol = (F.n_trees + 2) * 2.0 ** -24 * ref["abs"] * 1.01
    assert np.all(np.abs(out.cpu().numpy() - ref["sum"]) <= tol)


def test_empty_batch_and_wrong_forest_kind(small_regress, tiny_forest):
    F, X, _ = small_regress
    df = fp.fp_upload(fp.fp_pack_forest(F))
    out = df.predict_values(torch.empty((0, F.n_features), dtype=torch.float32, device="cuda"))
    assert out.shape == (0,)
    Xd = torch.from_numpy(X[:10]).cuda()
    with pytest.raises(fp.FPError) as e:
        df.predict(Xd)
    assert e.value.code == fp.FP_EINVAL
    cf = fp.fp_upload(fp.fp_pack_forest(tiny_forest))
    with pytest.raises(fp.FPError) as e:
        fp.fp_predict_values(cf, torch.zeros((4, tiny_forest.n_features), device="cuda"),
                             torch.empty(4, device="cuda"), 1.0, 0.0)
    assert e.value.code == fp.FP_EINVAL


@pytest.mark.parametrize("order", [fp.FP_PLAIN_OBS_FASTEST, fp.FP_PLAIN_TREE_FASTEST])
def test_plain_baseline_values(small_regress, order):
    F, X, ref = small_regress
    pf = fp.fp_plain_build(F)
    out = pf.predict_values(torch.from_numpy(X).cuda(), order)
    torch.cuda.synchronize()
    err = np.abs(out.cpu().numpy().astype(np.float64) - ref["out"])
    assert np.all(err <= oracle.value_tolerance(F, ref["abs"]))
    pf.release()


@pytest.mark.parametrize("name,layout", [("boosted", dict(bin_size=16, interleave_depth=5, head_select=1)),
                                         ("boosted", dict(bin_size=64, interleave_depth=5, head_select=2)),
                                         ("boosted", dict(bin_size=32, interleave_depth=3, head_select=3)),
                                         ("regress", dict(bin_size=4, interleave_depth=9, head_select=1))])
def test_value_workloads(name, layout):
    """The benchmark's value workloads, on 50,000 of their test rows."""
    F = datagen.forest(name)
    X, _ = datagen.test_rows(name, 50000)
    _check(F, X, oracle.predict_values(F, X, threads=oracle.default_threads()), **layout)
