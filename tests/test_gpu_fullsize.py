"""Full-size parity at the launch configurations bench.py times.

The HBM-resident workload (256 trees, 4,000,000 rows) runs in every layout and
launch the benchmark's autotuner may pick, and the image-shaped workload (128
trees, 1,000,000 rows) in the library defaults and the tuner's candidates.
Every row's votes and class are compared element by element with the oracle's
(computed once per workload on all host cores: about 80 s for the 4,000,000
HBM rows), and a seeded sample of rows also by per-tree leaf id."""
import numpy as np
import pytest

import datagen
import oracle
import paper_1806_07300_gb300 as fp
from bench import HBM_LAUNCHES, HBM_LAYOUTS, TUNE
from paper_1806_07300_gb300 import autotune as at

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SAMPLE = 20000


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


_DATA = {}


def _data(name, n):
    if name not in _DATA:
        _DATA.clear()
        X, _ = datagen.test_rows(name, n)
        _DATA[name] = (datagen.forest(name), X, torch.from_numpy(X).cuda())
    return _DATA[name]


_REF = {}


def _run(name, n, layout=None, launches=(None,)):
    forest, X, Xd = _data(name, n)
    params = {}
    if layout is not None:
        params = dict(zip(at.LAYOUT_KEYS, layout))
    df = fp.fp_upload(fp.fp_pack_forest(forest, **params))
    for launch in launches:
        if launch is not None:
            df.configure(**dict(zip(at.LAUNCH_KEYS, launch)))
        _check(df, forest, X, Xd, n)
    df.release()


def _check(df, forest, X, Xd, n):
    votes, cls = df.predict(Xd)
    torch.cuda.synchronize()
    assert df.sync_status() == fp.FP_OK
    v = votes.cpu().numpy().astype(np.uint32)
    c = cls.cpu().numpy()
    rng = np.random.Generator(np.random.PCG64(1234))
    idx = np.sort(rng.choice(n, size=min(SAMPLE, n), replace=False))
    idx[-1] = n - 1  # include the ragged last tile
    key = (id(forest), n)
    if key not in _REF:
        _REF.clear()
        full = oracle.predict(forest, X, leaves=False, threads=oracle.default_threads())
        sample = oracle.predict(forest, X[idx], votes=False, classes=False, threads=oracle.default_threads())
        _REF[key] = (full, sample["leaf"])
    ref, ref_leaf = _REF[key]
    # every row, element by element
    np.testing.assert_array_equal(v, ref["votes"])
    np.testing.assert_array_equal(c, ref["cls"])
    leaves = df.predict_leaves(torch.from_numpy(np.ascontiguousarray(X[idx])).cuda())
    torch.cuda.synchronize()
    np.testing.assert_array_equal(leaves.cpu().numpy(), ref_leaf)


@pytest.mark.parametrize("layout", HBM_LAYOUTS)
def test_hbm_workload_full_size(layout):
    _run("hbm", datagen.RECIPES["hbm"]["n_test"], layout, HBM_LAUNCHES)


@pytest.mark.parametrize("layout", [None, (2, 8, 3)] + list(TUNE["image"][0]))
def test_image_workload_full_size(layout):
    """The library defaults, a ranked-head layout, and every layout and launch
    the benchmark's tuner may pick for this workload."""
    _run("image", datagen.RECIPES["image"]["n_test"], layout,
         TUNE["image"][1] if layout in TUNE["image"][0] else (None,))


def _run_values(name, layout, launch):
    """Value workloads at full size: every row's output is finite, a seeded
    sample matches the oracle within the float32 bound, leaves exactly."""
    forest, X, Xd = _data(name, datagen.RECIPES[name]["n_test"])
    n = X.shape[0]
    df = fp.fp_upload(fp.fp_pack_forest(forest, **dict(zip(at.LAYOUT_KEYS, layout))))
    df.configure(**dict(zip(at.LAUNCH_KEYS, launch)))
    out = df.predict_values(Xd)
    torch.cuda.synchronize()
    assert df.sync_status() == fp.FP_OK
    o = out.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(o))
    rng = np.random.Generator(np.random.PCG64(4321))
    idx = np.sort(rng.choice(n, size=min(SAMPLE, n), replace=False))
    idx[-1] = n - 1
    ref = oracle.predict_values(forest, X[idx], threads=oracle.default_threads())
    assert np.all(np.abs(o[idx] - ref["out"]) <= oracle.value_tolerance(forest, ref["abs"]))
    leaves = df.predict_leaves(torch.from_numpy(np.ascontiguousarray(X[idx])).cuda())
    torch.cuda.synchronize()
    np.testing.assert_array_equal(leaves.cpu().numpy(), ref["leaf"])
    df.release()


@pytest.mark.parametrize("name", ["regress", "boosted"])
def test_value_workloads_full_size(name):
    from bench import TUNE
    layouts, launches = TUNE[name]
    for layout in layouts[:2]:
        for launch in launches[:2]:
            _run_values(name, layout, launch)
