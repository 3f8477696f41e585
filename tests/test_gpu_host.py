"""GPU parity for the host-buffer entry points (fp_predict_host,
fp_predict_values_host): rows in host memory go through the device in
chunks, copies on a copy stream overlapping the kernels, which alternate
between the caller's stream and a second library stream.  Classes, votes
and leaf-value outputs must equal the oracle's (bit for bit; values within
the float32 bound) for every chunking, including ragged last chunks, single
rows and pageable inputs, once the caller's stream alone is synchronised."""
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


@pytest.fixture(scope="module")
def tiny_df(tiny_forest):
    df = fp.fp_upload(fp.fp_pack_forest(tiny_forest, pass_bytes=8192))  # several passes
    assert df.info["passes"] > 1
    yield df
    df.release()


@pytest.mark.parametrize("n,chunk", [(10000, 0), (10000, 1000), (10000, 3333), (10000, 10000), (9999, 4096),
                                     (1, 0), (37, 8)])
def test_host_classes_and_votes(tiny_forest, tiny_rows, tiny_df, n, chunk):
    X = np.ascontiguousarray(tiny_rows[0][:n])
    ref = oracle.predict(tiny_forest, X)
    Xp = torch.from_numpy(X).pin_memory()
    votes = torch.empty((n, tiny_forest.n_classes), dtype=torch.int32).pin_memory()
    cls = torch.empty((n,), dtype=torch.int32).pin_memory()
    s = torch.cuda.current_stream()
    fp.fp_predict_host(tiny_df, Xp, votes, cls, chunk, s)
    s.synchronize()
    assert tiny_df.sync_status() == fp.FP_OK
    np.testing.assert_array_equal(cls.numpy(), ref["cls"])
    np.testing.assert_array_equal(votes.numpy().astype(np.uint32), ref["votes"])


@pytest.mark.parametrize("chunk", [0, 613])
def test_host_on_a_nonblocking_stream(tiny_forest, tiny_rows, tiny_df, chunk):
    """On a stream of the caller's own that does not synchronise with the
    legacy default stream: waiting for that stream alone covers every
    chunk's kernel and copies, those on the library's second stream too;
    then the same buffers are reused at once."""
    X = np.ascontiguousarray(tiny_rows[0][:9000])
    ref = oracle.predict(tiny_forest, X)
    Xp = torch.from_numpy(X).pin_memory()
    s = torch.cuda.Stream()
    for rep in range(2):
        votes = torch.full((9000, tiny_forest.n_classes), -1, dtype=torch.int32).pin_memory()
        cls = torch.full((9000,), -1, dtype=torch.int32).pin_memory()
        fp.fp_predict_host(tiny_df, Xp, votes, cls, chunk, s)
        s.synchronize()
        np.testing.assert_array_equal(cls.numpy(), ref["cls"])
        np.testing.assert_array_equal(votes.numpy().astype(np.uint32), ref["votes"])


def test_host_pageable_numpy_and_method(tiny_forest, tiny_rows, tiny_df):
    X = np.ascontiguousarray(tiny_rows[0][:5000])
    ref = oracle.predict(tiny_forest, X)
    cls = np.empty(5000, np.int32)
    s = torch.cuda.current_stream()
    fp.fp_predict_host(tiny_df, X, None, cls, 1024, s)  # ordinary host memory
    s.synchronize()
    np.testing.assert_array_equal(cls, ref["cls"])
    v, c = tiny_df.predict_host(torch.from_numpy(X), votes=True, chunk_rows=700)
    np.testing.assert_array_equal(c.numpy(), ref["cls"])
    np.testing.assert_array_equal(v.numpy().astype(np.uint32), ref["votes"])


def test_host_three_and_two_level_super_nodes(tiny_forest, tiny_rows):
    X = np.ascontiguousarray(tiny_rows[0])
    ref = oracle.predict(tiny_forest, X)
    for dl in (2, 3):
        df = fp.fp_upload(fp.fp_pack_forest(tiny_forest, bin_size=4, interleave_depth=2, deep_levels=dl))
        _, c = df.predict_host(torch.from_numpy(X).pin_memory(), chunk_rows=2048)
        np.testing.assert_array_equal(c.numpy(), ref["cls"])
        df.release()


def test_host_hbm_rows_match_device_path():
    """500,000 rows of the HBM-resident workload: the host path in 8 chunks
    (two compute streams, five passes each) gives the classes of the device
    path; a sample equals the oracle."""
    forest = datagen.forest("hbm")
    X, _ = datagen.test_rows("hbm", 500000)
    df = fp.fp_upload(fp.fp_pack_forest(forest))
    _, c_dev = df.predict(torch.from_numpy(X).cuda(), votes=False)
    _, c_host = df.predict_host(torch.from_numpy(X).pin_memory())
    torch.cuda.synchronize()
    np.testing.assert_array_equal(c_host.numpy(), c_dev.cpu().numpy())
    idx = np.random.default_rng(7).choice(500000, 3000, replace=False)
    idx[-1] = 499999
    np.testing.assert_array_equal(c_host.numpy()[idx], oracle.predict(forest, X[idx], threads=4)["cls"])
    df.release()


def test_host_values():
    X, y = datagen.gen_regression(41, 8000, 0, 1.0, 1.0)
    F = datagen.train_regression(X, y, 12, mtry=9, min_leaf=3, seed=41)
    Xt, _ = datagen.gen_regression(41, 7001, 1, 1.0, 1.0)
    ref = oracle.predict_values(F, Xt)
    df = fp.fp_upload(fp.fp_pack_forest(F, pass_bytes=65536))
    for chunk in (0, 1000, 7001):
        out = torch.empty((7001,), dtype=torch.float32).pin_memory()
        s = torch.cuda.current_stream()
        fp.fp_predict_values_host(df, torch.from_numpy(Xt).pin_memory(), out, df.value_scale, df.value_bias, chunk, s)
        s.synchronize()
        err = np.abs(out.numpy().astype(np.float64) - ref["out"])
        assert np.all(err <= oracle.value_tolerance(F, ref["abs"]))
    assert np.all(np.abs(df.predict_host(Xt, chunk_rows=3000).numpy() - ref["out"])
                  <= oracle.value_tolerance(F, ref["abs"]))
    df.release()


def test_host_errors(tiny_forest, tiny_df):
    X = np.zeros((4, tiny_forest.n_features), np.float32)
    out = np.zeros(4, np.float32)
    cls = np.zeros(4, np.int32)
    with pytest.raises(fp.FPError) as e:  # a classification forest has no leaf values
        fp.fp_predict_values_host(tiny_df, X, out, 1.0, 0.0)
    assert e.value.code == fp.FP_EINVAL
    with pytest.raises(fp.FPError) as e:
        fp.fp_predict_host(tiny_df, X, None, cls, -1)
    assert e.value.code == fp.FP_EINVAL
    with pytest.raises(TypeError):
        fp.fp_predict_host(tiny_df, torch.zeros((4, tiny_forest.n_features), device="cuda"), None, cls)
    fp.fp_predict_host(tiny_df, np.zeros((0, tiny_forest.n_features), np.float32), None, np.zeros(0, np.int32))


def test_host_allocation_failure_then_recovery(tiny_forest, tiny_rows, tiny_df):
    """An injected failure of the pipeline's device allocation returns
    FP_ENOMEM and leaves nothing behind; the next call classifies correctly."""
    X = torch.from_numpy(np.ascontiguousarray(tiny_rows[0][:3000])).pin_memory()
    cls = torch.empty((3000,), dtype=torch.int32).pin_memory()
    s = torch.cuda.current_stream()
    fp.fp_inject_fault(tiny_df, fp.FP_FAULT_ALLOC, 1)
    with pytest.raises(fp.FPError) as e:
        fp.fp_predict_host(tiny_df, X, None, cls, 1000, s)
    assert e.value.code == fp.FP_ENOMEM
    fp.fp_predict_host(tiny_df, X, None, cls, 1000, s)
    s.synchronize()
    np.testing.assert_array_equal(cls.numpy(), oracle.predict(tiny_forest, X.numpy())["cls"])
