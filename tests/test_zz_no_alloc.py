"""fp_predict_noalloc against fp_predict, through the C ABI.

The allocation-free entry point exists for callers that cannot allocate
device memory while they classify (a fixed device-memory budget, an
allocator lock held, or no driver allocation path allowed).  Its scratch is
a fixed device array inside the library instead of the stream-ordered pool.
This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process (the
first call on the device sets the array up)."""
import ctypes

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


def _call(df, X, votes, cls):
    """fp_predict_noalloc straight through the C ABI."""
    L = fp.lib()
    stream = torch.cuda.current_stream().cuda_stream
    rc = L.fp_predict_noalloc(df.handle, ctypes.c_void_p(X.data_ptr()), X.shape[0],
                              ctypes.c_void_p(votes.data_ptr()) if votes is not None else None,
                              ctypes.c_void_p(cls.data_ptr()) if cls is not None else None,
                              ctypes.c_void_p(stream))
    return rc


@pytest.mark.parametrize("pass_bytes", [2048, -1])
@pytest.mark.parametrize("deep_format", [1, 2])
def test_noalloc_matches_fp_predict_twice(pass_bytes, deep_format):
    """Two calls in a row give exactly fp_predict's votes and classes, and
    the oracle's, with scratch in use (several passes) and without (one
    pass), for three-level super-nodes of either format."""
    X, y = datagen.rows("tiny", 0)
    forest = datagen.train_forest(X, y, 4, 16, 4, seed=0)
    pk = fp.fp_pack_forest(forest, bin_size=2, interleave_depth=2, pass_bytes=pass_bytes, obs_tile=128,
                           deep_format=deep_format)
    assert pk.info()["deep_format"] == deep_format
    assert (pk.info()["passes"] > 1) == (pass_bytes > 0)
    df = fp.fp_upload(pk)
    Xt, _ = datagen.test_rows("tiny", 3001)
    Xd = torch.from_numpy(Xt).cuda()
    n, C = Xt.shape[0], forest.n_classes
    ref_v = torch.empty((n, C), dtype=torch.int32, device="cuda")
    ref_c = torch.empty((n,), dtype=torch.int32, device="cuda")
    fp.fp_predict(df, Xd, ref_v, ref_c)
    torch.cuda.synchronize()
    want = oracle.predict(forest, Xt, leaves=False)
    np.testing.assert_array_equal(ref_v.cpu().numpy().astype(np.uint32), want["votes"])
    np.testing.assert_array_equal(ref_c.cpu().numpy(), want["cls"])
    for _ in range(2):
        v = torch.full((n, C), -1, dtype=torch.int32, device="cuda")
        c = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        c_only = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        assert _call(df, Xd, v, c) == fp.FP_OK
        assert _call(df, Xd, None, c_only) == fp.FP_OK  # accumulator in the fixed array
        torch.cuda.synchronize()
        assert df.sync_status() == fp.FP_OK
        assert torch.equal(v, ref_v)
        assert torch.equal(c, ref_c)
        assert torch.equal(c_only, ref_c)
    df.release()


def test_noalloc_rejects_oversized_scratch():
    """A batch whose scratch would exceed the fixed array is refused before
    anything is enqueued."""
    X, y = datagen.rows("tiny", 0)
    forest = datagen.train_forest(X, y, 4, 16, 4, seed=0)
    df = fp.fp_upload(fp.fp_pack_forest(forest, bin_size=2, interleave_depth=2, pass_bytes=2048))
    Xd = torch.zeros((8, forest.n_features), dtype=torch.float32, device="cuda")
    c = torch.empty((8,), dtype=torch.int32, device="cuda")
    L = fp.lib()
    huge = (16 << 20) // (4 * forest.n_classes) + 4096  # rows whose accumulator alone exceeds 16 MiB
    rc = L.fp_predict_noalloc(df.handle, ctypes.c_void_p(Xd.data_ptr()), huge, None,
                              ctypes.c_void_p(c.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == fp.FP_EINVAL
    assert "scratch" in fp.fp_last_error()
    torch.cuda.synchronize()
    df.release()
