"""Failure detection on the device without faulting it.

The library's error paths run through fp_inject_fault: allocations that fail
(FP_ENOMEM from fp_upload and from per-call scratch), and bin-block waits that
run out (a flag makes the waits ignore completed copies, so the bounded poll
expires; the kernel records FP_ETIMEOUT in the forest's status word, lets its
own copies land and returns).  Each test then checks that the context is
still usable: the next call on the same forest gives the oracle's answers."""
import numpy as np
import pytest

import oracle
import paper_1806_07300_gb300 as fp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


@pytest.fixture(autouse=True)
def _clear_injection():
    yield
    fp.fp_inject_fault(None, fp.FP_FAULT_ALLOC, 0)


def _rows(tiny_rows, n):
    X, _ = tiny_rows
    return X[:n], torch.from_numpy(np.ascontiguousarray(X[:n])).cuda()


def test_injected_upload_allocation_failure(tiny_forest):
    pf = fp.fp_pack_forest(tiny_forest, bin_size=4, interleave_depth=3)
    fp.fp_inject_fault(None, fp.FP_FAULT_ALLOC, 1)
    with pytest.raises(fp.FPError) as e:
        fp.fp_upload(pf)
    assert e.value.code == fp.FP_ENOMEM
    df = fp.fp_upload(pf)  # the injection was used up
    assert df.sync_status() == fp.FP_OK
    df.release()


def test_injected_scratch_allocation_failure(tiny_forest, tiny_rows):
    """A forest swept in several passes needs scratch for a classes-only call."""
    Xh, Xd = _rows(tiny_rows, 3000)
    df = fp.fp_upload(fp.fp_pack_forest(tiny_forest, bin_size=2, interleave_depth=2, pass_bytes=2048))
    assert df.info["passes"] > 1
    fp.fp_inject_fault(None, fp.FP_FAULT_ALLOC, 1)
    with pytest.raises(fp.FPError) as e:
        df.predict(Xd, votes=False)
    assert e.value.code == fp.FP_ENOMEM
    _, c = df.predict(Xd, votes=False)
    assert df.sync_status() == fp.FP_OK
    np.testing.assert_array_equal(c.cpu().numpy(), oracle.predict(tiny_forest, Xh)["cls"])


@pytest.mark.parametrize("params", [dict(bin_size=4, interleave_depth=3),
                                    dict(bin_size=2, interleave_depth=2, pass_bytes=2048),
                                    dict(bin_size=4, interleave_depth=3, deep_format=2),
                                    dict(bin_size=4, interleave_depth=3, deep_levels=2)])
def test_stalled_bin_copy_times_out_and_recovers(tiny_forest, tiny_rows, params):
    """Every kind of super-node has its own compiled walk, each with the
    bounded bin wait: three-level of format 1 (the default here), of format
    2, and two-level."""
    Xh, Xd = _rows(tiny_rows, 5000)
    df = fp.fp_upload(fp.fp_pack_forest(tiny_forest, **params))
    fp.fp_inject_fault(df, fp.FP_FAULT_WAIT_LIMIT, 4096)
    fp.fp_inject_fault(df, fp.FP_FAULT_STALL_BIN_COPY, 1)
    df.predict(Xd)
    assert df.sync_status() == fp.FP_ETIMEOUT
    assert df.sync_status() == fp.FP_OK  # reading the status clears it
    df.predict_leaves(Xd)
    assert df.sync_status() == fp.FP_ETIMEOUT
    fp.fp_inject_fault(df, fp.FP_FAULT_STALL_BIN_COPY, 0)
    v, c = df.predict(Xd)
    assert df.sync_status() == fp.FP_OK
    ref = oracle.predict(tiny_forest, Xh)
    np.testing.assert_array_equal(v.cpu().numpy().astype(np.uint32), ref["votes"])
    np.testing.assert_array_equal(c.cpu().numpy(), ref["cls"])
    df.release()


@pytest.mark.parametrize("fmt_good,fmt_bad", [(0, 0), (1, 2)])
def test_stalled_forest_in_a_batched_launch(tiny_forest, tiny_rows, fmt_good, fmt_bad):
    """A stalled forest after a healthy one in one launch: the stalled
    forest's status records the timeout.  Work items are handed out batch by
    batch, so every item of the healthy forest was claimed before the first
    stalled item aborted a CTA; the healthy forest's status stays clean.  (A
    CTA that aborted records the timeout in the status of every later item it
    skips, whichever forest the item belongs to.)  With formats 1 and 2 the
    launch compiles in both walks."""
    Xh, Xd = _rows(tiny_rows, 2000)
    good = fp.fp_upload(fp.fp_pack_forest(tiny_forest, bin_size=8, interleave_depth=2, deep_format=fmt_good))
    bad = fp.fp_upload(fp.fp_pack_forest(tiny_forest, bin_size=8, interleave_depth=2, deep_format=fmt_bad))
    fp.fp_inject_fault(bad, fp.FP_FAULT_WAIT_LIMIT, 4096)
    fp.fp_inject_fault(bad, fp.FP_FAULT_STALL_BIN_COPY, 1)
    cls = [torch.empty((2000,), dtype=torch.int32, device="cuda") for _ in range(2)]
    fp.fp_predict_batched([good, bad], [Xd, Xd], None, cls)
    assert bad.sync_status() == fp.FP_ETIMEOUT
    assert good.sync_status() == fp.FP_OK
    fp.fp_inject_fault(bad, fp.FP_FAULT_STALL_BIN_COPY, 0)
    fp.fp_predict_batched([good, bad], [Xd, Xd], None, cls)
    assert bad.sync_status() == fp.FP_OK
    ref = oracle.predict(tiny_forest, Xh)["cls"]
    for c in cls:
        np.testing.assert_array_equal(c.cpu().numpy(), ref)


def test_inject_fault_rejects_bad_arguments(tiny_forest):
    df = fp.fp_upload(fp.fp_pack_forest(tiny_forest))
    for forest, kind, value in [(df, 99, 1), (df, fp.FP_FAULT_WAIT_LIMIT, 0), (df, fp.FP_FAULT_WAIT_LIMIT, 1 << 25),
                                (None, fp.FP_FAULT_WAIT_LIMIT, 10), (df, fp.FP_FAULT_STALL_BIN_COPY, 2),
                                (None, fp.FP_FAULT_ALLOC, -1)]:
        with pytest.raises(fp.FPError) as e:
            fp.fp_inject_fault(forest, kind, value)
        assert e.value.code == fp.FP_EINVAL
    df.release()
