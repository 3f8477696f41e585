"""The continuous-batching server: requests of different forests and sizes,
arriving from several threads while launches are in flight, each get exactly
the answer they get alone (and the oracle's)."""
import threading

import numpy as np
import pytest

import datagen
import oracle
from paper_1806_07300_gb300.serving import ForestServer, latency_summary

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


@pytest.fixture(scope="module")
def served():
    tiny = datagen.forest("tiny")
    b0 = datagen.forest("batched0")
    b2 = datagen.forest("batched2")
    rows = {"tiny": datagen.test_rows("tiny")[0], "b0": datagen.test_rows("batched0", 20000)[0],
            "b2": datagen.test_rows("batched2", 20000)[0]}
    return {"tiny": tiny, "b0": b0, "b2": b2}, rows


def _server(forests, **kw):
    srv = ForestServer(**kw)
    for name, f in forests.items():
        srv.add_forest(name, f, pass_bytes=(4096 if name == "b2" else 0))
    return srv


def _requests(rows, n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    names = sorted(rows)
    for _ in range(n):
        name = names[rng.integers(len(names))]
        m = int(np.clip(round(rng.lognormal(np.log(32), 1.5)), 1, 4096))
        start = int(rng.integers(0, rows[name].shape[0] - m))
        out.append((name, rows[name][start: start + m]))
    return out


def test_requests_past_stop_and_errors(served):
    """stop() answers every queued request; a wrong forest name or a submit
    after stop is refused; a request larger than max_rows is launched alone."""
    forests, rows = served
    srv = _server(forests, slots=2, max_rows=1000)
    srv.start()
    hs = [srv.submit("tiny", rows["tiny"][i * 50: i * 50 + 50]) for i in range(40)]
    srv.stop()
    for i, h in enumerate(hs):
        assert h.wait(0) and h.error is None and h.latency_s > 0
        np.testing.assert_array_equal(h.classes, oracle.predict(forests["tiny"], rows["tiny"][i * 50: i * 50 + 50],
                                                                leaves=False)["cls"])
    import paper_1806_07300_gb300 as fp
    with pytest.raises(fp.FPError):
        srv.submit("tiny", rows["tiny"][:10])
    with pytest.raises(KeyError):
        srv.submit("nope", rows["tiny"][:10])
    srv.close()
    srv2 = _server(forests, slots=1, max_rows=100).start()
    big = srv2.submit("tiny", rows["tiny"][:1001])
    small = srv2.submit("tiny", rows["tiny"][:7])
    assert big.wait(60) and small.wait(60) and big.error is None and small.error is None
    np.testing.assert_array_equal(big.classes, oracle.predict(forests["tiny"], rows["tiny"][:1001], leaves=False)["cls"])
    assert srv2.launches == 2
    srv2.close()


def test_mix_equals_alone_and_oracle(served):
    forests, rows = served
    reqs = _requests(rows, 300, seed=3)
    with _server(forests, slots=3, max_rows=20000, return_votes=True) as srv:
        handles = [None] * len(reqs)

        def client(lo, hi):
            for i in range(lo, hi):
                handles[i] = srv.submit(*reqs[i])

        ts = [threading.Thread(target=client, args=(k * 100, (k + 1) * 100)) for k in range(3)]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        for h in handles:
            assert h.wait(60) and h.error is None
        assert srv.launches >= 1
    # alone: a fresh server, one request at a time
    with _server(forests, slots=1, return_votes=True) as alone:
        for (name, X), h in zip(reqs[:60], handles[:60]):
            a = alone.submit(name, X)
            assert a.wait(60) and a.error is None
            np.testing.assert_array_equal(a.classes, h.classes)
            np.testing.assert_array_equal(a.votes, h.votes)
    for (name, X), h in zip(reqs, handles):
        ref = oracle.predict(forests[name], X, leaves=False)
        np.testing.assert_array_equal(h.classes, ref["cls"])
        np.testing.assert_array_equal(h.votes.astype(np.uint32), ref["votes"])
    s = latency_summary(handles)
    assert s["n"] == len(reqs) and s["p99_ms"] >= s["p50_ms"] > 0


def test_admission_waits_for_memory(served):
    """With free memory reported too small, launches wait for those in
    flight to finish instead of starting; every request still completes."""
    forests, rows = served
    reqs = _requests(rows, 60, seed=5)
    srv = _server(forests, slots=2, max_rows=1000)
    srv.set_free_bytes(srv.mem_margin - 1)  # never enough: each launch waits until none is in flight
    with srv:
        hs = [srv.submit(*r) for r in reqs]
        for h in hs:
            assert h.wait(60) and h.error is None
    assert srv.rejected_for_memory > 0
    for (name, X), h in zip(reqs, hs):
        np.testing.assert_array_equal(h.classes, oracle.predict(forests[name], X, leaves=False)["cls"])


def test_failed_launch_answers_its_requests(served):
    """A launch whose scratch allocation fails (injected on the host) answers
    its requests with FP_ENOMEM; the server keeps serving the next ones."""
    import paper_1806_07300_gb300 as fp
    forests, rows = served
    with _server(forests, slots=1) as srv:
        first = srv.submit("tiny", rows["tiny"][:40])
        assert first.wait(60) and first.error is None
        fp.fp_inject_fault(srv.forests["tiny"].df, fp.FP_FAULT_ALLOC, 1)
        bad = srv.submit("tiny", rows["tiny"][:40])
        assert bad.wait(60) and bad.error == "FP_ENOMEM"
        good = srv.submit("tiny", rows["tiny"][40:90])
        assert good.wait(60) and good.error is None
        np.testing.assert_array_equal(good.classes, oracle.predict(forests["tiny"], rows["tiny"][40:90],
                                                                   leaves=False)["cls"])


def test_launch_past_its_limit_retires_its_slot(served):
    """A launch still running when the completion poll's limit runs out is
    answered with FP_ETIMEOUT and its slot is retired, never reused while its
    work may still touch the slot's buffers; the other slot keeps serving
    exact answers; with no slot left in service a request is answered with
    FP_ETIMEOUT at once instead of waiting.  The slow launch is made on the
    host side: the forest's bin waits ignore completed copies until their
    bounded poll gives up (the kernel then ends by itself)."""
    import paper_1806_07300_gb300 as fp
    forests, rows = served
    X = rows["tiny"]

    def stall(srv, on):
        df = srv.forests["tiny"].df
        fp.fp_inject_fault(df, fp.FP_FAULT_WAIT_LIMIT, (1 << 18) if on else (1 << 24))
        fp.fp_inject_fault(df, fp.FP_FAULT_STALL_BIN_COPY, 1 if on else 0)
        srv.set_launch_timeout(0.0 if on else 60.0)

    srv = _server(forests, slots=2)
    with srv:
        warm = srv.submit("tiny", X[:64])
        assert warm.wait(60) and warm.error is None
        stall(srv, True)
        slow = srv.submit("tiny", X[:500])
        assert slow.wait(60) and slow.error == "FP_ETIMEOUT"
        assert srv.slots_in_service == 1
        stall(srv, False)
        good = [srv.submit("tiny", X[i * 100: (i + 1) * 100]) for i in range(20)]
        for i, h in enumerate(good):
            assert h.wait(60) and h.error is None
            np.testing.assert_array_equal(h.classes, oracle.predict(forests["tiny"], X[i * 100: (i + 1) * 100],
                                                                    leaves=False)["cls"])
        assert srv.slots_in_service == 1
    srv.forests["tiny"].df.sync_status()  # the slow kernel recorded its timeout; clear it
    srv.close()

    one = _server(forests, slots=1)
    with one:
        stall(one, True)
        slow = one.submit("tiny", X[:500])
        assert slow.wait(60) and slow.error == "FP_ETIMEOUT"
        assert one.slots_in_service == 0
        stall(one, False)
        after = one.submit("tiny", X[:10])
        assert after.wait(60) and after.error == "FP_ETIMEOUT"
    one.forests["tiny"].df.sync_status()
    one.close()
