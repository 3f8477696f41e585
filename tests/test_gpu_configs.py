"""Parity on the benchmark workloads' own forests through every classification
entry point (Section III-A: a layout must not change any prediction).

- the serving workload's fourth forest (64 trees, 50 classes, 100 features)
  through fp_predict and fp_predict_leaves, every test row;
- the HBM-resident forest (several passes, three-level super-nodes), the
  image-shaped forest (784 features, two-level super-nodes) and the wide
  forest in ONE fp_predict_batched launch, captured in a CUDA graph and
  replayed on new rows;
- the serving workload's four forests (tiny, image, hbm, wide) behind the
  continuous-batching server: each request's answer is the same alone and in
  the mix, and equals the oracle's.
Votes, classes and leaf ids are compared element by element with the oracle."""
import threading

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
def forests():
    return {k: datagen.forest(k) for k in ("tiny", "image", "hbm", "wide")}


def _oracle(forest, X, leaves=False):
    return oracle.predict(forest, X, leaves=leaves, threads=oracle.default_threads())


def test_wide_forest_every_row(forests):
    """64 trees, 50 classes, 100 features (its fields leave room for
    three-level super-nodes of format 2 only): all 100,000 test rows, in the
    library defaults and in three other layouts, one with two-level
    super-nodes."""
    f = forests["wide"]
    X, _ = datagen.test_rows("wide")
    ref = _oracle(f, X, leaves=True)
    Xd = torch.from_numpy(X).cuda()
    for params in ({}, dict(bin_size=16, interleave_depth=4, head_select=1),
                   dict(bin_size=2, interleave_depth=7, pass_bytes=1 << 20),
                   dict(bin_size=4, interleave_depth=5, deep_levels=2)):
        pk = fp.fp_pack_forest(f, **params)
        assert (pk.info()["deep_levels"], pk.info()["deep_format"]) == ((2, 0) if params.get("deep_levels") else (3, 2))
        df = fp.fp_upload(pk)
        votes, cls = df.predict(Xd)
        leaves = df.predict_leaves(Xd)
        torch.cuda.synchronize()
        assert df.sync_status() == fp.FP_OK
        np.testing.assert_array_equal(votes.cpu().numpy().astype(np.uint32), ref["votes"])
        np.testing.assert_array_equal(cls.cpu().numpy(), ref["cls"])
        np.testing.assert_array_equal(leaves.cpu().numpy(), ref["leaf"])
        df.release()


def test_batched_hbm_image_wide_one_launch_graph(forests):
    """The HBM-resident forest (5 passes, three-level super-nodes of format
    1), the image and wide forests (three-level super-nodes of format 2), a
    two-level packing of the HBM-resident forest and the tiny forest in one
    persistent launch, so every kind of walk runs in it; captured once,
    replayed on two sets of rows; every row compared with the oracle."""
    names = ["hbm", "image", "wide", "tiny", "hbm2"]
    sizes = [150_000, 20_011, 30_000, 4_099, 7_777]
    forests = dict(forests, hbm2=forests["hbm"])
    dfs = [fp.fp_upload(fp.fp_pack_forest(forests[k], deep_levels=2 if k == "hbm2" else 0)) for k in names]
    info = {k: d.info for k, d in zip(names, dfs)}
    assert info["hbm"]["passes"] > 1 and (info["hbm"]["deep_levels"], info["hbm"]["deep_format"]) == (3, 1)
    assert (info["image"]["deep_levels"], info["image"]["deep_format"]) == (3, 2)
    assert (info["wide"]["deep_levels"], info["wide"]["deep_format"]) == (3, 2)
    assert info["hbm2"]["deep_levels"] == 2
    pools = {k: datagen.test_rows(k if k != "hbm2" else "hbm", 2 * n)[0] for k, n in zip(names, sizes)}
    Xs = [torch.empty((n, forests[k].n_features), dtype=torch.float32, device="cuda") for k, n in zip(names, sizes)]
    votes = [torch.empty((n, forests[k].n_classes), dtype=torch.int32, device="cuda") for k, n in zip(names, sizes)]
    cls = [torch.empty((n,), dtype=torch.int32, device="cuda") for n in sizes]
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        for x in Xs:
            x.zero_()
        fp.fp_predict_batched(dfs, Xs, votes, cls, stream=stream)  # warm-up outside the graph
    stream.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        fp.fp_predict_batched(dfs, Xs, votes, cls, stream=torch.cuda.current_stream())
    for rep in range(2):
        Xh = [np.ascontiguousarray(pools[k][rep * n: (rep + 1) * n]) for k, n in zip(names, sizes)]
        for x, xh in zip(Xs, Xh):
            x.copy_(torch.from_numpy(xh))
        for v, c in zip(votes, cls):
            v.fill_(-1)
            c.fill_(-1)
        g.replay()
        torch.cuda.synchronize()
        for d in dfs:
            assert d.sync_status() == fp.FP_OK
        for k, xh, v, c in zip(names, Xh, votes, cls):
            ref = _oracle(forests[k], xh)
            np.testing.assert_array_equal(v.cpu().numpy().astype(np.uint32), ref["votes"], err_msg=k)
            np.testing.assert_array_equal(c.cpu().numpy(), ref["cls"], err_msg=k)
    for d in dfs:
        d.release()


def _requests(pools, n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    names = sorted(pools)
    out = []
    for _ in range(n):
        k = names[rng.integers(len(names))]
        m = int(np.clip(round(rng.lognormal(np.log(32), 1.5)), 1, 4096))
        s = int(rng.integers(0, pools[k].shape[0] - m))
        out.append((k, pools[k][s: s + m]))
    return out


def test_serving_workload_forests(forests):
    """Config 5's four forests behind one server: 240 requests from three
    threads (log-normal sizes, up to 4,096 rows), each answer equal alone and
    in the mix, and equal to the oracle's votes and classes."""
    from paper_1806_07300_gb300.serving import ForestServer
    pools = {k: datagen.test_rows(k, 40_000 if k != "tiny" else 10_000)[0] for k in forests}
    reqs = _requests(pools, 240, seed=17)
    srv = ForestServer(slots=3, max_rows=1 << 15, return_votes=True)
    for k, f in forests.items():
        srv.add_forest(k, f)
    with srv:
        handles = [None] * len(reqs)

        def client(lo, hi):
            for i in range(lo, hi):
                handles[i] = srv.submit(*reqs[i])

        ts = [threading.Thread(target=client, args=(j * 80, (j + 1) * 80)) for j in range(3)]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        for h in handles:
            assert h.wait(120) and h.error is None
    alone = ForestServer(slots=1, return_votes=True)
    for k, f in forests.items():
        alone.add_forest(k, f)
    with alone:
        for (k, X), h in zip(reqs[::4], handles[::4]):
            a = alone.submit(k, X)
            assert a.wait(120) and a.error is None
            np.testing.assert_array_equal(a.classes, h.classes)
            np.testing.assert_array_equal(a.votes, h.votes)
    srv.close()
    alone.close()
    for (k, X), h in zip(reqs, handles):
        ref = _oracle(forests[k], X)
        np.testing.assert_array_equal(h.classes, ref["cls"], err_msg=k)
        np.testing.assert_array_equal(h.votes.astype(np.uint32), ref["votes"], err_msg=k)
