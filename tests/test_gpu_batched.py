"""GPU parity of the batched path: many resident forests and uneven
observation batches in one persistent launch, captured in a CUDA graph and
replayed on new inputs.  Bit-exact against the oracle."""
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


def _outs(forests, Xs):
    votes = [torch.empty((x.shape[0], f.info["n_classes"]), dtype=torch.int32, device="cuda")
             for f, x in zip(forests, Xs)]
    cls = [torch.empty((x.shape[0],), dtype=torch.int32, device="cuda") for x in Xs]
    return votes, cls


def _check(forest_objs, Xh, votes, cls, sample=None):
    for F, X, v, c in zip(forest_objs, Xh, votes, cls):
        idx = np.arange(X.shape[0])
        if sample is not None and X.shape[0] > sample:
            idx = np.sort(np.random.Generator(np.random.PCG64(7)).choice(X.shape[0], sample, replace=False))
        ref = oracle.predict(F, X[idx], leaves=False, threads=oracle.default_threads())
        np.testing.assert_array_equal(v.cpu().numpy()[idx].astype(np.uint32), ref["votes"])
        np.testing.assert_array_equal(c.cpu().numpy()[idx], ref["cls"])


def test_batched_mixed_layouts_and_passes(tiny_forest, tiny_rows):
    """One launch over forests with different bins, heads, pass counts and
    bin-buffer counts (items of forests streaming through two and three
    buffers share CTAs)."""
    X, _ = tiny_rows
    params = [dict(bin_size=1, interleave_depth=0), dict(bin_size=4, interleave_depth=3),
              dict(bin_size=2, interleave_depth=1, pass_bytes=2048), dict(bin_size=16, interleave_depth=9, head_select=3),
              dict(bin_size=3, interleave_depth=5, pass_bytes=1),
              dict(bin_size=8, interleave_depth=4, head_select=1, bin_buffers=2),
              dict(bin_size=2, interleave_depth=6, head_select=1, pass_bytes=4096, bin_buffers=2),
              dict(bin_size=3, interleave_depth=3, pass_bytes=2048, bin_buffers=2),
              dict(bin_size=4, interleave_depth=5, head_select=2), dict(bin_size=2, interleave_depth=7, head_select=2,
                                                                         pass_bytes=8192, bin_buffers=2)]
    sizes = [1, 777, 31, 4096, 2500, 1500, 999, 3333, 2049, 640]
    forests = [fp.fp_upload(fp.fp_pack_forest(tiny_forest, **p)) for p in params]
    Xh = [X[i * 7: i * 7 + n] for i, n in enumerate(sizes)]
    Xs = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in Xh]
    votes, cls = _outs(forests, Xs)
    fp.fp_predict_batched(forests, Xs, votes, cls)
    torch.cuda.synchronize()
    for f in forests:
        assert f.sync_status() == fp.FP_OK
    _check([tiny_forest] * len(sizes), Xh, votes, cls)


def test_batched_classes_only_and_empty(tiny_forest, tiny_rows):
    X, _ = tiny_rows
    forests = [fp.fp_upload(fp.fp_pack_forest(tiny_forest, bin_size=2, interleave_depth=2, pass_bytes=4096))
               for _ in range(3)]
    Xh = [X[:100], X[:0], X[100:1100]]
    Xs = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in Xh]
    _, cls = _outs(forests, Xs)
    fp.fp_predict_batched(forests, Xs, None, cls)
    torch.cuda.synchronize()
    for x, c in zip(Xh, cls):
        np.testing.assert_array_equal(c.cpu().numpy(), oracle.predict(tiny_forest, x)["cls"])


def test_batched_graph_capture_and_replay(tiny_forest, tiny_rows):
    """The persistent launch is captured once in a CUDA graph; replays on new
    rows written into the same input buffers give the oracle's answers."""
    X, _ = tiny_rows
    forests = [fp.fp_upload(fp.fp_pack_forest(tiny_forest, bin_size=b, interleave_depth=d))
               for b, d in [(1, 4), (8, 2), (16, 6)]]
    sizes = [300, 1, 2049]
    Xs = [torch.empty((n, tiny_forest.n_features), dtype=torch.float32, device="cuda") for n in sizes]
    votes, cls = _outs(forests, Xs)
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        for x in Xs:
            x.zero_()
        fp.fp_predict_batched(forests, Xs, votes, cls, stream=stream)  # warm-up outside the graph
    stream.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        fp.fp_predict_batched(forests, Xs, votes, cls, stream=torch.cuda.current_stream())
    for rep in range(3):
        Xh = [X[(rep * 997 + i * 13) % 5000:][:n] for i, n in enumerate(sizes)]
        for x, xh in zip(Xs, Xh):
            x.copy_(torch.from_numpy(np.ascontiguousarray(xh)))
        g.replay()
        torch.cuda.synchronize()
        _check([tiny_forest] * 3, Xh, votes, cls)


def test_batched_workload_eight_forests():
    """The batched workload: 8 forests (32..512 trees, 8..200 features, 2..50
    classes), per-forest batches log-uniform over 1..100,000 rows, one
    persistent launch in a CUDA graph."""
    names = [f"batched{k}" for k in range(len(datagen.BATCHED_SPECS))]
    F = [datagen.forest(n) for n in names]
    sizes = datagen.batch_sizes()
    Xh = [datagen.test_rows(n, s)[0] for n, s in zip(names, sizes)]
    forests = [fp.fp_upload(fp.fp_pack_forest(f)) for f in F]
    Xs = [torch.from_numpy(x).cuda() for x in Xh]
    votes, cls = _outs(forests, Xs)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        fp.fp_predict_batched(forests, Xs, votes, cls, stream=stream)
    stream.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        fp.fp_predict_batched(forests, Xs, votes, cls, stream=torch.cuda.current_stream())
    for v in votes:
        v.fill_(-1)
    g.replay()
    torch.cuda.synchronize()
    _check(F, Xh, votes, cls, sample=5000)
