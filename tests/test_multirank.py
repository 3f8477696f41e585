"""The multi-rank host path of bench.py on CPU (gloo, two ranks).

The path shards by observations with no data exchange (replicas), so what
several ranks share is host logic: the timing reduction (the slowest rank's
time), and the rule that rank 0 alone prints the JSON line.  Both run here as
two processes on the gloo backend."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=ws)
    got = bench.max_over_ranks(10.0 * rank + 1.5, ws)
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
        f.write(repr(got))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo(tmp_path):
    ws = 2
    torch.multiprocessing.spawn(_rank_main, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, join=True)
    for r in range(ws):
        assert float((tmp_path / f"r{r}.txt").read_text()) == 11.5


def test_max_over_ranks_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, 1) == 3.25


def test_reference_arm_under_torchrun(tmp_path):
    """torchrun with two ranks: the reference arm runs on rank 0 only and one
    JSON line comes out."""
    env = dict(os.environ, FP_CACHE_DIR=os.environ.get("FP_CACHE_DIR", os.path.join(ROOT, ".fpcache")))
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={_free_port()}", os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--workload", "tiny", "--gpus", "2", "--steps", "2", "--warmup", "1"]
    r = subprocess.run(cmd, cwd=str(tmp_path), env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"


def test_profiled_traffic_lookup(tmp_path, monkeypatch):
    """bench.py takes DRAM traffic and sector counts from a committed capture
    only when the kernel sources still hash to the capture's fingerprint and
    the launch parameters match an entry exactly; it scales traffic by rows."""
    sys.path.insert(0, ROOT)
    import bench
    params = {"bin_size": 4, "interleave_depth": 9, "head_select": 2, "deep_levels": 3, "obs_tile": 992,
              "warps_per_cta": 32, "refill_lanes": 16, "bin_buffers": 2}
    (tmp_path / "profiles").mkdir()
    rec = {"fingerprint": bench.kernel_fingerprint(),
           "entries": [{"params": params, "rows": 1000, "dram_bytes_per_launch": 5000,
                        "global_load_sectors": 300, "global_load_requests": 12}]}
    (tmp_path / "profiles" / "traffic_hbm.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_fingerprint", lambda: rec["fingerprint"])
    t, how = bench.profiled_traffic("hbm", params, 4000)
    assert t == 20000 and "extrapolated" in how
    t, how = bench.profiled_traffic("hbm", params, 1000)
    assert t == 5000 and "extrapolated" not in how
    assert bench.profiled_entry("hbm", params)["global_load_sectors"] == 300
    assert bench.profiled_traffic("hbm", dict(params, refill_lanes=24), 4000)[0] is None
    assert bench.profiled_traffic("image", params, 4000)[0] is None
    monkeypatch.setattr(bench, "kernel_fingerprint", lambda: "0000000000000000")
    assert bench.profiled_traffic("hbm", params, 4000)[0] is None


def test_roofline_fraction_check(monkeypatch):
    """A roofline fraction far above 1 (bytes that never touch the resource)
    stops the bench instead of being printed, except under a profiler."""
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setattr(bench, "SKIP_ROOFLINE_CHECK", False)
    bench.check_roofline({"frac": 0.44, "hbm": {"frac": 0.02}})
    bench.check_roofline({"frac": 1.1, "hbm": {"frac": None}})
    with pytest.raises(RuntimeError):
        bench.check_roofline({"frac": 1.5})
    with pytest.raises(RuntimeError):
        bench.check_roofline({"frac": 0.5, "hbm": {"frac": 3.0}})
    monkeypatch.setattr(bench, "SKIP_ROOFLINE_CHECK", True)
    r = {"frac": 3.0}
    bench.check_roofline(r)
    assert r["check"].startswith("skipped")
