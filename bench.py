"""Benchmark: observations/s of packed-forest classification on GB300.

One step = one pass of the whole hot path (interleaved levels, Stat regions,
votes, argmax) over one batch of synthetic observations resident in HBM:
fp_predict(forest, X[n], out_votes, out_class).  Default workload: the
HBM-resident forest (256 CART trees of ~8*10^4 internal nodes, forest far
larger than L2) classifying 4,000,000 rows of 28 FP32 features.

Prints one JSON line (rank 0).  Besides the headline value it reports the
plain breadth-first GPU baseline on the same inputs (faster of its two thread
orders), the end-to-end figure through host buffers, the roofline of the
traversal kernel, and the CPU oracle timed on a bounded sample.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl packed|reference]
                    [--workload hbm|image|tiny] [--rows N]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "observations/sec/GPU packed vs plain-layout GPU; % L2/HBM roofline; p50/p99 ms"

WORKLOADS = {
    "hbm": dict(rows=4_000_000, desc="HBM-resident forest: 256 trees, 28 features, 2 classes, 500k training rows"),
    "image": dict(rows=1_000_000, desc="image-shaped: 128 trees, 784 features, 10 classes, 60k training rows"),
    "tiny": dict(rows=10_000, desc="tiny: 16 trees, 16 features, 4 classes, 2k training rows"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="packed", choices=["packed", "reference"])
    ap.add_argument("--workload", default="hbm", choices=sorted(WORKLOADS))
    ap.add_argument("--rows", type=int, default=0)
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU work of the oracle sample")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--bin-size", type=int, default=0)
    ap.add_argument("--depth", type=int, default=-1)
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--warps", type=int, default=0)
    ap.add_argument("--pass-bytes", type=int, default=0)
    return ap.parse_args()


# ------------------------------------------------------------ clocks sampler

class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


# ----------------------------------------------------------------- helpers

def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def cpu_sample(forest, X, target_s: float, threads: int):
    """Oracle on a bounded prefix of the workload's rows: returns obs/s,
    visits per observation and the sample size."""
    import oracle
    n = min(2000, X.shape[0])
    t0 = time.perf_counter()
    r = oracle.predict(forest, X[:n], leaves=False, votes=False, threads=threads)
    dt = max(time.perf_counter() - t0, 1e-6)
    m = int(min(X.shape[0], max(n, n * target_s / dt)))
    t0 = time.perf_counter()
    r = oracle.predict(forest, X[:m], leaves=False, votes=False, threads=threads)
    dt = time.perf_counter() - t0
    return m / dt, r["visits"] / m, m, dt


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if args.impl == "packed" else "gloo")
    return ws, rank, local


# --------------------------------------------------------------- reference

def run_reference(args, ws, rank):
    """The oracle as it stands, on the host cores, timed per step on a bounded
    sample of the same workload."""
    if rank != 0:
        return
    import datagen
    import oracle
    name = args.workload
    forest = datagen.forest(name)
    n_full = args.rows or WORKLOADS[name]["rows"]
    threads = oracle.default_threads()
    # size one step for ~2 s of CPU work so the whole run stays within minutes
    probe_rows = min(2000, n_full)
    X, _ = datagen.test_rows(name, probe_rows)
    t0 = time.perf_counter()
    oracle.predict(forest, X, leaves=False, votes=False, threads=threads)
    dt = max(time.perf_counter() - t0, 1e-6)
    m = int(min(n_full, max(probe_rows, probe_rows * 2.0 / dt)))
    X, _ = datagen.test_rows(name, m)
    for _ in range(args.warmup):
        oracle.predict(forest, X, leaves=False, votes=False, threads=threads)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.predict(forest, X, leaves=False, votes=False, threads=threads)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = m * args.steps / total
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "observations/s",
           "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": name, "desc": WORKLOADS[name]["desc"], "rows_per_step": m, "n_trees": forest.n_trees},
           "cpu_baseline": {"value": value, "unit": "observations/s", "cores": threads, "kind": "oracle",
                            "sample": f"first {m} of the workload's {n_full} test rows per step"},
           "e2e": {"value": value, "unit": "observations/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# ------------------------------------------------------------------ packed

def run_packed(args, ws, rank, local):
    import torch
    import datagen
    import paper_1806_07300_gb300 as fp

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    name = args.workload
    n = args.rows or WORKLOADS[name]["rows"]
    forest = datagen.forest(name)
    Xh, _ = datagen.test_rows(name, n)
    F, C, T = forest.n_features, forest.n_classes, forest.n_trees

    pk = fp.fp_pack_forest(forest, bin_size=args.bin_size, interleave_depth=args.depth, obs_tile=args.tile,
                           warps_per_cta=args.warps, pass_bytes=args.pass_bytes)
    df = fp.fp_upload(pk)
    info = df.info
    stream = torch.cuda.Stream(device=dev)
    X = torch.from_numpy(Xh).to(dev)
    votes = torch.empty((n, C), dtype=torch.int32, device=dev)
    cls = torch.empty((n,), dtype=torch.int32, device=dev)
    torch.cuda.synchronize()

    def step():
        fp.fp_predict(df, X, votes, cls, stream=stream)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    status = df.sync_status(stream)
    if status != fp.FP_OK:
        raise RuntimeError(f"kernel status {status}: {fp.fp_last_error()}")

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for i in range(args.steps):
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    stop.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    total_ms = start.elapsed_time(stop)
    per_launch_ms = [a.elapsed_time(b) for a, b in ev]
    if ws > 1:
        import torch.distributed as dist
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = ws * n * args.steps / (total_ms / 1e3)

    # plain breadth-first baseline, both thread orders, same inputs
    plain = None
    if not args.no_plain:
        pf = fp.fp_plain_build(forest)
        pv = torch.empty((n, C), dtype=torch.int32, device=dev)
        pc = torch.empty((n,), dtype=torch.int32, device=dev)
        best = None
        for order, oname in ((fp.FP_PLAIN_OBS_FASTEST, "obs_fastest"), (fp.FP_PLAIN_TREE_FASTEST, "tree_fastest")):
            fp.fp_plain_predict(pf, X, order, pv, pc, stream=stream)
            torch.cuda.synchronize()
            ks = max(2, args.steps // 4)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(ks):
                fp.fp_plain_predict(pf, X, order, pv, pc, stream=stream)
            b.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b) / ks
            ok = bool(torch.equal(pc, cls))
            cand = {"order": oname, "value": n / (ms / 1e3), "ms_per_step": ms, "same_classes": ok}
            if best is None or cand["value"] > best["value"]:
                best = cand
        plain = dict(best, unit="observations/s", layout_bytes=pf.nbytes())
        pf.release()

    # end to end through host buffers: pinned X in, classes out, every step
    Xpin = torch.from_numpy(Xh).pin_memory()
    cls_host = torch.empty((n,), dtype=torch.int32).pin_memory()
    Xd2 = torch.empty_like(X)
    e2e_steps = max(3, args.steps // 2)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        a.record(stream)
        for _ in range(e2e_steps):
            Xd2.copy_(Xpin, non_blocking=True)
            fp.fp_predict(df, Xd2, None, cls, stream=stream)
            cls_host.copy_(cls, non_blocking=True)
        b.record(stream)
    torch.cuda.synchronize()
    e2e_ms = a.elapsed_time(b) / e2e_steps
    e2e = {"value": ws * n / (e2e_ms / 1e3), "unit": "observations/s", "h2d_bytes_per_step": int(Xpin.numel() * 4),
           "d2h_bytes_per_step": int(cls_host.numel() * 4), "ms_per_step": e2e_ms}

    if rank != 0:
        return
    # CPU oracle on a bounded sample; its visit count gives the algorithmic bytes
    import oracle
    threads = oracle.default_threads()
    cpu_value, visits_per_obs, m, cpu_s = cpu_sample(forest, Xh, args.cpu_seconds, threads)
    bytes_per_obs = 8.0 * visits_per_obs + 4.0 * F + 4.0 * C + 4.0
    avg_launch_ms = statistics.mean(per_launch_ms)
    achieved = bytes_per_obs * n / (avg_launch_ms / 1e3) / 1e9
    peak, peak_kind = measured_peaks()
    out = {
        "metric": METRIC, "value": value, "unit": "observations/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded generators; CART forest trained at start)",
        "config": {"workload": name, "desc": WORKLOADS[name]["desc"], "rows": n, "n_trees": T, "n_features": F,
                   "n_classes": C, "bin_size": info["bin_size"], "interleave_depth": info["interleave_depth"],
                   "obs_tile": info["obs_tile"], "warps_per_cta": info["warps_per_cta"], "passes": info["passes"],
                   "forest_bytes": info["total_bytes"], "parallelism": f"replicas x{ws}",
                   "l2": "inputs larger than L2 (rows %.0f MB, forest %.0f MB); no flush" %
                         (Xh.nbytes / 1e6, info["total_bytes"] / 1e6)},
        "plain_baseline": plain,
        "packed_vs_plain": (value / ws / plain["value"]) if plain else None,
        "e2e": e2e,
        "gpu_launches": args.steps,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "peak_kind": peak_kind,
                     "kernel": "fp_traverse_kernel<false>", "avg_launch_ms": avg_launch_ms,
                     "bytes_per_obs": bytes_per_obs, "visits_per_obs": visits_per_obs,
                     "node_visits_per_s": visits_per_obs * n / (avg_launch_ms / 1e3)},
        "cpu_baseline": {"value": cpu_value, "unit": "observations/s", "cores": threads, "kind": "oracle",
                         "sample": f"first {m} of {n} rows ({cpu_s:.1f} s)"},
        "clocks": clk,
    }
    print(json.dumps(out))
    df.release()


def main():
    args = parse()
    ws, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_packed(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
