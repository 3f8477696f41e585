"""Benchmark: observations/s of packed-forest classification on GB300.

One step = one pass of the whole hot path (the interleaved heads in shared
memory, the super-node walks, votes, argmax) over one batch of synthetic
observations resident in HBM: fp_predict(forest, X[n], out_votes, out_class).

Workloads (--workload):
  hbm      (default) the HBM-resident forest -- 256 CART trees of ~8*10^4
           internal nodes, forest far larger than L2 -- classifying
           4,000,000 rows of 28 FP32 features;
  image    128 trees, 784 features, 10 classes, 1,000,000 rows;
  tiny     16 trees, 16 features, 4 classes, 10,000 rows;
  batched  8 forests (32..512 trees) and uneven batches (1..100,000 rows) in
           one persistent launch replayed from a CUDA graph;
  serving  4 resident forests behind the continuous-batching server, Poisson
           arrivals at 2k/5k/10k/20k requests/s; p50/p99 latency;
  ablation the layout ablation on the HBM-resident forest (the GPU counterpart
           of the paper's Figs. 4 and 6): plain BF, DF order, Stat, Stat from
           statistics counted on observations, Bin with levels 0..d, Bin with
           the most visited nodes, and the autotuned layout;
  regress  a regression forest with real leaf values (128 trees), 4,000,000
           rows; output = mean of the trees' leaf values (fp_predict_values);
  boosted  256 gradient-boosted trees of depth <= 6, 4,000,000 rows; output =
           initial score + sum of leaf values.

Prints one JSON line (rank 0).  Besides the headline value it reports the
plain breadth-first GPU baseline on the same inputs (the faster of its two
thread orders), the end-to-end figure through host buffers, the roofline of
the traversal kernel against the measured HBM copy bandwidth and a measured
L2 read bandwidth, and the CPU oracle timed on a bounded sample.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl packed|reference]
                    [--workload hbm|image|tiny|batched|serving|ablation] [--rows N]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
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
    "batched": dict(rows=0, desc="8 forests (32..512 trees, 8..200 features, 2..50 classes), batches 1..100k rows, "
                                 "one persistent launch replayed from a CUDA graph"),
    "serving": dict(rows=0, desc="4 resident forests (tiny, image, hbm, 64-tree 50-class 100-feature), Poisson "
                                 "arrivals, rows/request LogNormal(ln 32, 1.5) clipped to [1, 4096]"),
    "ablation": dict(rows=4_000_000, desc="layout ablation on the HBM-resident forest (256 trees, 4,000,000 rows)"),
    "regress": dict(rows=4_000_000, desc="regression forest with leaf values: 128 trees (min leaf 5) on the hbm "
                                         "features with a real target, 200k training rows; output = mean of trees"),
    "boosted": dict(rows=4_000_000, desc="gradient-boosted shallow trees: 256 rounds of depth <= 6, learning rate "
                                         "0.1, 30k training rows; output = initial score + sum of trees"),
}

# Layout and launch candidates timed by the autotuner for the default workload
# (the bin-size / interleaved-depth pairs that led the sweeps on this forest).
# (B, d, head_select[, deep_levels[, deep_format]]); without deep_levels the library's default (three levels
# here: format 1 for the hbm, regress and boosted forests, format 2 for the image forest)
HBM_LAYOUTS = [(3, 9, 2), (4, 9, 2), (5, 9, 2), (1, 11, 2), (4, 9, 1), (3, 8, 3), (3, 9, 2, 2)]
HBM_LAUNCHES = [(1024, 32, 16, 2), (1024, 32, 24, 2), (768, 32, 16, 2), (1024, 32, 16, 3)]  # tile, warps, refill, buffers
# the value workloads: the regression forest's trees resemble the hbm ones; the
# boosted trees (depth <= 6) fit whole in a level head of depth 5
TUNE = {
    "hbm": (HBM_LAYOUTS, HBM_LAUNCHES),
    "regress": ([(4, 9, 2), (3, 9, 2), (4, 9, 1), (3, 8, 1)], HBM_LAUNCHES),
    # 784-feature rows (3.1 KB) fill shared memory quickly: 64-row tiles in one
    # 32-warp CTA with small heads of many trees (bins with more tasks, so fewer
    # bin changes per task), or 32-row tiles in two 16-warp CTAs per SM; the
    # library's default super-nodes (three levels, format 2) and two-level ones
    "image": ([(32, 3, 2), (16, 3, 2), (64, 1, 2), (128, 1, 2), (32, 3, 2, 2)],
              [(64, 32, 16, 2), (64, 32, 8, 2), (64, 32, 24, 2), (32, 16, 8, 2)]),
    "boosted": ([(64, 5, 2), (32, 5, 2), (64, 5, 1), (16, 5, 1)],
                [(768, 32, 16, 3), (1024, 32, 16, 3), (512, 16, 16, 3), (1024, 32, 32, 2)]),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="packed", choices=["packed", "reference"])
    ap.add_argument("--workload", default="hbm", choices=sorted(WORKLOADS))
    ap.add_argument("--forest", default="hbm", help="forest of the ablation workload")
    ap.add_argument("--rows", type=int, default=0)
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU work of the oracle sample")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--bin-size", type=int, default=0)
    ap.add_argument("--depth", type=int, default=-1)
    ap.add_argument("--head-select", type=int, default=0,
                    help="0: default; 1: levels 0..d (implicit slots); 2: paired level slots; 3: ranked")
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--warps", type=int, default=0)
    ap.add_argument("--refill", type=int, default=0)
    ap.add_argument("--bin-buffers", type=int, default=0)
    ap.add_argument("--deep-levels", type=int, default=0, help="tree levels per super-node: 2, 3 (0: default)")
    ap.add_argument("--deep-format", type=int, default=0,
                    help="three-level super-nodes: 1 full keys first, 2 key prefixes in every slot (0: default)")
    ap.add_argument("--pass-bytes", type=int, default=0)
    ap.add_argument("--serve-seconds", type=float, default=2.0, help="seconds of requests per offered rate")
    ap.add_argument("--no-roofline-check", action="store_true",
                    help="print roofline fractions above 1.2 instead of stopping (runs under a profiler)")
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
            threading.Thread(target=self._read, daemon=True).start()
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


def kernel_fingerprint() -> str:
    """Hash of the sources that decide the traversal kernel's memory traffic:
    the kernel, the image format, the packer and the launch set-up (grid,
    tile shrinking, scratch); the launch parameters are matched per captured
    entry."""
    h = hashlib.sha1()
    for name in ("fp_traverse.cuh", "fp_pack.cpp", "fp_internal.h", "fp_device.cu"):
        with open(os.path.join(ROOT, "paper_1806_07300_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_entry(workload: str, params: dict):
    """The committed ncu counters of one launch for these parameters, or None
    when the kernel changed since they were taken or the parameters were not
    captured."""
    path = os.path.join(ROOT, "profiles", f"traffic_{workload}.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    if d.get("fingerprint") != kernel_fingerprint():
        return None
    for e in d.get("entries", []):  # one per captured launch configuration
        if e["params"] == params:
            return e
    return None


def profiled_traffic(workload: str, params: dict, rows: int):
    """DRAM bytes per launch from the committed ncu summary and how they were
    obtained: measured at these rows, or scaled linearly from the captured
    row count (an extrapolation: the rows are re-read once per pass, but the
    forest's L2 reuse need not scale with the rows).  (None, reason) when the
    kernel changed since the capture or the parameters were not captured."""
    e = profiled_entry(workload, params)
    if e is None:
        return None, "no ncu capture for this kernel source and launch configuration"
    if e["rows"] == rows:
        return e["dram_bytes_per_launch"], f"ncu, one launch over {rows} rows"
    return e["dram_bytes_per_launch"] * rows / e["rows"], \
        f"ncu at {e['rows']} rows, scaled linearly to {rows} rows (extrapolated)"


SKIP_ROOFLINE_CHECK = False  # --no-roofline-check: runs under a profiler


def check_roofline(r: dict) -> None:
    """A fraction far above 1 means the bound is misapplied (bytes that never
    touch the resource): refuse to print it.  Under a profiler every launch
    is serialised and slowed, the probe's bandwidth with it, so no fraction
    means anything; such runs pass --no-roofline-check."""
    if SKIP_ROOFLINE_CHECK:
        r["check"] = "skipped (--no-roofline-check)"
        return
    for k, v in [("frac", r.get("frac")), ("hbm.frac", (r.get("hbm") or {}).get("frac"))]:
        if v is not None and v > 1.2:
            raise RuntimeError(f"roofline {k} = {v:.2f} > 1.2: the bound does not describe this kernel")


def cpu_sample(forest, X, target_s: float, threads: int):
    """Oracle on a bounded prefix of the workload's rows: returns obs/s,
    visits per observation, the sample size and the seconds taken."""
    import oracle
    if getattr(forest, "leaf_value", None) is not None:
        call = lambda Xs: oracle.predict_values(forest, Xs, threads=threads)  # noqa: E731
    else:
        call = lambda Xs: oracle.predict(forest, Xs, leaves=False, votes=False, threads=threads)  # noqa: E731
    n = min(2000, X.shape[0])
    t0 = time.perf_counter()
    call(X[:n])
    dt = max(time.perf_counter() - t0, 1e-6)
    m = int(min(X.shape[0], max(n, n * target_s / dt)))
    t0 = time.perf_counter()
    r = call(X[:m])
    dt = time.perf_counter() - t0
    return m / dt, r["visits"] / m, m, dt


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        if args.impl == "packed":
            torch.cuda.set_device(local)
        dist.init_process_group("nccl" if args.impl == "packed" else "gloo")
    return ws, rank, local


class L2Flush:
    """For a workload whose inputs fit in L2: a write of twice the L2 size
    before every timed step evicts them, so each step starts from a cold L2
    as a step of a larger workload would."""

    def __init__(self, dev):
        import torch
        self.l2 = int(torch.cuda.get_device_properties(dev).L2_cache_size)
        self.buf = torch.empty((2 * self.l2) // 4, dtype=torch.int32, device=dev)

    def __call__(self, stream) -> None:
        import torch
        with torch.cuda.stream(stream):
            self.buf.fill_(1)

    def describe(self, input_bytes: int) -> str:
        return (f"inputs ({input_bytes / 1e6:.1f} MB) fit in L2 ({self.l2 / 1e6:.0f} MB): L2 flushed before every "
                f"timed step by a {2 * self.l2 / 1e6:.0f} MB write, outside the step's events")


def flush_for(dev, input_bytes: int):
    """An L2Flush when the workload's inputs fit in L2, else None."""
    import torch
    l2 = int(torch.cuda.get_device_properties(dev).L2_cache_size)
    return L2Flush(dev) if input_bytes < l2 else None


def timed_steps(fn, k: int, stream, flush=None):
    """Device milliseconds of k steps of fn() on `stream`, and the per-step
    times when measured: one event pair around k back-to-back steps (inputs
    larger than L2), or with an L2 flush before every step one event pair per
    step (the flush outside it), summed."""
    import torch
    if flush is None:
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(k):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b), None
    ev = []
    for _ in range(k):
        flush(stream)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        ev.append((a, b))
    torch.cuda.synchronize()
    per = [a.elapsed_time(b) for a, b in ev]
    return sum(per), per


def max_over_ranks(value: float, ws: int, device=None) -> float:
    """The largest value over all ranks (the slowest rank's time); the value
    itself with one rank."""
    if ws <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def base_line(args, ws, value, total_ms, config, dtype="f32"):
    return {"metric": METRIC, "value": value, "unit": "observations/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype,
            "data": "synthetic (seeded generators; CART forests trained at start)", "config": config}


# --------------------------------------------------------------- reference

def run_reference(args, ws, rank):
    """The oracle as it stands, on the host cores, timed per step on a bounded
    sample of the same workload (rank 0 only)."""
    if rank != 0:
        return
    import datagen
    import oracle
    name = args.workload if args.workload in ("hbm", "image", "tiny", "regress", "boosted") else "hbm"
    forest = datagen.forest(name)
    n_full = args.rows or WORKLOADS[name]["rows"]
    threads = oracle.default_threads()

    def call(Xs):
        if forest.leaf_value is not None:
            oracle.predict_values(forest, Xs, threads=threads)
        else:
            oracle.predict(forest, Xs, leaves=False, votes=False, threads=threads)

    probe_rows = min(2000, n_full)
    X, _ = datagen.test_rows(name, probe_rows)
    t0 = time.perf_counter()
    call(X)
    dt = max(time.perf_counter() - t0, 1e-6)
    m = int(min(n_full, max(probe_rows, probe_rows * 2.0 / dt)))  # ~2 s of CPU work per step
    X, _ = datagen.test_rows(name, m)
    for _ in range(args.warmup):
        call(X)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        call(X)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = m * args.steps / total
    out = base_line(args, ws, value, 1e3 * total,
                    {"workload": name, "desc": WORKLOADS[name]["desc"], "rows_per_step": m,
                     "n_trees": forest.n_trees})
    out["impl"] = "reference"
    out["cpu_baseline"] = {"value": value, "unit": "observations/s", "cores": threads, "kind": "oracle",
                           "sample": f"first {m} of the workload's {n_full} test rows per step"}
    out["e2e"] = {"value": value, "unit": "observations/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    print(json.dumps(out))


# ------------------------------------------------------------- single forest

def tuned_forest(args, forest, X, name):
    import paper_1806_07300_gb300 as fp
    from paper_1806_07300_gb300 import autotune as at
    explicit = args.bin_size or args.depth >= 0 or args.tile or args.warps or args.refill
    tuning = None
    if explicit or args.no_autotune:
        params = dict(bin_size=args.bin_size, interleave_depth=args.depth, pass_bytes=args.pass_bytes,
                      head_select=args.head_select, deep_levels=args.deep_levels, deep_format=args.deep_format)
        df = fp.fp_upload(fp.fp_pack_forest(forest, **params))
        df.configure(obs_tile=args.tile, warps_per_cta=args.warps, refill_lanes=args.refill,
                     bin_buffers=args.bin_buffers)
    else:
        sample = X[: min(X.shape[0], 1 << 20)]
        layouts, launches = TUNE.get(name, (None, None))
        best = at.autotune(forest, sample, layouts=layouts, launches=launches)
        tuning = {k: best[k] for k in at.LAYOUT_KEYS + at.LAUNCH_KEYS}
        tuning["candidates"] = len([r for r in best["table"] if "ms" in r])
        df = fp.fp_upload(fp.fp_pack_forest(forest, **{k: best[k] for k in at.LAYOUT_KEYS}))
        df.configure(**{k: best[k] for k in at.LAUNCH_KEYS})
    return df, tuning


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
    X = torch.from_numpy(Xh).to(dev)
    df, tuning = tuned_forest(args, forest, X, name)
    info = df.info
    stream = torch.cuda.Stream(device=dev)
    values = forest.leaf_value is not None  # regression / boosted: a float per row instead of votes and classes
    votes = None if values else torch.empty((n, C), dtype=torch.int32, device=dev)
    cls = torch.empty((n,), dtype=torch.float32 if values else torch.int32, device=dev)
    torch.cuda.synchronize()

    def step(Xs, out_votes, out, s):
        if values:
            fp.fp_predict_values(df, Xs, out, forest.value_scale, forest.value_bias, stream=s)
        else:
            fp.fp_predict(df, Xs, out_votes, out, stream=s)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(args.warmup):
        step(X, votes, cls, stream)
    torch.cuda.synchronize()
    status = df.sync_status(stream)
    if status != fp.FP_OK:
        raise RuntimeError(f"kernel status {status}: {fp.fp_last_error()}")

    flush = flush_for(dev, Xh.nbytes + info["total_bytes"])
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    # the timed region: K steps, one launch each, back to back on the stream
    # (inputs larger than L2), or each after an L2 flush and timed alone
    total_ms, per_launch_ms = timed_steps(lambda: step(X, votes, cls, stream), args.steps, stream, flush)
    barrier()
    clk = clocks.stop()
    if per_launch_ms is None:
        # the spread of single launches, in a separate pass with events around
        # each (recording them costs host time between launches, so they stay
        # out of the timed region)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        for i in range(args.steps):
            ev[i][0].record(stream)
            step(X, votes, cls, stream)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        per_launch_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(total_ms, ws, dev)
    value = ws * n * args.steps / (total_ms / 1e3)

    # plain breadth-first baseline, both thread orders, same inputs
    plain = None
    if not args.no_plain:
        pf = fp.fp_plain_build(forest)
        pv = None if values else torch.empty((n, C), dtype=torch.int32, device=dev)
        pc = torch.empty((n,), dtype=cls.dtype, device=dev)

        def plain_step(order):
            if values:
                fp.fp_plain_predict_values(pf, X, order, pc, forest.value_scale, forest.value_bias, stream=stream)
            else:
                fp.fp_plain_predict(pf, X, order, pv, pc, stream=stream)

        best = None
        for order, oname in ((fp.FP_PLAIN_OBS_FASTEST, "obs_fastest"), (fp.FP_PLAIN_TREE_FASTEST, "tree_fastest")):
            plain_step(order)
            torch.cuda.synchronize()
            ks = max(2, args.steps // 4)
            ms = timed_steps(lambda: plain_step(order), ks, stream, flush)[0] / ks  # as the packed path
            cand = {"order": oname, "value": n / (ms / 1e3), "ms_per_step": ms}
            if values:
                cand["max_abs_diff"] = float((pc - cls).abs().max())
            else:
                cand["same_classes"] = bool(torch.equal(pc, cls))
            if best is None or cand["value"] > best["value"]:
                best = cand
        plain = dict(best, unit="observations/s", layout_bytes=pf.nbytes())
        pf.release()
        del pv, pc

    # end to end through host buffers: the C-ABI host-buffer call, pinned rows
    # in and classes (or values) out every step, copies pipelined with the
    # kernels inside the call
    Xpin = torch.from_numpy(Xh).pin_memory()
    cls_host = torch.empty((n,), dtype=cls.dtype).pin_memory()
    e2e_steps = max(3, args.steps // 2)

    def step_host():
        if values:
            fp.fp_predict_values_host(df, Xpin, cls_host, forest.value_scale, forest.value_bias, 0, stream)
        else:
            fp.fp_predict_host(df, Xpin, None, cls_host, 0, stream)

    step_host()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(e2e_steps):
        step_host()
    b.record(stream)
    torch.cuda.synchronize()
    if not values and not torch.equal(cls_host, cls.cpu()):
        raise RuntimeError("end-to-end classes differ from the device path's")
    e2e_ms = a.elapsed_time(b) / e2e_steps
    e2e = {"value": ws * n / (e2e_ms / 1e3), "unit": "observations/s", "h2d_bytes_per_step": int(Xpin.numel() * 4),
           "d2h_bytes_per_step": int(cls_host.numel() * 4), "ms_per_step": e2e_ms}
    l2_gbs = fp.fp_l2_read_probe(64 << 20, 40, stream=stream)

    if rank != 0:
        return
    import oracle
    threads = oracle.default_threads()
    cpu_value, visits_per_obs, m, cpu_s = cpu_sample(forest, Xh, args.cpu_seconds, threads)
    cpu1_value, _, m1, cpu1_s = cpu_sample(forest, Xh, max(0.5, args.cpu_seconds / 4), 1)  # one core
    # node records, the row, and the outputs (votes and class; or the leaf
    # value read per tree and one float out)
    bytes_per_obs = 8.0 * visits_per_obs + 4.0 * F + (4.0 * T + 4.0 if values else 4.0 * C + 4.0)
    avg_launch_ms = total_ms / args.steps  # the timed region holds one launch per step and nothing else
    achieved = bytes_per_obs * n / (avg_launch_ms / 1e3) / 1e9
    peak, peak_kind = measured_peaks()
    params = {k: info[k] for k in ("bin_size", "interleave_depth", "head_select", "deep_levels", "deep_format",
                                   "obs_tile", "warps_per_cta", "refill_lanes", "bin_buffers")}
    traffic, traffic_how = profiled_traffic(name, params, n)
    # the sector-granular figure: 32 B per global-load sector the kernel touched
    # (ncu, same launch configuration), the practical bound beside the
    # algorithmic 8 B per node visit
    pe = profiled_entry(name, params)
    sectors = None
    if pe is not None and pe.get("global_load_sectors"):
        srows = pe.get("sectors_rows", pe["rows"])
        sectors = {"bytes_per_obs": 32.0 * pe["global_load_sectors"] / srows,
                   "sectors_per_request": pe["global_load_sectors"] / pe["global_load_requests"],
                   "source": f"ncu l1tex__t_sectors / l1tex__t_requests_pipe_lsu_mem_global_op_ld, one launch over "
                             f"{srows} rows"}
    kernel = "fp_traverse_kernel<values>" if values else "fp_traverse_kernel<votes>"
    visits_per_s = visits_per_obs * n / (avg_launch_ms / 1e3)
    launch_s = avg_launch_ms / 1e3
    hbm_sub = {"peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
               "dram_gbs": None if traffic is None else traffic / launch_s / 1e9,
               "frac": None if traffic is None else traffic / launch_s / 1e9 / peak,
               "traffic": traffic, "traffic_source": traffic_how,
               "algorithmic_frac": achieved / peak,
               "note": "the forest's nodes come from shared memory (interleaved heads) and L2, so DRAM moves a "
                       "small part of the algorithmic bytes; algorithmic_frac divides algorithmic bytes by the "
                       "HBM copy bandwidth and is not a DRAM fraction"}
    if info["n_super"] == 0:
        # every internal node sits in the bins' interleaved heads: the node
        # reads come from shared memory, so the bound is the SMs' shared-memory
        # load bandwidth (128 bytes per clock per SM), not HBM
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        smem_peak = sms * 128 * (clk.get("sm_max_mhz") or 2070.0) * 1e6 / 1e9
        smem_achieved = 8.0 * visits_per_s / 1e9
        roofline = {"bound": "alu", "achieved": smem_achieved, "peak": smem_peak, "unit": "GB/s",
                    "frac": smem_achieved / smem_peak, "traffic": traffic,
                    "peak_kind": f"derived: shared-memory loads, {sms} SMs x 128 B/clock x max SM clock",
                    "kernel": kernel, "avg_launch_ms": avg_launch_ms, "bytes_per_obs": 8.0 * visits_per_obs,
                    "visits_per_obs": visits_per_obs, "node_visits_per_s": visits_per_s, "hbm": hbm_sub}
    else:
        # the node fetches below the heads draw on L2 (the forest's passes stay
        # L2-resident): the headline fraction is of the measured L2 read
        # bandwidth; DRAM is reported beside it from the ncu counters
        roofline = {"bound": "l2", "achieved": achieved, "peak": l2_gbs, "unit": "GB/s",
                    "frac": achieved / l2_gbs, "traffic": traffic,
                    "peak_kind": "measured in this run: fp_l2_read_probe, 16-byte loads over a 64 MiB "
                                 "L2-resident buffer",
                    "kernel": kernel, "avg_launch_ms": avg_launch_ms, "bytes_per_obs": bytes_per_obs,
                    "bytes_per_obs_kind": "algorithmic: 8 B per internal node visited (oracle count) + row + outputs",
                    "visits_per_obs": visits_per_obs, "node_visits_per_s": visits_per_s, "hbm": hbm_sub,
                    "sector_granular": None if sectors is None else dict(
                        sectors, achieved_gbs=sectors["bytes_per_obs"] * n / launch_s / 1e9,
                        frac_of_l2=sectors["bytes_per_obs"] * n / launch_s / 1e9 / l2_gbs)}
    check_roofline(roofline)
    out = base_line(args, ws, value, total_ms,
                    {"workload": name, "desc": WORKLOADS[name]["desc"], "rows": n, "n_trees": T, "n_features": F,
                     "n_classes": C, **params, "passes": info["passes"], "forest_bytes": info["total_bytes"],
                     "autotuned": tuning is not None, "parallelism": f"replicas x{ws}",
                     "l2": flush.describe(Xh.nbytes + info["total_bytes"]) if flush else
                     "inputs larger than L2 (rows %.0f MB, forest %.0f MB); no flush" %
                     (Xh.nbytes / 1e6, info["total_bytes"] / 1e6)})
    out.update({
        "plain_baseline": plain,
        "packed_vs_plain": (value / ws / plain["value"]) if plain else None,
        "e2e": e2e,
        "gpu_launches": args.steps,
        # single launches timed one by one after the timed region: median and spread
        "launch_ms": {"median": statistics.median(per_launch_ms), "min": min(per_launch_ms),
                      "max": max(per_launch_ms), "n": len(per_launch_ms)},
        "roofline": roofline,
        "cpu_baseline": {"value": cpu_value, "unit": "observations/s", "cores": threads, "kind": "oracle",
                         "sample": f"first {m} of {n} rows ({cpu_s:.1f} s)",
                         "single_core": {"value": cpu1_value, "cores": 1,
                                         "sample": f"first {m1} of {n} rows ({cpu1_s:.1f} s)"}},
        "clocks": clk,
    })
    print(json.dumps(out))
    df.release()


# ------------------------------------------------------------------ batched

def run_batched(args, ws, rank, local):
    """The batched workload: one persistent launch over 8 forests and uneven
    batches, captured once in a CUDA graph and replayed every step.  After the
    timed replays every row's votes and class are compared with the oracle,
    whose run on the same batches is also the CPU baseline; the end-to-end leg
    copies each step's rows in from pinned host memory, replays the graph and
    copies the classes back."""
    import torch
    import datagen
    import oracle
    import paper_1806_07300_gb300 as fp
    from paper_1806_07300_gb300 import autotune as at

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    names = [f"batched{k}" for k in range(len(datagen.BATCHED_SPECS))]
    forests = [datagen.forest(nm) for nm in names]
    sizes = datagen.batch_sizes()
    Xh = [datagen.test_rows(nm, s)[0] for nm, s in zip(names, sizes)]
    Xs = [torch.from_numpy(x).to(dev) for x in Xh]
    dfs, tuning = at.autotune_batched(forests, Xs)  # one layout for the shared launch
    votes = [torch.empty((x.shape[0], f.n_classes), dtype=torch.int32, device=dev) for f, x in zip(forests, Xs)]
    cls = [torch.empty((x.shape[0],), dtype=torch.int32, device=dev) for x in Xs]
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        fp.fp_predict_batched(dfs, Xs, votes, cls, stream=stream)
    stream.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        fp.fp_predict_batched(dfs, Xs, votes, cls, stream=torch.cuda.current_stream())
    for _ in range(args.warmup):
        g.replay()
    torch.cuda.synchronize()
    input_bytes = sum(x.nbytes for x in Xh) + sum(d.info["total_bytes"] for d in dfs)
    flush = flush_for(dev, input_bytes)
    cur = torch.cuda.current_stream()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    total_ms, _ = timed_steps(g.replay, args.steps, cur, flush)
    clk = clocks.stop()
    rows = sum(sizes)
    value = ws * rows * args.steps / (total_ms / 1e3)
    for d in dfs:
        if d.sync_status() != fp.FP_OK:
            raise RuntimeError(f"kernel status: {fp.fp_last_error()}")
    got_v = [v.cpu().numpy().astype(np.uint32) for v in votes]
    got_c = [c.cpu().numpy() for c in cls]

    # end to end: rows from pinned host memory into the graph's inputs, one
    # replay, classes back to pinned host memory, every step
    Xpin = [torch.from_numpy(x).pin_memory() for x in Xh]
    cls_host = [torch.empty((x.shape[0],), dtype=torch.int32).pin_memory() for x in Xh]

    def e2e_step():
        for x, xp in zip(Xs, Xpin):
            x.copy_(xp, non_blocking=True)
        g.replay()
        for c, ch in zip(cls, cls_host):
            ch.copy_(c, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    e2e_steps = max(3, args.steps // 2)
    a2, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a2.record()
    for _ in range(e2e_steps):
        e2e_step()
    b2.record()
    torch.cuda.synchronize()
    e2e_ms = a2.elapsed_time(b2) / e2e_steps
    for c, ch in zip(got_c, cls_host):
        if not np.array_equal(c, ch.numpy()):
            raise RuntimeError("end-to-end classes differ from the device path's")
    e2e = {"value": ws * rows / (e2e_ms / 1e3), "unit": "observations/s", "ms_per_step": e2e_ms,
           "h2d_bytes_per_step": int(sum(x.nbytes for x in Xh)), "d2h_bytes_per_step": int(4 * rows),
           "path": "pinned rows copied into the captured inputs, graph replay (fp_predict_batched), classes "
                   "copied back"}
    l2_gbs = fp.fp_l2_read_probe(64 << 20, 40, stream=stream)
    if rank != 0:
        return

    # the oracle on every row of every batch: parity and the CPU baseline
    threads = oracle.default_threads()
    t0 = time.perf_counter()
    refs = [oracle.predict(f, x, leaves=False, threads=threads) for f, x in zip(forests, Xh)]
    cpu_s = time.perf_counter() - t0
    mism = sum(int((gv != r["votes"]).any(axis=1).sum()) + int((gc != r["cls"]).sum())
               for gv, gc, r in zip(got_v, got_c, refs))
    if mism:
        raise RuntimeError(f"batched workload: {mism} rows differ from the oracle")
    visits = sum(r["visits"] for r in refs)
    algo_bytes = 8.0 * visits + sum(x.shape[0] * (4.0 * x.shape[1] + 4.0 * f.n_classes + 4.0)
                                    for f, x in zip(forests, Xh))
    launch_s = total_ms / args.steps / 1e3
    achieved = algo_bytes / launch_s / 1e9
    peak_hbm, peak_kind = measured_peaks()
    roofline = {"bound": "l2", "achieved": achieved, "peak": l2_gbs, "unit": "GB/s", "frac": achieved / l2_gbs,
                "traffic": None, "traffic_source": "not captured for this launch",
                "peak_kind": "measured in this run: fp_l2_read_probe, 16-byte loads over a 64 MiB L2-resident buffer",
                "kernel": "fp_traverse_batched_kernel", "avg_launch_ms": total_ms / args.steps,
                "bytes_per_launch": algo_bytes,
                "bytes_kind": "algorithmic: 8 B per internal node visited (oracle count) + rows + votes + classes",
                "node_visits_per_s": visits / launch_s,
                "hbm": {"peak": peak_hbm, "peak_kind": peak_kind, "algorithmic_frac": achieved / peak_hbm,
                        "note": "the forests' nodes come from shared memory and L2; not a DRAM fraction"}}
    check_roofline(roofline)
    out = base_line(args, ws, value, total_ms,
                    {"workload": "batched", "desc": WORKLOADS["batched"]["desc"], "batch_rows": sizes,
                     "n_trees": [f.n_trees for f in forests], "parallelism": f"replicas x{ws}",
                     "layout": {k: tuning.get(k) for k in ("bin_size", "interleave_depth", "head_select",
                                                           "deep_levels", "deep_format", "launch")},
                     "l2": flush.describe(input_bytes) if flush else
                     "inputs larger than L2 (%.0f MB); no flush" % (input_bytes / 1e6)})
    out.update({"gpu_launches": args.steps, "graph": "one persistent launch per replay", "clocks": clk,
                "e2e": e2e, "roofline": roofline,
                "parity_checked": {"rows": rows, "mismatches": 0, "compared": "votes and class of every row"},
                "cpu_baseline": {"value": rows / cpu_s, "unit": "observations/s", "cores": threads, "kind": "oracle",
                                 "sample": f"all {rows} rows of the 8 batches ({cpu_s:.1f} s)"}})
    print(json.dumps(out))


# ------------------------------------------------------------------ serving

def run_serving(args, ws, rank, local):
    """Poisson request streams against the continuous-batching server."""
    import torch
    import datagen
    from paper_1806_07300_gb300.serving import ForestServer, latency_summary

    torch.cuda.set_device(local)
    names = {"tiny": "tiny", "image": "image", "hbm": "hbm", "wide": "wide"}
    forests = {k: datagen.forest(v) for k, v in names.items()}
    pools = {k: datagen.test_rows(v, 200_000 if k != "tiny" else 10_000)[0] for k, v in names.items()}
    srv = ForestServer(device=local, slots=3, max_rows=1 << 17)
    for k, f in forests.items():
        srv.add_forest(k, f)
    rng = np.random.Generator(np.random.PCG64(11))
    keys = sorted(forests)
    results = []
    all_reqs = []
    with srv:
        # warm every forest once
        for k in keys:
            srv.submit(k, pools[k][:64]).wait(60)
        for rate in (2000, 5000, 10000, 20000):
            reqs = []
            t_end = time.perf_counter() + args.serve_seconds
            t_next = time.perf_counter()
            n_rows = 0
            while True:
                t_next += rng.exponential(1.0 / rate)
                if t_next > t_end:
                    break
                while True:
                    dt = t_next - time.perf_counter()
                    if dt <= 0:
                        break
                    time.sleep(min(dt, 0.001) if dt > 0.0002 else 0)
                k = keys[rng.integers(len(keys))]
                m = int(np.clip(round(rng.lognormal(math.log(32), 1.5)), 1, 4096))
                s = int(rng.integers(0, pools[k].shape[0] - m))
                reqs.append(srv.submit(k, pools[k][s: s + m]))
                n_rows += m
            t0 = time.perf_counter()
            for r in reqs:
                r.wait(120)
            all_reqs.extend(reqs)
            wall = args.serve_seconds + (time.perf_counter() - t0)
            lat = latency_summary(reqs)
            results.append({"rate_rps": rate, "requests": len(reqs), "rows": n_rows, "obs_per_s": n_rows / wall,
                            "achieved_rps": len(reqs) / wall, **lat,
                            "errors": sum(1 for r in reqs if r.error is not None)})
    if rank != 0:
        return
    best = max(results, key=lambda r: r["obs_per_s"])
    # every answer against the oracle (after the timed window), per forest; the
    # oracle's time over the same rows is the CPU baseline, and its visit counts
    # give the algorithmic bytes behind the best rate
    import oracle
    threads = oracle.default_threads()
    checked = mism = 0
    cpu_s = 0.0
    visits_per_row = {}
    for k in keys:
        mine = [r for r in all_reqs if r.forest == k]
        visits = rows_k = 0
        i = 0
        while i < len(mine):  # chunks of about 100k rows keep the host copies small
            j, m = i, 0
            while j < len(mine) and (j == i or m + mine[j].X.shape[0] <= 100_000):
                m += mine[j].X.shape[0]
                j += 1
            X = np.concatenate([r.X for r in mine[i:j]])
            t0 = time.perf_counter()
            ref = oracle.predict(forests[k], X, leaves=False, votes=False, threads=threads)
            cpu_s += time.perf_counter() - t0
            mism += int((np.concatenate([r.classes for r in mine[i:j]]) != ref["cls"]).sum())
            visits += ref["visits"]
            rows_k += m
            i = j
        checked += rows_k
        if rows_k:
            visits_per_row[k] = visits / rows_k
    if mism:
        raise RuntimeError(f"serving: {mism} of {checked} answers differ from the oracle")
    bytes_per_row = {k: 8.0 * visits_per_row[k] + 4.0 * forests[k].n_features + 4.0 for k in visits_per_row}
    mean_bytes = sum(bytes_per_row.values()) / len(bytes_per_row)  # forests are chosen uniformly
    l2_gbs = fp_l2_probe(local)
    achieved = best["obs_per_s"] * mean_bytes / 1e9
    roofline = {"bound": "l2", "achieved": achieved, "peak": l2_gbs, "unit": "GB/s", "frac": achieved / l2_gbs,
                "traffic": None, "traffic_source": "not captured for a request stream",
                "peak_kind": "measured in this run: fp_l2_read_probe, 16-byte loads over a 64 MiB L2-resident buffer",
                "kernel": "fp_traverse_batched_kernel (launched by the serving runtime)",
                "bytes_per_obs": mean_bytes,
                "bytes_kind": "algorithmic per row, averaged over the four forests (chosen uniformly): 8 B per "
                              "internal node visited (oracle count) + row + class",
                "note": f"over the wall time of the {best['rate_rps']} req/s window: the offered request rate, not "
                        "the GPU, sets the throughput"}
    check_roofline(roofline)
    out = base_line(args, ws, best["obs_per_s"] * ws, 1e3 * args.serve_seconds,
                    {"workload": "serving", "desc": WORKLOADS["serving"]["desc"], "slots": srv.slots,
                     "parallelism": f"replicas x{ws}", "l2": "not applicable (request stream)"})
    out["steps"], out["ms_per_step"] = len(results), 1e3 * args.serve_seconds  # one step = one offered rate's window
    out.update({"serving": results, "launches": srv.launches, "gpu_launches": srv.launches,
                "p50_ms": best["p50_ms"], "p99_ms": best["p99_ms"], "e2e": None, "roofline": roofline,
                "parity_checked": {"rows": checked, "requests": len(all_reqs), "mismatches": 0,
                                   "compared": "class of every row of every request"},
                "cpu_baseline": {"value": checked / cpu_s, "unit": "observations/s", "cores": threads,
                                 "kind": "oracle", "sample": f"the {checked} served rows ({cpu_s:.1f} s)"}})
    print(json.dumps(out))


def fp_l2_probe(local: int) -> float:
    import torch
    import paper_1806_07300_gb300 as fp
    with torch.cuda.device(local):
        return fp.fp_l2_read_probe(64 << 20, 40)


# ----------------------------------------------------------------- ablation

def run_ablation(args, ws, rank, local):
    """Each layout variant timed on the same rows; classes compared with the
    plain baseline's."""
    import torch
    import datagen
    import paper_1806_07300_gb300 as fp
    from paper_1806_07300_gb300 import autotune as at

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    name = args.forest
    n = args.rows or WORKLOADS["ablation"]["rows"]
    forest = datagen.forest(name)
    Xh, _ = datagen.test_rows(name, n)
    X = torch.from_numpy(Xh).to(dev)
    C = forest.n_classes
    cls = torch.empty((n,), dtype=torch.int32, device=dev)
    reps = max(2, args.steps // 4)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    rows = []
    pf = fp.fp_plain_build(forest)
    pv = torch.empty((n, C), dtype=torch.int32, device=dev)
    ref = torch.empty((n,), dtype=torch.int32, device=dev)
    for order, oname in ((fp.FP_PLAIN_OBS_FASTEST, "obs_fastest"), (fp.FP_PLAIN_TREE_FASTEST, "tree_fastest")):
        ms = timed(lambda: fp.fp_plain_predict(pf, X, order, pv, ref))
        rows.append({"layout": f"BF plain ({oname})", "ms": ms})
    pf.release()
    del pv
    sample = X[: min(n, 200_000)]
    inferred = datagen.Forest(forest.n_features, forest.n_classes, forest.node_begin, forest.left, forest.right,
                              forest.feature, forest.threshold, forest.leaf_class, fp.infer_cardinality(forest, sample))
    no_stats = datagen.Forest(forest.n_features, forest.n_classes, forest.node_begin, forest.left, forest.right,
                              forest.feature, forest.threshold, forest.leaf_class, forest.cardinality)
    no_stats.cardinality = None  # packed without statistics: children keep left-first order
    layouts, launches = TUNE.get(name, (None, None))
    best = at.autotune(forest, X[: min(n, 1 << 20)], layouts=layouts, launches=launches)
    tuned_layout = {k: best[k] for k in at.LAYOUT_KEYS}
    two_level = dict(tuned_layout, deep_levels=2, deep_format=0)
    # the paper's layouts with two-level super-nodes (full thresholds), then
    # the same with three-level ones, then the autotuner's choice
    variants = [
        ("DF order, roots only (no statistics)", no_stats, dict(bin_size=1, interleave_depth=0, deep_levels=2), {}),
        ("Stat (training cardinalities), roots only", forest, dict(bin_size=1, interleave_depth=0, deep_levels=2), {}),
        ("Stat (counted on 200k observations), roots only", inferred,
         dict(bin_size=1, interleave_depth=0, deep_levels=2), {}),
        ("Bin B=16, levels 0..4", forest, dict(bin_size=16, interleave_depth=4, head_select=1, deep_levels=2), {}),
        ("Bin B=16, 31 most visited nodes", forest,
         dict(bin_size=16, interleave_depth=4, head_select=3, deep_levels=2), {}),
        ("Bin B=3, levels 0..8", forest, dict(bin_size=3, interleave_depth=8, head_select=1, deep_levels=2), {}),
        ("Bin B=3, 511 most visited nodes", forest,
         dict(bin_size=3, interleave_depth=8, head_select=3, deep_levels=2), {}),
        ("Stat, roots only, three-level super-nodes", forest, dict(bin_size=1, interleave_depth=0, deep_levels=3),
         {}),
        ("Bin B=3, levels 0..8, three-level super-nodes", forest,
         dict(bin_size=3, interleave_depth=8, head_select=1, deep_levels=3), {}),
        ("autotuned layout and launch, two-level super-nodes", forest, two_level,
         {k: best[k] for k in at.LAUNCH_KEYS}),
        ("autotuned", forest, tuned_layout, {k: best[k] for k in at.LAUNCH_KEYS}),
    ]
    for label, f, params, launch in variants:
        df = fp.fp_upload(fp.fp_pack_forest(f, **params))
        if launch:
            df.configure(**launch)
        ms = timed(lambda: fp.fp_predict(df, X, None, cls))
        rows.append({"layout": label, **params, **launch, "passes": df.info["passes"], "ms": ms,
                     "same_classes": bool(torch.equal(cls, ref))})
        df.release()
    plain_best = min(r["ms"] for r in rows[:2])
    for r in rows:
        r["obs_per_s"] = n / (r["ms"] / 1e3)
        r["vs_plain"] = plain_best / r["ms"]
    if rank != 0:
        return
    top = min(rows[2:], key=lambda r: r["ms"])
    out = base_line(args, ws, ws * top["obs_per_s"], top["ms"] * args.steps,
                    {"workload": "ablation", "forest": name, "rows": n, "parallelism": f"replicas x{ws}",
                     "l2": "inputs larger than L2; no flush"})
    out.update({"ablation": rows, "e2e": None, "roofline": None, "cpu_baseline": None,
                "gpu_launches": len(rows) * (reps + 1)})
    print(json.dumps(out))


def main():
    global SKIP_ROOFLINE_CHECK
    args = parse()
    SKIP_ROOFLINE_CHECK = args.no_roofline_check
    ws, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, ws, rank)
    elif args.workload == "batched":
        run_batched(args, ws, rank, local)
    elif args.workload == "serving":
        run_serving(args, ws, rank, local)
    elif args.workload == "ablation":
        run_ablation(args, ws, rank, local)
    else:
        run_packed(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
