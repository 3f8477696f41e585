"""Autotuner for the packed layout and the traversal launch.

Searches the paper's two layout parameters -- stripe width B (trees per bin)
and interleaved depth d (Section III-A; Fig. 2 sweeps the same pair) -- with
the kind of head (the interleaved levels 0..d, or the most visited nodes),
and the launch parameters of the traversal kernel (observations per tile, warps
per CTA, ring refill level) by timing fp_predict on a sample of the caller's
observations.  Results are cached per (forest, device, sample size) in a JSON
file, so a resident forest is tuned once.  All timing runs through the C ABI.
"""
from __future__ import annotations

import hashlib
import json
import os
import time

import numpy as np

from . import FPError, fp_pack_forest, fp_predict, fp_predict_values, fp_upload

_BLOCK_LIMIT = 48 * 1024  # bytes of one bin's interleaved block considered by default
LAYOUT_KEYS = ("bin_size", "interleave_depth", "head_select", "deep_levels", "deep_format")
_SEARCH_VERSION = "deep3-v8"  # cached results of an older search space are not reused
LAUNCH_KEYS = ("obs_tile", "warps_per_cta", "refill_lanes", "bin_buffers")


def block_bytes(bin_size: int, depth: int, head_select: int = 1) -> int:
    """Size of a bin's interleaved block when every tree fills its head
    (paired level heads: (4^J - 1)/3 records of 16 bytes, J = (d+1)/2)."""
    stride = bin_size | 1
    k = (1 << (depth + 1)) - 1
    if head_select == 2:
        return stride * (k // 3) * 16 + stride * (k + 1) * 4
    return stride * k * 8 + stride * (k + 1) * 4


def candidate_layouts(n_trees: int, limit: int = _BLOCK_LIMIT, max_layouts: int | None = None
                      ) -> list[tuple[int, ...]]:
    """(B, d, head_select[, deep_levels]) tuples to try: for bins of 1, 3, 8,
    16 and 64 trees, the deepest paired level head (head_select 2, d odd) and
    the deepest level head (head_select 1) whose block fits the limit, and a
    small paired head (d = 3), which leaves shared memory to tiles of wide
    rows or to a second CTA per SM; one ranked head (head_select 3); all with
    the library's default super-nodes, and the first paired head of bins of
    3 again with two-level super-nodes."""
    out = []

    def add(c):
        if c not in out:
            out.append(c)

    for B in (1, 3, 8, 16, 64):
        B = min(B, n_trees)
        odd = [d for d in (1, 3, 5, 7, 9, 11) if block_bytes(B, d, 2) <= limit]
        if odd:
            add((B, max(odd), 2))
        add((B, max(d for d in range(12) if block_bytes(B, d) <= limit or d == 0), 1))
        add((B, 3, 2))
    B = min(3, n_trees)
    add((B, min(9, max(d for d in range(10) if block_bytes(B, d, 3) <= limit or d == 0)), 3))
    first3 = [c for c in out if c[0] == B and c[2] == 2]
    if first3:
        add(first3[0] + (2,))
    if max_layouts is not None and len(out) > max_layouts:
        idx = np.linspace(0, len(out) - 1, max_layouts).round().astype(int)
        out = [out[i] for i in sorted(set(idx))]
    return out


def candidate_launches(default_tile: int) -> list[tuple[int, int, int, int]]:
    """(obs_tile, warps_per_cta, refill_lanes, bin_buffers) tuples."""
    tiles = sorted({default_tile, max(32, default_tile // 2 // 32 * 32)}, reverse=True)
    return [(t, w, r, nb) for t in tiles for w in (32, 16) for r in (16, 8) for nb in (3, 2)]


def forest_key(forest) -> str:
    h = hashlib.sha1()
    for name in ("node_begin", "left", "right", "feature", "threshold", "leaf_class", "cardinality"):
        a = getattr(forest, name, None)
        if a is None:
            continue
        a = np.ascontiguousarray(a)
        h.update(name.encode())
        h.update(np.int64(a.size).tobytes())
        step = max(1, a.size // 65536)  # a sample of the arrays keeps hashing cheap
        h.update(a[::step].tobytes())
    return h.hexdigest()[:16]


def _cache_path() -> str:
    root = os.environ.get("FP_CACHE_DIR") or os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                                                          ".fpcache")
    os.makedirs(root, exist_ok=True)
    return os.path.join(root, "autotune.json")


def _time_predict(df, X, out, reps: int) -> float:
    """Milliseconds per call: classes (int32 out) or, for a forest with leaf
    values, the value output (float32 out); at least `reps` calls, more for
    short ones."""
    import torch
    if out.dtype == torch.float32:
        call = lambda: fp_predict_values(df, X, out, df.value_scale, df.value_bias)  # noqa: E731
    else:
        call = lambda: fp_predict(df, X, None, out)  # noqa: E731
    call()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    call()
    b.record()
    torch.cuda.synchronize()
    # short calls (small batches) are repeated until about 20 ms are timed
    reps = max(reps, min(500, int(20.0 / max(a.elapsed_time(b), 1e-3))))
    a.record()
    for _ in range(reps):
        call()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def _same(ref, out) -> bool:
    """Classes must agree exactly; value outputs (float sums in no fixed
    order) to within a relative 1e-4."""
    import torch
    if out.dtype != torch.float32:
        return bool(torch.equal(ref, out))
    return bool(torch.all((ref - out).abs() <= 1e-4 * (1.0 + ref.abs())))


def autotune(forest, X, layouts=None, launches=None, reps: int = 3, use_cache: bool = True,
             verbose: bool = False) -> dict:
    """Time every (layout, launch) candidate on the device rows X (a CUDA
    float32 tensor [n][n_features]) and return the fastest as a dict of
    fp_pack_forest keyword arguments plus "ms" and the full "table"."""
    import torch
    key = f"{forest_key(forest)}:{torch.cuda.get_device_name()}:{X.shape[0]}:{_SEARCH_VERSION}"
    path = _cache_path()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            with open(path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
        if key in cache:
            return cache[key]
    layouts = layouts or candidate_layouts(forest.n_trees)
    values = getattr(forest, "leaf_value", None) is not None
    cls = torch.empty((X.shape[0],), dtype=torch.float32 if values else torch.int32, device=X.device)
    table = []
    ref = None
    for lay in layouts:
        B, d = lay[0], lay[1]
        sel = lay[2] if len(lay) > 2 else 0  # 0: the library's default head kind
        dl = lay[3] if len(lay) > 3 else 0   # 0: the library's default super-nodes
        fmt = lay[4] if len(lay) > 4 else 0  # 0: the library's default three-level format
        t0 = time.perf_counter()
        try:
            df = fp_upload(fp_pack_forest(forest, bin_size=B, interleave_depth=d, head_select=sel, deep_levels=dl,
                                          deep_format=fmt))
        except FPError as e:
            table.append(dict(bin_size=B, interleave_depth=d, head_select=sel, deep_levels=dl, deep_format=fmt,
                              error=str(e)))
            continue
        dl, fmt = df.info["deep_levels"], df.info["deep_format"]
        pack_s = time.perf_counter() - t0
        for launch in (launches or candidate_launches(df.info["obs_tile"])):
            tile, warps, refill = launch[:3]
            nbuf = launch[3] if len(launch) > 3 else 3
            try:
                df.configure(obs_tile=tile, warps_per_cta=warps, refill_lanes=refill, bin_buffers=nbuf)
            except FPError as e:
                table.append(dict(bin_size=B, interleave_depth=d, head_select=sel, deep_levels=dl, deep_format=fmt,
                                  obs_tile=tile, warps_per_cta=warps, refill_lanes=refill, bin_buffers=nbuf,
                                  error=str(e)))
                continue
            ms = _time_predict(df, X, cls, reps)
            if ref is None:
                ref = cls.clone()
            same = _same(ref, cls)
            row = dict(bin_size=B, interleave_depth=d, head_select=sel, deep_levels=dl, deep_format=fmt,
                       obs_tile=df.info["obs_tile"],
                       warps_per_cta=warps, bin_buffers=nbuf,
                       refill_lanes=refill, passes=df.info["passes"], ms=ms, pack_s=pack_s, same_classes=same)
            table.append(row)
            if verbose:
                print(json.dumps(row), flush=True)
        df.release()
    timed = [r for r in table if "ms" in r]
    if not timed:
        raise RuntimeError("autotune: no candidate could run")
    if not all(r["same_classes"] for r in timed):
        raise RuntimeError("autotune: candidates disagree on classes")
    best = min(timed, key=lambda r: r["ms"])
    result = {k: best[k] for k in LAYOUT_KEYS + LAUNCH_KEYS}
    result["ms"] = best["ms"]
    result["rows"] = int(X.shape[0])
    result["table"] = table
    if use_cache:
        cache[key] = result
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f)
        os.replace(tmp, path)
    return result


def upload_tuned(forest, X, **kw):
    """Autotune on X, then pack, upload and configure the forest with the best
    parameters.  Returns (DeviceForest, tuning result)."""
    best = autotune(forest, X, **kw)
    df = fp_upload(fp_pack_forest(forest, **{k: best[k] for k in LAYOUT_KEYS}))
    df.configure(**{k: best[k] for k in LAUNCH_KEYS})
    return df, best


# (B, d, head_select[, deep_levels[, deep_format]]): with two-level super-nodes,
# or three-level ones of format 2, for all, every forest of the launch has the
# same kind of super-node (one walk compiled into the batched kernel); by
# default forests of few features and classes take format 1, the others 2
BATCHED_LAYOUTS = [(3, 9, 2), (3, 9, 2, 2), (3, 9, 2, 3, 2), (8, 7, 2), (8, 7, 2, 2), (8, 7, 2, 3, 2), (4, 8, 1),
                   (16, 5, 2)]
BATCHED_LAUNCHES = [(0, 32, 16, 3), (0, 32, 32, 3)]


def autotune_batched(forests, Xs, layouts=None, launches=None, reps: int = 10) -> tuple[list, dict]:
    """Tune one persistent launch over several forests (fp_predict_batched):
    every forest gets the same layout and launch parameters, and each
    candidate is timed as the whole batched call, since the forests share its
    CTAs (per-forest tuning does not predict the shared launch).  Returns
    (device forests configured with the best candidate, result dict)."""
    import torch
    from . import fp_predict_batched
    table, best, best_dfs = [], None, None
    votes = [torch.empty((x.shape[0], f.n_classes), dtype=torch.int32, device=x.device) for f, x in zip(forests, Xs)]
    cls = [torch.empty((x.shape[0],), dtype=torch.int32, device=x.device) for x in Xs]
    for lay in (layouts or BATCHED_LAYOUTS):
        B, d, sel = lay[:3]
        dl = lay[3] if len(lay) > 3 else 0
        fmt = lay[4] if len(lay) > 4 else 0
        try:
            dfs = [fp_upload(fp_pack_forest(f, bin_size=min(B, f.n_trees), interleave_depth=d, head_select=sel,
                                            deep_levels=dl, deep_format=fmt)) for f in forests]
        except FPError as e:
            table.append(dict(bin_size=B, interleave_depth=d, head_select=sel, deep_levels=dl, deep_format=fmt,
                              error=str(e)))
            continue
        for launch in (launches or BATCHED_LAUNCHES):
            tile, warps, refill, nbuf = launch
            try:
                for df in dfs:
                    df.configure(obs_tile=tile, warps_per_cta=warps, refill_lanes=refill, bin_buffers=nbuf)
            except FPError as e:
                table.append(dict(bin_size=B, interleave_depth=d, head_select=sel, deep_levels=dl, deep_format=fmt,
                                  launch=launch, error=str(e)))
                continue
            fp_predict_batched(dfs, Xs, votes, cls)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(reps):
                fp_predict_batched(dfs, Xs, votes, cls)
            b.record()
            torch.cuda.synchronize()
            row = dict(bin_size=B, interleave_depth=d, head_select=sel, deep_levels=dl, deep_format=fmt,
                       launch=list(launch), ms=a.elapsed_time(b) / reps)
            table.append(row)
            if best is None or row["ms"] < best["ms"]:
                if best_dfs is not None and best_dfs[0] is not dfs:
                    for df in best_dfs[0]:  # the previous best layout's forests
                        df.release()
                best, best_dfs = row, (dfs, launch)
        if best_dfs is None or best_dfs[0] is not dfs:
            for df in dfs:
                df.release()
    if best is None:
        raise RuntimeError("autotune_batched: no candidate could run")
    dfs, launch = best_dfs
    tile, warps, refill, nbuf = launch
    for df in dfs:
        df.configure(obs_tile=tile, warps_per_cta=warps, refill_lanes=refill, bin_buffers=nbuf)
    return dfs, dict(best, table=table)
