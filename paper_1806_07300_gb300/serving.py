"""Continuous-batching classification server over resident packed forests.

Forests stay resident on the device.  Requests (a few rows for one forest)
arrive from any thread; a batcher thread groups whatever has arrived into one
persistent launch over all the forests involved (fp_predict_batched), so
requests of different sizes and forests share a launch.  Up to `slots`
launches are in flight at once, each on its own CUDA stream: requests that
arrive while earlier launches run are admitted as soon as a slot and enough
device memory are free (free memory from torch.cuda.mem_get_info, minus a
margin), and their work overlaps on the device with the launches in flight.
A completion thread polls each launch's event and hands every request its
classes (and votes) back; latency is measured from submit to completion.

Every step of classification runs in the CUDA library; this module only
moves rows and results between host and device and schedules launches.
"""
from __future__ import annotations

import collections
import threading
import time

import numpy as np

from . import FPError, fp_pack_forest, fp_predict_batched, fp_upload


class Request:
    """One classification request; wait() blocks until its result is ready."""

    __slots__ = ("forest", "X", "t_submit", "t_done", "classes", "votes", "error", "_done")

    def __init__(self, forest: str, X: np.ndarray):
        self.forest = forest
        self.X = X
        self.t_submit = time.perf_counter()
        self.t_done = None
        self.classes = None
        self.votes = None
        self.error = None
        self._done = threading.Event()

    def wait(self, timeout: float | None = None) -> bool:
        return self._done.wait(timeout)

    @property
    def latency_s(self) -> float | None:
        return None if self.t_done is None else self.t_done - self.t_submit


class _Resident:
    def __init__(self, name, df, n_features, n_classes):
        self.name = name
        self.df = df
        self.F = n_features
        self.C = n_classes


class ForestServer:
    """Serve classification requests for several resident forests.

    slots            launches in flight at most (one CUDA stream each)
    max_rows         rows per launch at most
    mem_margin       device bytes kept free when admitting a launch
    return_votes     also return per-class vote counts
    """

    def __init__(self, device: int = 0, slots: int = 2, max_rows: int = 1 << 18, mem_margin: int = 256 << 20,
                 return_votes: bool = False, max_wait_s: float = 0.0):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", device)
        self.slots = slots
        self.max_rows = max_rows
        self.mem_margin = mem_margin
        self.return_votes = return_votes
        self.max_wait_s = max_wait_s
        self.forests: dict[str, _Resident] = {}
        self._queue: collections.deque[Request] = collections.deque()
        self._cv = threading.Condition()
        self._inflight: collections.deque = collections.deque()
        self._free_slots = list(range(slots))
        self._slot_cv = threading.Condition()
        self._streams = [torch.cuda.Stream(device=self.device) for _ in range(slots)]
        self._pin_in = [None] * slots   # pinned staging of each slot's rows
        self._pin_out = [None] * slots  # pinned landing of each slot's classes and votes
        self._stop = False
        self._batcher_done = False
        self._threads: list[threading.Thread] = []
        self.completed: list[Request] = []
        self.launches = 0
        self.rejected_for_memory = 0

    # ------------------------------------------------------------ forests
    def add_forest(self, name: str, forest, **pack_params) -> None:
        """Pack, upload and keep a forest resident under `name`."""
        with self.torch.cuda.device(self.device):
            df = fp_upload(fp_pack_forest(forest, **pack_params))
        self.forests[name] = _Resident(name, df, forest.n_features, forest.n_classes)

    def add_device_forest(self, name: str, df, n_features: int, n_classes: int) -> None:
        self.forests[name] = _Resident(name, df, n_features, n_classes)

    # ------------------------------------------------------------ requests
    def submit(self, forest: str, X: np.ndarray) -> Request:
        if forest not in self.forests:
            raise KeyError(forest)
        X = np.ascontiguousarray(X, dtype=np.float32)
        if X.ndim != 2 or X.shape[1] != self.forests[forest].F:
            raise ValueError("rows must be [m][n_features] of the forest")
        req = Request(forest, X)
        with self._cv:
            self._queue.append(req)
            self._cv.notify()
        return req

    def start(self) -> "ForestServer":
        self._stop = False
        self._batcher_done = False
        self._threads = [threading.Thread(target=self._batcher, daemon=True),
                         threading.Thread(target=self._completer, daemon=True)]
        for t in self._threads:
            t.start()
        return self

    def stop(self) -> None:
        with self._cv:
            self._stop = True
            self._cv.notify_all()
        with self._slot_cv:
            self._slot_cv.notify_all()
        for t in self._threads:
            t.join()

    def __enter__(self):
        return self.start()

    def __exit__(self, *exc):
        self.stop()

    # ------------------------------------------------------------ internals
    def _take_batch(self) -> list[Request]:
        """Requests for one launch: FIFO, up to max_rows rows (at least one request)."""
        with self._cv:
            while not self._queue and not self._stop:
                self._cv.wait(0.05)
            if self._stop and not self._queue:
                return []
            if self.max_wait_s > 0:
                deadline = self._queue[0].t_submit + self.max_wait_s
                while (sum(r.X.shape[0] for r in self._queue) < self.max_rows and time.perf_counter() < deadline
                       and not self._stop):
                    self._cv.wait(max(0.0, deadline - time.perf_counter()))
            batch, rows = [], 0
            while self._queue and (not batch or rows + self._queue[0].X.shape[0] <= self.max_rows):
                r = self._queue.popleft()
                batch.append(r)
                rows += r.X.shape[0]
            return batch

    def _pinned(self, bufs: list, slot: int, nbytes: int):
        """A slot's pinned host buffer of at least nbytes (grown by doubling).
        A slot is reused only after its launch completed, so reuse is safe."""
        b = bufs[slot]
        if b is None or b.numel() < nbytes:
            size = max(nbytes, 1 << 20, 2 * (b.numel() if b is not None else 0))
            bufs[slot] = b = self.torch.empty(size, dtype=self.torch.uint8, pin_memory=True)
        return b

    def _admit(self, nbytes: int) -> bool:
        info = getattr(self, "_admit_info", None) or self.torch.cuda.mem_get_info
        free, _ = info(self.device)
        return free >= nbytes + self.mem_margin

    def _batcher(self) -> None:
        try:
            self._batch_loop()
        finally:
            with self._slot_cv:
                self._batcher_done = True
                self._slot_cv.notify_all()

    def _batch_loop(self) -> None:
        torch = self.torch
        while True:
            batch = self._take_batch()
            if not batch:
                return
            # group by forest, keeping arrival order within a forest
            groups: dict[str, list[Request]] = collections.OrderedDict()
            for r in batch:
                groups.setdefault(r.forest, []).append(r)
            nbytes = sum(sum(r.X.shape[0] for r in rs) * 4 * (self.forests[n].F + self.forests[n].C + 1)
                         for n, rs in groups.items())
            while not self._admit(nbytes):  # wait for launches in flight to free memory
                self.rejected_for_memory += 1
                with self._slot_cv:
                    if not self._inflight:
                        break
                    self._slot_cv.wait(0.01)
            with self._slot_cv:
                while not self._free_slots and not self._stop:
                    self._slot_cv.wait(0.05)
                if not self._free_slots:
                    for r in batch:
                        r.error = "server stopped"
                        r._done.set()
                    return
                slot = self._free_slots.pop()
            stream = self._streams[slot]
            try:
                names = list(groups)
                rows = [sum(r.X.shape[0] for r in groups[nm]) for nm in names]
                in_bytes = [m * self.forests[nm].F * 4 for nm, m in zip(names, rows)]
                out_words = [m * (1 + (self.forests[nm].C if self.return_votes else 0)) for nm, m in zip(names, rows)]
                pin_in = self._pinned(self._pin_in, slot, sum(in_bytes))
                pin_out = self._pinned(self._pin_out, slot, 4 * sum(out_words))
                with torch.cuda.device(self.device), torch.cuda.stream(stream):
                    forests, Xs, votes, classes, spans, outs = [], [], [], [], [], []
                    off_in = off_out = 0
                    for nm, m, nb, nw in zip(names, rows, in_bytes, out_words):
                        res = self.forests[nm]
                        rs = groups[nm]
                        xh = pin_in[off_in: off_in + nb].view(torch.float32).view(m, res.F)
                        xn = xh.numpy()
                        o = 0
                        for r in rs:  # gather the requests' rows into pinned memory
                            xn[o: o + r.X.shape[0]] = r.X
                            o += r.X.shape[0]
                        xd = xh.to(self.device, non_blocking=True)
                        c = torch.empty((m,), dtype=torch.int32, device=self.device)
                        v = torch.empty((m, res.C), dtype=torch.int32, device=self.device) if self.return_votes else None
                        forests.append(res.df)
                        Xs.append(xd)
                        votes.append(v)
                        classes.append(c)
                        spans.append((rs, None))
                        outs.append((off_out, m, res.C))
                        off_in += nb
                        off_out += nw
                    fp_predict_batched(forests, Xs, votes if self.return_votes else None, classes, stream=stream)
                    ow = pin_out.view(torch.int32)
                    c_host, v_host = [], ([] if self.return_votes else None)
                    for (oo, m, C), c, v in zip(outs, classes, votes):
                        ch = ow[oo: oo + m]
                        ch.copy_(c, non_blocking=True)
                        c_host.append(ch)
                        if self.return_votes:
                            vh = ow[oo + m: oo + m + m * C].view(m, C)
                            vh.copy_(v, non_blocking=True)
                            v_host.append(vh)
                    ev = torch.cuda.Event()
                    ev.record(stream)
                self.launches += 1
                with self._slot_cv:
                    self._inflight.append((ev, slot, spans, c_host, v_host, (Xs, votes, classes)))
                    self._slot_cv.notify_all()
            except (FPError, RuntimeError) as e:
                for r in batch:
                    r.error = str(e)
                    r._done.set()
                with self._slot_cv:
                    self._free_slots.append(slot)
                    self._slot_cv.notify_all()

    def _completer(self) -> None:
        while True:
            with self._slot_cv:
                while not self._inflight:
                    if self._batcher_done:
                        return
                    self._slot_cv.wait(0.01)
                ev, slot, spans, c_host, v_host, keep = self._inflight[0]
            deadline = time.perf_counter() + 60.0
            while not ev.query():  # bounded poll of the launch's completion
                if time.perf_counter() > deadline:
                    for rs, _ in spans:
                        for r in rs:
                            r.error = "launch did not complete in 60 s"
                            r._done.set()
                    break
                time.sleep(20e-6)
            now = time.perf_counter()
            for gi, (rs, _) in enumerate(spans):
                cl = c_host[gi].numpy()
                vo = v_host[gi].numpy() if v_host is not None else None
                off = 0
                for r in rs:
                    m = r.X.shape[0]
                    if r.error is None:
                        r.classes = cl[off: off + m].copy()
                        if vo is not None:
                            r.votes = vo[off: off + m].copy()
                        r.t_done = now
                    off += m
                    self.completed.append(r)
                    r._done.set()
            with self._slot_cv:
                self._inflight.popleft()
                self._free_slots.append(slot)
                self._slot_cv.notify_all()
            del keep


def latency_summary(requests) -> dict:
    lat = np.array([r.latency_s for r in requests if r.latency_s is not None])
    if lat.size == 0:
        return {"n": 0}
    return {"n": int(lat.size), "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3)}
