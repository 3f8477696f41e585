"""Continuous-batching classification server over resident packed forests.

Forests stay resident on the device.  Requests (a few rows for one forest)
arrive from any thread and go to the library's serving runtime
(`fp_server_*` in include/forest_pack.h): its batcher thread groups whatever
has arrived into one persistent launch over all the forests involved
(fp_predict_batched), so requests of different sizes and forests share a
launch; up to `slots` launches are in flight, each on its own CUDA stream,
admitted once a slot and enough free device memory are available; its
completion thread copies each request's classes (and votes) back and wakes
the waiters.  Batching, admission, staging and completion all run in native
threads of the library; this module only keeps the request objects and their
buffers alive and exposes the results.
"""
from __future__ import annotations

import ctypes
import threading

import numpy as np

from . import _ERRNAMES, FP_ETIMEOUT, FP_OK, _check, fp_pack_forest, fp_upload, lib


class Request:
    """One classification request; wait() blocks until its result is ready."""

    __slots__ = ("forest", "X", "classes", "votes", "error", "_handle", "_status", "_latency", "__weakref__")

    def __init__(self, forest: str, X: np.ndarray, classes: np.ndarray, votes: np.ndarray | None, handle):
        self.forest = forest
        self.X = X              # kept alive until the request is answered
        self.classes = classes  # filled in by the library's completion thread
        self.votes = votes
        self.error = None
        self._handle = handle
        self._status = None
        self._latency = None

    def wait(self, timeout: float | None = None) -> bool:
        if self._status is not None:
            return True
        rc = lib().fp_request_wait(self._handle, -1.0 if timeout is None else float(timeout))
        if rc == FP_ETIMEOUT and lib().fp_request_latency(self._handle) < 0:
            return False  # not answered yet
        self._status = rc
        self._latency = lib().fp_request_latency(self._handle)
        if rc != FP_OK:  # the launch's message was recorded on a library thread; the code names the failure
            self.error = _ERRNAMES.get(rc, str(rc))
        return True

    @property
    def latency_s(self) -> float | None:
        if self._latency is None:
            t = lib().fp_request_latency(self._handle)
            return None if t < 0 else t
        return self._latency

    def _release(self) -> None:
        if self._handle is not None:
            lib().fp_request_release(self._handle)
            self._handle = None


class _Resident:
    def __init__(self, name, df, n_features, n_classes, fid):
        self.name = name
        self.df = df
        self.F = n_features
        self.C = n_classes
        self.id = fid


class ForestServer:
    """Serve classification requests for several resident forests.

    slots            launches in flight at most (one CUDA stream each)
    max_rows         rows per launch at most (a larger request is launched alone)
    mem_margin       device bytes kept free when admitting a launch
    return_votes     also return per-class vote counts
    max_wait_s       let a batch grow until its oldest request waited this long
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
        self.completed: list[Request] = []
        self._lock = threading.Lock()
        self._started = False
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(lib().fp_server_create(self.device.index, slots, max_rows, mem_margin, int(return_votes),
                                          float(max_wait_s), ctypes.byref(h)), "fp_server_create")
        self._h = h

    # ------------------------------------------------------------ forests
    def add_forest(self, name: str, forest, **pack_params) -> None:
        """Pack, upload and keep a forest resident under `name`."""
        with self.torch.cuda.device(self.device):
            df = fp_upload(fp_pack_forest(forest, **pack_params))
        self.add_device_forest(name, df, forest.n_features, forest.n_classes)

    def add_device_forest(self, name: str, df, n_features: int, n_classes: int) -> None:
        fid = ctypes.c_int32()
        _check(lib().fp_server_add_forest(self._h, df.handle, ctypes.byref(fid)), "fp_server_add_forest")
        self.forests[name] = _Resident(name, df, n_features, n_classes, fid.value)

    # ------------------------------------------------------------ requests
    def submit(self, forest: str, X: np.ndarray) -> Request:
        res = self.forests.get(forest)
        if res is None:
            raise KeyError(forest)
        X = np.ascontiguousarray(X, dtype=np.float32)
        if X.ndim != 2 or X.shape[1] != res.F:
            raise ValueError("rows must be [m][n_features] of the forest")
        m = X.shape[0]
        classes = np.empty(m, np.int32)
        votes = np.empty((m, res.C), np.uint32) if self.return_votes else None
        h = ctypes.c_void_p()
        _check(lib().fp_server_submit(self._h, res.id, X.ctypes.data, m, classes.ctypes.data,
                                      votes.ctypes.data if votes is not None else None, ctypes.byref(h)),
               "fp_server_submit")
        req = Request(forest, X, classes, votes, h)
        with self._lock:
            self.completed.append(req)  # kept (with its buffers) until the server stops
        return req

    def start(self) -> "ForestServer":
        _check(lib().fp_server_start(self._h), "fp_server_start")
        self._started = True
        return self

    def stop(self) -> None:
        """Answer every queued request, then stop the library's threads."""
        if self._h is not None and self._started:
            _check(lib().fp_server_stop(self._h), "fp_server_stop")
            for r in self.completed:
                r.wait()

    def close(self) -> None:
        """Stop, release the requests' handles and the server."""
        if self._h is None:
            return
        self.stop()
        for r in self.completed:
            r._release()
        lib().fp_server_release(self._h)
        self._h = None

    def __enter__(self):
        return self.start()

    def __exit__(self, *exc):
        self.stop()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ state
    def _stats(self):
        a, b = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().fp_server_stats(self._h, ctypes.byref(a), ctypes.byref(b)), "fp_server_stats")
        return a.value, b.value

    @property
    def launches(self) -> int:
        return self._stats()[0]

    @property
    def rejected_for_memory(self) -> int:
        return self._stats()[1]

    @property
    def slots_in_service(self) -> int:
        """Slots not retired (a slot whose launch outlived the completion
        poll's limit is never reused)."""
        v = ctypes.c_int32()
        _check(lib().fp_server_slots_in_service(self._h, ctypes.byref(v)), "fp_server_slots_in_service")
        return v.value

    def set_launch_timeout(self, seconds: float) -> None:
        """The completion poll's limit per launch (default 60 s)."""
        _check(lib().fp_server_set_launch_timeout(self._h, float(seconds)), "fp_server_set_launch_timeout")

    def set_free_bytes(self, free_bytes: int) -> None:
        """Tests: the free device memory the admission check sees (-1: the device's)."""
        _check(lib().fp_server_set_free_bytes(self._h, int(free_bytes)), "fp_server_set_free_bytes")


def latency_summary(requests) -> dict:
    lat = np.array([r.latency_s for r in requests if r.latency_s is not None])
    if lat.size == 0:
        return {"n": 0}
    return {"n": int(lat.size), "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3)}
