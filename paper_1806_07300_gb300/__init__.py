"""Python binding of the forest-packing C ABI (include/forest_pack.h).

Argument marshalling only: every step of classification runs in the CUDA
library ``libforestpack.so`` built in-tree for sm_103a.  There is no CPU
fallback; importing the binding fails loudly when the library is missing.
PyTorch supplies device memory and streams.

Names follow the C ABI: :func:`fp_pack_forest`, :func:`fp_upload`,
:func:`fp_predict`, :func:`fp_predict_leaves`, :func:`fp_predict_batched`,
:func:`fp_sync_status`, :func:`fp_release`, the plain baseline
:func:`fp_plain_build` / :func:`fp_plain_predict`, plus small wrapper classes.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

LIB_PATH = _build.LIB

FP_OK, FP_EINVAL, FP_ENOMEM, FP_ECUDA, FP_EUNSUPPORTED, FP_ETIMEOUT, FP_EDEVICE = 0, -1, -2, -3, -4, -5, -6
FP_PLAIN_OBS_FASTEST, FP_PLAIN_TREE_FASTEST = 0, 1
_ERRNAMES = {-1: "FP_EINVAL", -2: "FP_ENOMEM", -3: "FP_ECUDA", -4: "FP_EUNSUPPORTED", -5: "FP_ETIMEOUT",
             -6: "FP_EDEVICE"}


class FPError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


class fp_forest_desc(ctypes.Structure):
    _fields_ = [("n_trees", ctypes.c_int32), ("n_features", ctypes.c_int32), ("n_classes", ctypes.c_int32),
                ("tree_node_begin", ctypes.c_void_p), ("left", ctypes.c_void_p), ("right", ctypes.c_void_p),
                ("feature", ctypes.c_void_p), ("threshold", ctypes.c_void_p), ("leaf_class", ctypes.c_void_p),
                ("cardinality", ctypes.c_void_p), ("leaf_value", ctypes.c_void_p)]


class fp_pack_params(ctypes.Structure):
    _fields_ = [("bin_size", ctypes.c_int32), ("interleave_depth", ctypes.c_int32), ("obs_tile", ctypes.c_int32),
                ("warps_per_cta", ctypes.c_int32), ("pass_bytes", ctypes.c_int64), ("refill_lanes", ctypes.c_int32),
                ("head_select", ctypes.c_int32), ("bin_buffers", ctypes.c_int32), ("deep_levels", ctypes.c_int32),
                ("deep_format", ctypes.c_int32)]


class fp_packed_info(ctypes.Structure):
    _fields_ = [("n_trees", ctypes.c_int32), ("n_features", ctypes.c_int32), ("n_classes", ctypes.c_int32),
                ("bin_size", ctypes.c_int32), ("interleave_depth", ctypes.c_int32), ("n_bins", ctypes.c_int32),
                ("obs_tile", ctypes.c_int32), ("warps_per_cta", ctypes.c_int32),
                ("n_internal", ctypes.c_int64), ("n_super", ctypes.c_int64), ("head_bytes", ctypes.c_int64),
                ("deep_bytes", ctypes.c_int64),
                ("total_bytes", ctypes.c_int64), ("parity_bytes", ctypes.c_int64),
                ("max_head_bytes", ctypes.c_int32), ("passes", ctypes.c_int32), ("refill_lanes", ctypes.c_int32),
                ("head_nodes", ctypes.c_int32), ("head_select", ctypes.c_int32), ("bin_buffers", ctypes.c_int32),
                ("deep_levels", ctypes.c_int32), ("deep_format", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class fp_batch(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("n", ctypes.c_int64), ("out_votes", ctypes.c_void_p),
                ("out_class", ctypes.c_void_p)]


# every symbol include/forest_pack.h declares
EXPORTS = ["fp_pack_forest", "fp_packed_info_get", "fp_packed_image", "fp_upload", "fp_predict",
           "fp_predict_leaves", "fp_predict_batched", "fp_configure", "fp_predict_noalloc", "fp_sync_status", "fp_device_info_get", "fp_release_packed",
           "fp_release", "fp_last_error", "fp_plain_build", "fp_plain_predict", "fp_plain_bytes",
           "fp_plain_release", "fp_l2_read_probe", "fp_count_leaves", "fp_inject_fault", "fp_predict_values",
           "fp_plain_predict_values", "fp_predict_host", "fp_predict_values_host", "fp_server_create",
           "fp_server_add_forest", "fp_server_start", "fp_server_submit", "fp_request_wait", "fp_request_latency",
           "fp_request_release", "fp_server_stop", "fp_server_stats", "fp_server_set_free_bytes",
           "fp_server_release", "fp_cardinality_from_leaf_counts", "fp_infer_cardinality",
           "fp_server_set_launch_timeout", "fp_server_slots_in_service", "fp_shard_trees", "fp_pack_forest_trees",
           "fp_votes_argmax"]

_lib = None
_lock = threading.Lock()


def build(force: bool = False, verbose: bool = False) -> str:
    return _build.build(force=force, verbose=verbose)


def lib() -> ctypes.CDLL:
    """Load libforestpack.so (building it first if its sources are newer)."""
    global _lib
    with _lock:
        if _lib is None:
            if not _build.up_to_date():
                _build.build()
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"CUDA library {LIB_PATH} is missing; run __graft_entry__.build()")
            L = ctypes.CDLL(LIB_PATH)
            P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
            sig = {
                "fp_pack_forest": ([ctypes.POINTER(fp_forest_desc), ctypes.POINTER(fp_pack_params),
                                    ctypes.POINTER(P)], ctypes.c_int),
                "fp_packed_info_get": ([P, ctypes.POINTER(fp_packed_info)], ctypes.c_int),
                "fp_packed_image": ([P, ctypes.POINTER(i64)], P),
                "fp_upload": ([P, P, ctypes.POINTER(P)], ctypes.c_int),
                "fp_predict": ([P, P, i64, P, P, P], ctypes.c_int),
                "fp_configure": ([P, ctypes.POINTER(fp_pack_params)], ctypes.c_int),
                "fp_predict_noalloc": ([P, P, i64, P, P, P], ctypes.c_int),
                "fp_predict_leaves": ([P, P, i64, P, P], ctypes.c_int),
                "fp_predict_batched": ([P, P, i32, P], ctypes.c_int),
                "fp_sync_status": ([P, P], ctypes.c_int),
                "fp_device_info_get": ([P, ctypes.POINTER(fp_packed_info)], ctypes.c_int),
                "fp_release_packed": ([P], None),
                "fp_release": ([P], None),
                "fp_last_error": ([], ctypes.c_char_p),
                "fp_plain_build": ([ctypes.POINTER(fp_forest_desc), P, ctypes.POINTER(P)], ctypes.c_int),
                "fp_plain_predict": ([P, P, i64, i32, P, P, P], ctypes.c_int),
                "fp_plain_bytes": ([P], i64),
                "fp_plain_release": ([P], None),
                "fp_l2_read_probe": ([P, i64, ctypes.c_int32, P, ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
                "fp_count_leaves": ([P, i64, i32, P, P, P, P], ctypes.c_int),
                "fp_inject_fault": ([P, i32, i64], ctypes.c_int),
                "fp_predict_values": ([P, P, i64, ctypes.c_float, ctypes.c_float, P, P], ctypes.c_int),
                "fp_plain_predict_values": ([P, P, i64, i32, ctypes.c_float, ctypes.c_float, P, P], ctypes.c_int),
                "fp_predict_host": ([P, P, i64, P, P, i64, P], ctypes.c_int),
                "fp_predict_values_host": ([P, P, i64, ctypes.c_float, ctypes.c_float, P, i64, P], ctypes.c_int),
                "fp_server_create": ([i32, i32, i64, i64, i32, ctypes.c_double, ctypes.POINTER(P)], ctypes.c_int),
                "fp_server_add_forest": ([P, P, ctypes.POINTER(i32)], ctypes.c_int),
                "fp_server_start": ([P], ctypes.c_int),
                "fp_server_submit": ([P, i32, P, i64, P, P, ctypes.POINTER(P)], ctypes.c_int),
                "fp_request_wait": ([P, ctypes.c_double], ctypes.c_int),
                "fp_request_latency": ([P], ctypes.c_double),
                "fp_request_release": ([P], None),
                "fp_server_stop": ([P], ctypes.c_int),
                "fp_server_stats": ([P, ctypes.POINTER(i64), ctypes.POINTER(i64)], ctypes.c_int),
                "fp_server_set_free_bytes": ([P, i64], ctypes.c_int),
                "fp_server_release": ([P], None),
                "fp_server_set_launch_timeout": ([P, ctypes.c_double], ctypes.c_int),
                "fp_shard_trees": ([ctypes.POINTER(fp_forest_desc), i32, i32, i32, ctypes.POINTER(i32),
                                    ctypes.POINTER(i32)], ctypes.c_int),
                "fp_pack_forest_trees": ([ctypes.POINTER(fp_forest_desc), ctypes.POINTER(fp_pack_params), i32, i32,
                                          ctypes.POINTER(P)], ctypes.c_int),
                "fp_votes_argmax": ([P, i64, i32, P, P], ctypes.c_int),
                "fp_server_slots_in_service": ([P, ctypes.POINTER(i32)], ctypes.c_int),
                "fp_cardinality_from_leaf_counts": ([ctypes.POINTER(fp_forest_desc), P, P], ctypes.c_int),
                "fp_infer_cardinality": ([P, ctypes.POINTER(fp_forest_desc), P, i64, i64, P, P], ctypes.c_int),
            }
            for name, (args, res) in sig.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
    return _lib


def fp_last_error() -> str:
    return lib().fp_last_error().decode()


def _check(rc: int, what: str) -> None:
    if rc != FP_OK:
        msg = fp_last_error()
        raise FPError(rc, msg if msg.startswith(what) else f"{what}: {msg}")


# ----------------------------------------------------------------- helpers

def _np(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def make_desc(forest, keep: list) -> fp_forest_desc:
    """fp_forest_desc over a forest object with the datagen.Forest fields.
    ``keep`` collects the arrays that must outlive the descriptor."""
    arrs = [_np(forest.node_begin, np.int64), _np(forest.left, np.int32), _np(forest.right, np.int32),
            _np(forest.feature, np.int32), _np(forest.threshold, np.float32), _np(forest.leaf_class, np.int32)]
    card = getattr(forest, "cardinality", None)
    arrs.append(_np(card, np.int64) if card is not None else None)
    keep.extend(a for a in arrs if a is not None)
    d = fp_forest_desc()
    d.n_trees = int(forest.n_trees)
    d.n_features = int(forest.n_features)
    d.n_classes = int(forest.n_classes)
    (d.tree_node_begin, d.left, d.right, d.feature, d.threshold, d.leaf_class) = [a.ctypes.data for a in arrs[:6]]
    d.cardinality = arrs[6].ctypes.data if arrs[6] is not None else None
    lv = getattr(forest, "leaf_value", None)
    if lv is not None:
        lv = _np(lv, np.float32)
        keep.append(lv)
        d.leaf_value = lv.ctypes.data
    return d


def _stream_ptr(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dptr(t, dtype, shape=None, name="tensor"):
    """Device pointer of a CUDA tensor after checking dtype, contiguity and shape."""
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return t.data_ptr()


def _hptr(t, dtype, shape=None, name="array"):
    """Host pointer of a CPU torch tensor or numpy array after checking dtype,
    contiguity and shape."""
    if t is None:
        return None
    import numpy as np
    import torch
    if isinstance(t, torch.Tensor):
        if t.is_cuda:
            raise TypeError(f"{name} must be in host memory")
        if t.dtype != dtype:
            raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
        ok, ptr = t.is_contiguous(), t.data_ptr()
    elif isinstance(t, np.ndarray):
        want = {torch.float32: np.float32, torch.int32: np.int32}[dtype]
        if t.dtype != want:
            raise TypeError(f"{name} must be {np.dtype(want)}, got {t.dtype}")
        ok, ptr = t.flags["C_CONTIGUOUS"], t.ctypes.data
    else:
        raise TypeError(f"{name} must be a CPU tensor or a numpy array")
    if not ok:
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return ptr


# ------------------------------------------------------------ C-ABI mirrors

def fp_pack_forest(forest, bin_size: int = 0, interleave_depth: int = -1, obs_tile: int = 0,
                   warps_per_cta: int = 0, pass_bytes: int = 0, refill_lanes: int = 0,
                   head_select: int = 0, bin_buffers: int = 0, deep_levels: int = 0,
                   deep_format: int = 0) -> "PackedForest":
    keep: list = []
    desc = make_desc(forest, keep)
    params = fp_pack_params(bin_size, interleave_depth, obs_tile, warps_per_cta, pass_bytes, refill_lanes,
                            head_select, bin_buffers, deep_levels, deep_format)
    out = ctypes.c_void_p()
    _check(lib().fp_pack_forest(ctypes.byref(desc), ctypes.byref(params), ctypes.byref(out)), "fp_pack_forest")
    return PackedForest(out.value, forest)


def fp_shard_trees(forest, bin_size: int, n_shards: int, shard: int) -> tuple[int, int]:
    """Trees [begin, end) of one shard of a tree-bin split (whole bins,
    balanced by expected visits)."""
    keep: list = []
    desc = make_desc(forest, keep)
    b, e = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().fp_shard_trees(ctypes.byref(desc), bin_size, n_shards, shard, ctypes.byref(b), ctypes.byref(e)),
           "fp_shard_trees")
    return b.value, e.value


def fp_pack_forest_trees(forest, tree_begin: int, tree_end: int, bin_size: int = 0, interleave_depth: int = -1,
                         obs_tile: int = 0, warps_per_cta: int = 0, pass_bytes: int = 0, refill_lanes: int = 0,
                         head_select: int = 0, bin_buffers: int = 0, deep_levels: int = 0,
                         deep_format: int = 0) -> "PackedForest":
    """fp_pack_forest over the trees [tree_begin, tree_end) of `forest`."""
    keep: list = []
    desc = make_desc(forest, keep)
    params = fp_pack_params(bin_size, interleave_depth, obs_tile, warps_per_cta, pass_bytes, refill_lanes,
                            head_select, bin_buffers, deep_levels, deep_format)
    out = ctypes.c_void_p()
    _check(lib().fp_pack_forest_trees(ctypes.byref(desc), ctypes.byref(params), tree_begin, tree_end,
                                      ctypes.byref(out)), "fp_pack_forest_trees")
    return PackedForest(out.value, None)


def fp_votes_argmax(votes, out_class, stream=None) -> None:
    """out_class[i] = the lowest class with the most votes[i] (device tensors)."""
    T = _torch()
    n, C = votes.shape
    vp = _dptr(votes, T.int32, None, "votes")
    cp = _dptr(out_class, T.int32, (n,), "out_class")
    _check(lib().fp_votes_argmax(vp, n, C, cp, _stream_ptr(stream)), "fp_votes_argmax")


def fp_upload(packed: "PackedForest", stream=None) -> "DeviceForest":
    out = ctypes.c_void_p()
    _check(lib().fp_upload(packed.handle, _stream_ptr(stream), ctypes.byref(out)), "fp_upload")
    df = DeviceForest(out.value, packed.info())
    src = packed.forest
    if src is not None and getattr(src, "leaf_value", None) is not None:
        df.value_scale, df.value_bias = src.value_scale, src.value_bias
    return df


def fp_predict(forest: "DeviceForest", X, out_votes=None, out_class=None, stream=None) -> None:
    n = X.shape[0]
    info = forest.info
    xp = _dptr(X, _torch().float32, (n, info["n_features"]), "X")
    vp = _dptr(out_votes, _torch().int32, (n, info["n_classes"]), "out_votes") if out_votes is not None else None
    cp = _dptr(out_class, _torch().int32, (n,), "out_class") if out_class is not None else None
    _check(lib().fp_predict(forest.handle, xp, n, vp, cp, _stream_ptr(stream)), "fp_predict")


def fp_predict_values(forest: "DeviceForest", X, out, scale: float, bias: float, stream=None) -> None:
    """Forests with leaf values: out[i] = bias + scale * sum of leaf values."""
    n = X.shape[0]
    xp = _dptr(X, _torch().float32, (n, forest.info["n_features"]), "X")
    op = _dptr(out, _torch().float32, (n,), "out")
    _check(lib().fp_predict_values(forest.handle, xp, n, scale, bias, op, _stream_ptr(stream)), "fp_predict_values")


def fp_predict_host(forest: "DeviceForest", X_host, out_votes_host=None, out_class_host=None, chunk_rows: int = 0,
                    stream=None) -> None:
    """fp_predict for rows and results in host memory (pinned for overlap);
    the results are there once `stream` completes."""
    n = X_host.shape[0]
    info = forest.info
    xp = _hptr(X_host, _torch().float32, (n, info["n_features"]), "X_host")
    vp = _hptr(out_votes_host, _torch().int32, (n, info["n_classes"]), "out_votes_host")
    cp = _hptr(out_class_host, _torch().int32, (n,), "out_class_host")
    _check(lib().fp_predict_host(forest.handle, xp, n, vp, cp, chunk_rows, _stream_ptr(stream)), "fp_predict_host")


def fp_predict_values_host(forest: "DeviceForest", X_host, out_host, scale: float, bias: float, chunk_rows: int = 0,
                           stream=None) -> None:
    """fp_predict_values for rows and results in host memory."""
    n = X_host.shape[0]
    xp = _hptr(X_host, _torch().float32, (n, forest.info["n_features"]), "X_host")
    op = _hptr(out_host, _torch().float32, (n,), "out_host")
    _check(lib().fp_predict_values_host(forest.handle, xp, n, scale, bias, op, chunk_rows, _stream_ptr(stream)),
           "fp_predict_values_host")


def fp_predict_noalloc(forest: "DeviceForest", X, out_votes=None, out_class=None, stream=None) -> None:
    """fp_predict that allocates no device memory (scratch from a fixed
    16 MiB array inside the library; see include/forest_pack.h)."""
    n = X.shape[0]
    info = forest.info
    xp = _dptr(X, _torch().float32, (n, info["n_features"]), "X")
    vp = _dptr(out_votes, _torch().int32, (n, info["n_classes"]), "out_votes") if out_votes is not None else None
    cp = _dptr(out_class, _torch().int32, (n,), "out_class") if out_class is not None else None
    _check(lib().fp_predict_noalloc(forest.handle, xp, n, vp, cp, _stream_ptr(stream)), "fp_predict_noalloc")


def fp_predict_leaves(forest: "DeviceForest", X, out_leaf, stream=None) -> None:
    n = X.shape[0]
    info = forest.info
    xp = _dptr(X, _torch().float32, (n, info["n_features"]), "X")
    lp = _dptr(out_leaf, _torch().int32, (n, info["n_trees"]), "out_leaf")
    _check(lib().fp_predict_leaves(forest.handle, xp, n, lp, _stream_ptr(stream)), "fp_predict_leaves")


def fp_predict_batched(forests, Xs, out_votes=None, out_class=None, stream=None) -> None:
    k = len(forests)
    arr = (fp_batch * max(k, 1))()
    handles = (ctypes.c_void_p * max(k, 1))()
    T = _torch()
    for i, (f, X) in enumerate(zip(forests, Xs)):
        n = X.shape[0]
        arr[i].X = _dptr(X, T.float32, (n, f.info["n_features"]), "X")
        arr[i].n = n
        v = out_votes[i] if out_votes is not None else None
        c = out_class[i] if out_class is not None else None
        arr[i].out_votes = _dptr(v, T.int32, (n, f.info["n_classes"]), "out_votes") if v is not None else None
        arr[i].out_class = _dptr(c, T.int32, (n,), "out_class") if c is not None else None
        handles[i] = f.handle
    _check(lib().fp_predict_batched(handles, arr, k, _stream_ptr(stream)), "fp_predict_batched")


def fp_sync_status(forest: "DeviceForest", stream=None) -> int:
    return lib().fp_sync_status(forest.handle, _stream_ptr(stream))


FP_FAULT_ALLOC, FP_FAULT_WAIT_LIMIT, FP_FAULT_STALL_BIN_COPY = 1, 2, 3


def fp_inject_fault(forest, kind: int, value: int) -> None:
    """Fault injection for failure-detection tests: FP_FAULT_ALLOC (forest may
    be None) makes the next `value` device allocations fail with FP_ENOMEM;
    FP_FAULT_WAIT_LIMIT bounds a bin-block wait to `value` polls;
    FP_FAULT_STALL_BIN_COPY=1 makes the forest's bin waits run out, so its
    launches record FP_ETIMEOUT (0 restores)."""
    handle = forest.handle if forest is not None else None
    _check(lib().fp_inject_fault(handle, kind, value), "fp_inject_fault")


def fp_release(forest: "DeviceForest") -> None:
    forest.release()


def _torch():
    import torch
    return torch


class PackedForest:
    """Host image made by fp_pack_forest (library-owned)."""

    def __init__(self, handle: int, forest=None):
        self.handle = handle
        self.forest = forest

    def info(self) -> dict:
        i = fp_packed_info()
        _check(lib().fp_packed_info_get(self.handle, ctypes.byref(i)), "fp_packed_info_get")
        return i.as_dict()

    def image(self) -> np.ndarray:
        """A copy of the packed image bytes."""
        nbytes = ctypes.c_int64()
        p = lib().fp_packed_image(self.handle, ctypes.byref(nbytes))
        if not p:
            raise FPError(FP_EINVAL, fp_last_error())
        return np.frombuffer((ctypes.c_uint8 * nbytes.value).from_address(p), dtype=np.uint8).copy()

    def release(self) -> None:
        if self.handle:
            lib().fp_release_packed(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


class DeviceForest:
    """A packed forest resident on the current device (fp_upload)."""

    value_scale = None  # forests with leaf values: the scale and bias of their output
    value_bias = None

    def __init__(self, handle: int, info: dict):
        self.handle = handle
        i = fp_packed_info()
        _check(lib().fp_device_info_get(handle, ctypes.byref(i)), "fp_device_info_get")
        self.info = i.as_dict()

    def configure(self, obs_tile: int = 0, warps_per_cta: int = 0, refill_lanes: int = 0,
                  bin_buffers: int = 0) -> None:
        """Change launch parameters (fp_configure); layout stays as packed."""
        params = fp_pack_params(0, -1, obs_tile, warps_per_cta, 0, refill_lanes, 0, bin_buffers, 0)
        _check(lib().fp_configure(self.handle, ctypes.byref(params)), "fp_configure")
        i = fp_packed_info()
        _check(lib().fp_device_info_get(self.handle, ctypes.byref(i)), "fp_device_info_get")
        self.info = i.as_dict()

    def predict(self, X, votes: bool = True, classes: bool = True, stream=None):
        T = _torch()
        n = X.shape[0]
        v = T.empty((n, self.info["n_classes"]), dtype=T.int32, device=X.device) if votes else None
        c = T.empty((n,), dtype=T.int32, device=X.device) if classes else None
        fp_predict(self, X, v, c, stream)
        return v, c

    def predict_values(self, X, scale: float | None = None, bias: float | None = None, stream=None):
        """bias + scale * the sum of leaf values per row (a float32 tensor);
        scale and bias default to those of the forest that was packed."""
        T = _torch()
        out = T.empty((X.shape[0],), dtype=T.float32, device=X.device)
        fp_predict_values(self, X, out, self.value_scale if scale is None else scale,
                          self.value_bias if bias is None else bias, stream)
        return out

    def predict_host(self, X_host, votes: bool = False, classes: bool = True, chunk_rows: int = 0, stream=None):
        """Rows in host memory (a CPU tensor or numpy array; pinned tensors
        let copies overlap the kernels) to host results: (votes, classes) as
        pinned int32 tensors, or for a forest with leaf values the float32
        outputs; waits for the stream."""
        T = _torch()
        n = X_host.shape[0]
        s = stream if stream is not None else T.cuda.current_stream()
        if self.value_scale is not None:  # a forest with leaf values
            out = T.empty((n,), dtype=T.float32).pin_memory()
            fp_predict_values_host(self, X_host, out, self.value_scale, self.value_bias, chunk_rows, s)
            s.synchronize()
            return out
        v = T.empty((n, self.info["n_classes"]), dtype=T.int32).pin_memory() if votes else None
        c = T.empty((n,), dtype=T.int32).pin_memory() if classes else None
        fp_predict_host(self, X_host, v, c, chunk_rows, s)
        s.synchronize()
        return v, c

    def predict_leaves(self, X, stream=None):
        T = _torch()
        out = T.empty((X.shape[0], self.info["n_trees"]), dtype=T.int32, device=X.device)
        fp_predict_leaves(self, X, out, stream)
        return out

    def sync_status(self, stream=None) -> int:
        return fp_sync_status(self, stream)

    def release(self) -> None:
        if self.handle:
            lib().fp_release(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


class PlainForest:
    """The plain breadth-first baseline resident on the current device."""

    def __init__(self, forest, stream=None):
        keep: list = []
        desc = make_desc(forest, keep)
        out = ctypes.c_void_p()
        _check(lib().fp_plain_build(ctypes.byref(desc), _stream_ptr(stream), ctypes.byref(out)), "fp_plain_build")
        self.handle = out.value
        self.n_trees, self.n_features, self.n_classes = forest.n_trees, forest.n_features, forest.n_classes
        self.value_scale = getattr(forest, "value_scale", 1.0)
        self.value_bias = getattr(forest, "value_bias", 0.0)

    def nbytes(self) -> int:
        return lib().fp_plain_bytes(self.handle)

    def predict(self, X, order: int = FP_PLAIN_OBS_FASTEST, out_votes=None, out_class=None, stream=None):
        T = _torch()
        n = X.shape[0]
        if out_votes is None:
            out_votes = T.empty((n, self.n_classes), dtype=T.int32, device=X.device)
        if out_class is None:
            out_class = T.empty((n,), dtype=T.int32, device=X.device)
        fp_plain_predict(self, X, order, out_votes, out_class, stream)
        return out_votes, out_class

    def predict_values(self, X, order: int = FP_PLAIN_OBS_FASTEST, out=None, stream=None):
        T = _torch()
        if out is None:
            out = T.empty((X.shape[0],), dtype=T.float32, device=X.device)
        fp_plain_predict_values(self, X, order, out, self.value_scale, self.value_bias, stream)
        return out

    def release(self) -> None:
        if self.handle:
            lib().fp_plain_release(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


def fp_l2_read_probe(nbytes: int = 64 << 20, iters: int = 50, stream=None) -> float:
    """L2 read bandwidth in GB/s over an L2-resident buffer (fp_l2_read_probe)."""
    T = _torch()
    buf = T.zeros(nbytes // 4, dtype=T.int32, device="cuda")
    ms = ctypes.c_float(0.0)
    _check(lib().fp_l2_read_probe(buf.data_ptr(), buf.numel() * 4, iters, _stream_ptr(stream), ctypes.byref(ms)),
           "fp_l2_read_probe")
    return buf.numel() * 4 * iters / (ms.value / 1e3) / 1e9


def fp_count_leaves(out_leaf, node_begin, leaf_count, status, stream=None) -> None:
    """Add the leaves reached in out_leaf ([n][T] int32, device) to leaf_count
    (int64 per node, device); node_begin is the forest's [T+1] offsets (device)."""
    T = _torch()
    n, nt = out_leaf.shape
    lp = _dptr(out_leaf, T.int32, None, "out_leaf")
    nb = _dptr(node_begin, T.int64, (nt + 1,), "node_begin")
    cp = _dptr(leaf_count, T.int64, None, "leaf_count")
    sp = _dptr(status, T.int32, None, "status")
    _check(lib().fp_count_leaves(lp, n, nt, nb, cp, sp, _stream_ptr(stream)), "fp_count_leaves")


def fp_cardinality_from_leaf_counts(forest, leaf_count) -> np.ndarray:
    """Node cardinalities from per-node leaf counts (host int64, one per node
    of `forest`): the library sums each internal node from its children."""
    keep = []
    desc = make_desc(forest, keep)
    cnt = _np(leaf_count, np.int64)
    if cnt.shape != (forest.n_nodes,):
        raise ValueError("leaf_count must hold one int64 per node")
    out = np.empty(forest.n_nodes, np.int64)
    _check(lib().fp_cardinality_from_leaf_counts(ctypes.byref(desc), cnt.ctypes.data, out.ctypes.data),
           "fp_cardinality_from_leaf_counts")
    return out


def infer_cardinality(forest, X, device_forest=None, stream=None, chunk_rows: int = 0):
    """Cardinalities of every node of `forest` counted from the observations
    X (CUDA float32 [n][n_features]) by fp_infer_cardinality: leaves reached
    on the device, counted per node, each internal node the sum of its
    children.  Returns an int64 numpy array aligned with the node arrays."""
    T = _torch()
    df = device_forest or fp_upload(fp_pack_forest(forest), stream)
    n = X.shape[0]
    xp = _dptr(X, T.float32, (n, forest.n_features), "X")
    keep = []
    desc = make_desc(forest, keep)
    out = np.empty(forest.n_nodes, np.int64)
    _check(lib().fp_infer_cardinality(df.handle, ctypes.byref(desc), xp, n, chunk_rows, out.ctypes.data,
                                      _stream_ptr(stream)), "fp_infer_cardinality")
    return out


def fp_plain_build(forest, stream=None) -> PlainForest:
    return PlainForest(forest, stream)


def fp_plain_predict_values(pf: PlainForest, X, order, out, scale: float, bias: float, stream=None) -> None:
    T = _torch()
    n = X.shape[0]
    xp = _dptr(X, T.float32, (n, pf.n_features), "X")
    op = _dptr(out, T.float32, (n,), "out")
    _check(lib().fp_plain_predict_values(pf.handle, xp, n, order, scale, bias, op, _stream_ptr(stream)),
           "fp_plain_predict_values")


def fp_plain_predict(pf: PlainForest, X, order, out_votes, out_class=None, stream=None) -> None:
    T = _torch()
    n = X.shape[0]
    xp = _dptr(X, T.float32, (n, pf.n_features), "X")
    vp = _dptr(out_votes, T.int32, (n, pf.n_classes), "out_votes")
    cp = _dptr(out_class, T.int32, (n,), "out_class") if out_class is not None else None
    _check(lib().fp_plain_predict(pf.handle, xp, n, order, vp, cp, _stream_ptr(stream)), "fp_plain_predict")
