"""Host-side reader of the library's packed image (format in
paper_1806_07300_gb300/csrc/fp_internal.h), written independently of the CUDA
kernel: it lets CPU tests check the packer's records without a GPU."""
from __future__ import annotations

import numpy as np

HDR = np.dtype([("magic", "<u4"), ("version", "<u4"), ("n_trees", "<i4"), ("n_features", "<i4"),
                ("n_classes", "<i4"), ("bin_size", "<i4"), ("depth", "<i4"), ("n_bins", "<i4"),
                ("n_passes", "<i4"), ("head_nodes", "<i4"), ("head_select", "<i4"), ("obs_tile", "<i4"),
                ("warps_per_cta", "<i4"), ("max_head_bytes", "<i4"), ("refill_lanes", "<i4"), ("bin_buffers", "<i4"), ("n_super", "<i8"),
                ("off_bins", "<i8"), ("off_passes", "<i8"), ("off_tree_base", "<i8"), ("off_heads", "<i8"),
                ("off_deep", "<i8"), ("off_pheads", "<i8"), ("off_deep_leaf", "<i8"), ("class_bytes", "<i8"),
                ("total_bytes", "<i8"), ("head_bytes_total", "<i8"), ("pass_bytes", "<i8"), ("n_internal", "<i8"),
                ("n_values", "<i8"), ("off_values", "<i8"), ("deep_levels", "<i4"), ("feature_bits", "<i4"),
                ("class_bits", "<i4"), ("deep_format", "<i4"), ("off_deep_keys", "<i8"), ("values3_base", "<i8"),
                ("key_lo", "<u4"), ("key_hi", "<u4"), ("key_shl", "<u4"), ("key_flag", "<u4"),
                ("key_gap_a", "<u4"), ("key_gap_b", "<u4"), ("key_gap_d", "<u4"), ("reserved1", "<u4")],
               align=True)
BIN = np.dtype([("head_off", "<u4"), ("head_bytes", "<u4"), ("first_tree", "<i4"), ("width", "<i4"),
                ("phead_off", "<u4"), ("stride", "<i4"), ("nranks", "<i4"), ("nexits", "<i4")])
PASS = np.dtype([("bin_begin", "<i4"), ("bin_end", "<i4")])

LEAF = 0x80000000


def obs_key(x) -> np.ndarray:
    """Order keys of observation values: unsigned compares of keys order like
    the floats (-0 as +0; NaN above everything)."""
    a = np.asarray(x, dtype=np.float32)
    u = np.ascontiguousarray(a).reshape(-1).view(np.uint32).copy()
    nan = (u & 0x7FFFFFFF) > 0x7F800000
    u[u == 0x80000000] = 0
    k = np.where(u >> 31 == 1, ~u, u | np.uint32(0x80000000)).astype(np.uint32)
    k[nan] = 0xFFFFFFFF
    return k.reshape(a.shape)


def thr_key(t) -> np.ndarray:
    """Order keys of thresholds: as obs_key, but a NaN threshold gets 0 (every
    observation goes right of it, as x <= NaN never holds)."""
    k = np.array(obs_key(t))
    k[np.isnan(np.asarray(t, dtype=np.float32))] = 0
    return k


def _popc8(v: np.ndarray) -> np.ndarray:
    v = v.astype(np.int64)
    return sum((v >> i) & 1 for i in range(8))


class Image:
    def __init__(self, img: np.ndarray):
        self.img = img
        h = np.frombuffer(img[:HDR.itemsize].tobytes(), HDR)[0]
        self.h = {k: int(h[k]) for k in HDR.names}
        g = self.h
        self.bins = np.frombuffer(img[g["off_bins"]: g["off_bins"] + BIN.itemsize * g["n_bins"]].tobytes(), BIN)
        self.passes = np.frombuffer(img[g["off_passes"]: g["off_passes"] + 8 * g["n_passes"]].tobytes(), PASS)
        self.tree_base = img[g["off_tree_base"]: g["off_tree_base"] + 4 * g["n_trees"]].view("<u4")
        deep = img[g["off_deep"]: g["off_deep"] + 32 * g["n_super"]]
        self.sw = deep.view("<u4").reshape(-1, 8)          # super-node words
        self.sthr = deep.view("<f4").reshape(-1, 8)[:, :3]  # two levels: thresholds of v, left, right
        # thresholds are order keys with three-level super-nodes (remapped
        # ones in format 2), else floats
        self.keys = g["deep_levels"] == 3
        self.fmt = g["deep_format"] if self.keys else 0
        ne = 8 if g["deep_levels"] == 3 else 4
        dl = img[g["off_deep_leaf"]: g["off_deep_leaf"] + 4 * ne * g["n_super"]].view("<i4")
        self.deep_leaf = dl.reshape(-1, ne)
        if g["deep_levels"] == 3:
            nk = 8 if self.fmt == 2 else 4
            dk = img[g["off_deep_keys"]: g["off_deep_keys"] + 4 * nk * g["n_super"]].view("<u4")
            self.deep_keys = dk.reshape(-1, nk)  # full keys of slots 3..6 (format 1) or 0..6 (format 2)
        self.ties = 0  # three levels: compares decided by the full keys in the last walk
        # forests with leaf values: a leaf reference names a slot of this table
        self.values = img[g["off_values"]: g["off_values"] + 4 * g["n_values"]].view("<f4")

    def head(self, b: int):
        """(threshold keys [nranks][stride], meta [nranks][stride], exits
        [nexits][stride], exit leaf ids [nexits][stride]) of bin b's
        interleaved block; for paired level heads thr is [nranks][stride][3]
        (node, left and right child) and meta [nranks][stride] the packed
        features."""
        g, bn = self.h, self.bins[b]
        st, nr, ne = int(bn["stride"]), int(bn["nranks"]), int(bn["nexits"])
        base = g["off_heads"] + int(bn["head_off"])
        rec = 16 if g["head_select"] == 2 else 8
        recs = self.img[base: base + rec * nr * st]
        if rec == 16:
            thr = recs.view("<u4").reshape(nr, st, 4)[:, :, :3]
            meta = recs.view("<u4").reshape(nr, st, 4)[:, :, 3]
        else:
            thr = recs.view("<u4")[0::2].reshape(nr, st)
            meta = recs.view("<u4")[1::2].reshape(nr, st)
        exits = self.img[base + rec * nr * st: base + rec * nr * st + 4 * ne * st].view("<u4").reshape(ne, st)
        pb = g["off_pheads"] + int(bn["phead_off"])
        par = self.img[pb: pb + 4 * ne * st].view("<i4").reshape(ne, st)
        return thr, meta, exits, par

    def remap(self, k) -> np.ndarray:
        """The format-2 map V of order keys: the run of keys from key_gap_a
        to key_gap_b collapsed onto key_gap_a (keys from key_gap_b up move
        down by key_gap_d), then clamped to [key_lo, key_hi] and shifted up
        by key_shl below key_flag."""
        g = self.h
        k = np.asarray(k, np.int64)
        k = np.where(k >= g["key_gap_b"], k - g["key_gap_d"], np.minimum(k, g["key_gap_a"]))
        c = np.clip(k, g["key_lo"], g["key_hi"]) - g["key_lo"]
        return ((c << g["key_shl"]) | g["key_flag"]).astype(np.int64) & 0xFFFFFFFF

    def word(self, t) -> np.ndarray:
        """A threshold as the image stores it: its key (remapped in format 2;
        a NaN threshold stays 0), or its float bits."""
        if not self.keys:
            return np.array(t, dtype=np.float32).view(np.uint32)
        k = thr_key(t)
        if self.fmt == 2:
            k = np.where(k == 0, 0, self.remap(k)).astype(np.uint32)
        return k

    def walk(self, X: np.ndarray):
        """Leaf id and class (or value slot) per (observation, tree), decoding
        the records; X holds float observations, compared through their keys
        when the image stores keys."""
        g = self.h
        if self.keys:
            X = obs_key(X).astype(np.int64)
            if self.fmt == 2:
                X = self.remap(X)
        else:
            X = np.asarray(X, dtype=np.float32)
        self.ties = 0
        n, T = X.shape[0], g["n_trees"]
        leaf = np.full((n, T), -2, np.int32)
        cls = np.full((n, T), -2, np.int32)
        rows = np.arange(n)
        for b in range(g["n_bins"]):
            thr, meta, exits, par = self.head(b)
            if not self.keys:
                thr = thr.view(np.float32)
            bn = self.bins[b]
            for k in range(int(bn["width"])):
                t = int(bn["first_tree"]) + k
                nr = int(bn["nranks"])
                hr = np.zeros(n, np.int64)
                if g["head_select"] == 1:  # implicit slots: children 2s+1 and 2s+2, d+1 steps
                    assert nr == 2 ** (g["depth"] + 1) - 1
                    for _ in range(g["depth"] + 1):
                        m = meta[hr, k].astype(np.int64)
                        right = ~(X[rows, m >> 22] <= thr[hr, k])
                        hr = 2 * hr + 1 + right
                elif g["head_select"] == 2:  # paired records: successors 4q+1 .. 4q+4
                    assert nr == (4 ** ((g["depth"] + 1) // 2) - 1) // 3
                    for _ in range((g["depth"] + 1) // 2):
                        m = meta[hr, k].astype(np.int64)
                        th = thr[hr, k]
                        d0 = ~(X[rows, m & 1023] <= th[:, 0])
                        f1 = np.where(d0, (m >> 20) & 1023, (m >> 10) & 1023)
                        d1 = ~(X[rows, f1] <= np.where(d0, th[:, 2], th[:, 1]))
                        hr = 4 * hr + 1 + 2 * d0 + d1
                busy = np.full(n, g["head_select"] == 3)  # ranked heads: explicit targets
                while np.any(busy):
                    a = rows[busy]
                    m = meta[hr[a], k].astype(np.int64)
                    right = ~(X[a, m >> 22] <= thr[hr[a], k])
                    hr[a] = np.where(right, (m >> 11) & 2047, m & 2047)
                    busy[a] = hr[a] < nr
                e = hr - nr
                ref = exits[e, k]
                lf = (ref & LEAF) != 0
                cls[lf, t] = (ref[lf] & 0x7FFFFFFF).astype(np.int32)
                leaf[lf, t] = par[e[lf], k]
                state = np.where(lf, 2, 1).astype(np.int8)
                idx = np.where(lf, -1, ref.astype(np.int64))  # super-node references are global
                while np.any(state == 1):
                    a = rows[state == 1]
                    g_idx = idx[a]
                    if g["deep_levels"] == 3:
                        step = self._step3p if self.fmt == 2 else self._step3
                        ex, nref, c3 = step(X, a, g_idx)
                        fin = (nref & LEAF) != 0
                        fa = a[fin]
                        cls[fa, t] = c3[fin]
                        leaf[fa, t] = self.deep_leaf[g_idx[fin], ex[fin]]
                        state[fa] = 2
                        idx[a[~fin]] = nref[~fin]
                        continue
                    w = self.sw[g_idx]
                    th = self.sthr[g_idx]
                    f0 = (w[:, 3] & 1023).astype(np.int64)
                    d0 = ~(X[a, f0] <= th[:, 0])
                    f1 = np.where(d0, (w[:, 3] >> 20) & 1023, (w[:, 3] >> 10) & 1023).astype(np.int64)
                    t1 = np.where(d0, th[:, 2], th[:, 1])
                    d1 = ~(X[a, f1] <= t1)
                    slot = 2 * d0.astype(np.int64) + d1.astype(np.int64)
                    nref = w[np.arange(len(a)), 4 + slot]
                    fin = (nref & LEAF) != 0
                    fa = a[fin]
                    cls[fa, t] = (nref[fin] & 0x7FFFFFFF).astype(np.int32)
                    leaf[fa, t] = self.deep_leaf[g_idx[fin], slot[fin]]
                    state[fa] = 2
                    idx[a[~fin]] = nref[~fin]
        return leaf, cls

    def _step3(self, X, a, g_idx):
        """One three-level super-node per row of a: (exit, next reference or
        LEAF, class or value slot).  The first two levels compare full keys;
        the last decides by its key prefix, checked wherever the prefixes
        differ to agree with the full key; ties are counted."""
        g = self.h
        fb, cb = g["feature_bits"], g["class_bits"]
        fm, s2 = (1 << fb) - 1, 2 * fb + 2 * cb
        w = self.sw[g_idx].astype(np.int64)
        K = self.deep_keys[g_idx].astype(np.int64)
        ar = np.arange(len(a))
        e0 = X[a, (w[:, 3] >> fb) & fm] > w[:, 0]
        n1 = np.where(e0, w[:, 2], w[:, 1])
        e1 = X[a, (np.where(e0, w[:, 5], w[:, 4]) >> fb) & fm] > n1
        j = 2 * e0.astype(np.int64) + e1.astype(np.int64)
        n2 = w[ar, 3 + j]
        k2 = X[a, n2 & fm]
        e2 = k2 > K[ar, j]
        p2, t2 = (k2 >> s2) > (n2 >> s2), (k2 >> s2) == (n2 >> s2)
        assert np.all(t2 | (p2 == e2)), "a key prefix decided against the full key"
        self.ties += int(np.sum(t2))
        ex = 2 * j + e2.astype(np.int64)
        mask = w[:, 7] >> 24
        is_leaf = ((mask >> ex) & 1) == 1
        nref = g_idx.astype(np.int64) + (w[:, 7] & 0xFFFFFF) + _popc8(~mask & ((1 << ex) - 1))
        nref = np.where(is_leaf, LEAF, nref)
        if g["n_values"]:
            c3 = g["values3_base"] + 8 * g_idx.astype(np.int64) + ex
        else:
            c3 = (n2 >> (2 * fb + cb * e2.astype(np.int64))) & ((1 << cb) - 1)
        return ex, nref, c3.astype(np.int32)

    def _step3p(self, X, a, g_idx):
        """One three-level super-node of format 2 per row of a: every slot's
        word holds the top bits of its remapped key over its feature (and, in
        the last level, the exits' classes).  The walk follows the full keys
        of the side table; every compare where the row's top bits differ from
        the slot's must agree with the word compare, and the others (ties)
        are counted."""
        g = self.h
        fb, cb = g["feature_bits"], g["class_bits"]
        fm = (1 << fb) - 1
        w = self.sw[g_idx].astype(np.int64)
        K = self.deep_keys[g_idx].astype(np.int64)
        ar = np.arange(len(a))

        def decide(slot_word, full, low):
            x = X[a, slot_word & fm]
            e = x > full
            differ = (x >> low) != (slot_word >> low)
            assert np.all(~differ | ((x > slot_word) == e)), "a key prefix decided against the full key"
            self.ties += int(np.sum(~differ))
            return e

        e0 = decide(w[:, 0], K[:, 0], fb)
        i1 = 1 + e0.astype(np.int64)
        e1 = decide(w[ar, i1], K[ar, i1], fb)
        j = 2 * e0.astype(np.int64) + e1.astype(np.int64)
        n2 = w[ar, 3 + j]
        e2 = decide(n2, K[ar, 3 + j], fb + 2 * cb)
        ex = 2 * j + e2.astype(np.int64)
        mask = w[:, 7] >> 24
        is_leaf = ((mask >> ex) & 1) == 1
        nref = g_idx.astype(np.int64) + (w[:, 7] & 0xFFFFFF) + _popc8(~mask & ((1 << ex) - 1))
        nref = np.where(is_leaf, LEAF, nref)
        if g["n_values"]:
            c3 = g["values3_base"] + 8 * g_idx.astype(np.int64) + ex
        else:
            c3 = (n2 >> (fb + cb * e2.astype(np.int64))) & ((1 << cb) - 1)
        return ex, nref, c3.astype(np.int32)
