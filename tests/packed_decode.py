"""Host-side reader of the library's packed image (format in
paper_1806_07300_gb300/csrc/fp_internal.h), written independently of the CUDA
kernel: it lets CPU tests check the packer's records without a GPU."""
from __future__ import annotations

import numpy as np

HDR = np.dtype([("magic", "<u4"), ("version", "<u4"), ("n_trees", "<i4"), ("n_features", "<i4"),
                ("n_classes", "<i4"), ("bin_size", "<i4"), ("depth", "<i4"), ("n_bins", "<i4"),
                ("n_passes", "<i4"), ("slots", "<i4"), ("links", "<i4"), ("obs_tile", "<i4"),
                ("warps_per_cta", "<i4"), ("max_head_bytes", "<i4"), ("n_deep", "<i8"), ("off_bins", "<i8"),
                ("off_passes", "<i8"), ("off_tree_base", "<i8"), ("off_heads", "<i8"), ("off_deep", "<i8"),
                ("off_pheads", "<i8"), ("off_deep_leaf", "<i8"), ("class_bytes", "<i8"), ("total_bytes", "<i8"),
                ("head_bytes_total", "<i8"), ("pass_bytes", "<i8")], align=True)
BIN = np.dtype([("head_off", "<u4"), ("head_bytes", "<u4"), ("first_tree", "<i4"), ("width", "<i4"),
                ("phead_off", "<u4"), ("pad", "<u4", 3)])
PASS = np.dtype([("bin_begin", "<i4"), ("bin_end", "<i4")])

LEAF = 0x80000000
HOT_RIGHT = 1 << 21
COLD_LEAF = 1 << 20
BOTH_LEAF = 1 << 19
PAYLOAD = 0x7FFFF


class Image:
    def __init__(self, img: np.ndarray):
        self.img = img
        h = np.frombuffer(img[:HDR.itemsize].tobytes(), HDR)[0]
        self.h = {k: int(h[k]) for k in HDR.names}
        g = self.h
        self.bins = np.frombuffer(img[g["off_bins"]: g["off_bins"] + BIN.itemsize * g["n_bins"]].tobytes(), BIN)
        self.passes = np.frombuffer(img[g["off_passes"]: g["off_passes"] + 8 * g["n_passes"]].tobytes(), PASS)
        self.tree_base = img[g["off_tree_base"]: g["off_tree_base"] + 4 * g["n_trees"]].view("<u4")
        deep = img[g["off_deep"]: g["off_deep"] + 8 * g["n_deep"]]
        self.deep_thr = deep.view("<f4")[0::2]
        self.deep_meta = deep.view("<u4")[1::2]
        dl = img[g["off_deep_leaf"]: g["off_deep_leaf"] + 8 * g["n_deep"]].view("<i4")
        self.deep_leaf = dl.reshape(-1, 2)

    def head(self, b: int):
        """(thr [S][w], meta [S][w], link [L][w], parity [S+L][w]) of bin b."""
        g, bn = self.h, self.bins[b]
        w, S, L = int(bn["width"]), g["slots"], g["links"]
        base = g["off_heads"] + int(bn["head_off"])
        recs = self.img[base: base + 8 * S * w]
        thr = recs.view("<f4")[0::2].reshape(S, w)
        meta = recs.view("<u4")[1::2].reshape(S, w)
        link = self.img[base + 8 * S * w: base + 8 * S * w + 4 * L * w].view("<u4").reshape(L, w)
        pb = g["off_pheads"] + int(bn["phead_off"])
        par = self.img[pb: pb + 4 * (S + L) * w].view("<i4").reshape(S + L, w)
        return thr, meta, link, par

    def walk(self, X: np.ndarray):
        """Leaf id and class per (observation, tree), decoding the records."""
        g = self.h
        n, T, S = X.shape[0], g["n_trees"], g["slots"]
        leaf = np.full((n, T), -2, np.int32)
        cls = np.full((n, T), -2, np.int32)
        rows = np.arange(n)
        for b in range(g["n_bins"]):
            thr, meta, link, par = self.head(b)
            bn = self.bins[b]
            for k in range(int(bn["width"])):
                t = int(bn["first_tree"]) + k
                s = np.zeros(n, np.int64)
                idx = np.full(n, -1, np.int64)
                state = np.zeros(n, np.int8)  # 0 head, 1 deep, 2 done
                while np.any(state == 0):
                    a = rows[state == 0]
                    m = meta[s[a], k]
                    is_leaf = (m & LEAF) != 0
                    la = a[is_leaf]
                    cls[la, t] = (m[is_leaf] & 0x7FFFFFFF).astype(np.int32)
                    leaf[la, t] = par[s[la], k]
                    state[la] = 2
                    a, m = a[~is_leaf], m[~is_leaf]
                    x = X[a, m.astype(np.int64)]
                    right = ~(x <= thr[s[a], k])
                    s[a] = 2 * s[a] + 1 + right
                    out = a[s[a] >= S]
                    e = link[s[out] - S, k]
                    el = (e & LEAF) != 0
                    cls[out[el], t] = (e[el] & 0x7FFFFFFF).astype(np.int32)
                    leaf[out[el], t] = par[s[out[el]], k]
                    state[out[el]] = 2
                    idx[out[~el]] = e[~el]
                    state[out[~el]] = 1
                base = int(self.tree_base[t])
                while np.any(state == 1):
                    a = rows[state == 1]
                    g_idx = base + idx[a]
                    m = self.deep_meta[g_idx]
                    x = X[a, (m >> 22).astype(np.int64)]
                    right = ~(x <= self.deep_thr[g_idx])
                    pay = m & PAYLOAD
                    both = (m & BOTH_LEAF) != 0
                    hot = (right.astype(np.uint32) == ((m >> 21) & 1)) & ~both
                    cold_leaf = (m & COLD_LEAF) != 0
                    fin = both | (~hot & cold_leaf)
                    c = np.where(both, np.where(right, pay >> 9, pay & 511), pay)
                    fa = a[fin]
                    cls[fa, t] = c[fin].astype(np.int32)
                    leaf[fa, t] = self.deep_leaf[g_idx[fin], right[fin].astype(np.int64)]
                    state[fa] = 2
                    idx[a[hot]] += 1
                    jump = ~fin & ~hot
                    idx[a[jump]] = pay[jump]
        return leaf, cls
