// fp_pack.cpp -- host layout builder: trained forest -> packed image.
//
// Implements the layout of Section III-A of the paper, adapted to 8-byte
// records and a GPU that stages each bin's interleaved block in shared memory:
//   DF-  (Section III-A): leaves are not stored; the parent record carries the
//        leaf's class (the paper's shared per-class nodes, folded into the
//        parent so no extra load is spent on them);
//   Stat (Section III-A): below the interleaved levels each tree is laid out
//        depth-first with the child of larger training cardinality placed
//        immediately after its parent (left on ties); when one child is a leaf
//        the internal child is the adjacent one;
//   Bin  (Section III-A, Fig. 2, Fig. 3): trees [bB, (b+1)B) form bin b; the
//        nodes of levels 0..d of the bin's trees are interleaved slot by slot
//        (head[s*width + k]), so the roots of all trees of a bin are
//        contiguous (Fig. 2: depth 0 = roots only); level d+1 is a row of
//        4-byte links into each tree's Stat region.
// The image format is described in fp_internal.h.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/forest_pack.h"
#include "fp_internal.h"
#include "fp_common.h"

namespace {
thread_local std::string g_last_error;
}

void fp_set_error(const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
}

extern "C" const char *fp_last_error(void) { return g_last_error.c_str(); }

struct fp_packed_forest {
    FpImageHeader hdr;
    std::vector<uint8_t> image;
};

namespace {

int64_t align_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

struct TreeRef {
    const int32_t *L, *R, *Fe, *Cl;
    const float *Th;
    const int64_t *Card;
    int64_t m;
    bool leaf(int32_t v) const { return L[v] < 0; }
};

// Validate one tree: child ids in range, leaves consistent, every node
// reachable from the root at most once (a tree, not a graph).
int validate_tree(const TreeRef &t, int32_t F, int32_t C, int32_t ti, std::vector<uint8_t> &seen) {
    if (t.m < 1) {
        fp_set_error("tree %d has no nodes", ti);
        return FP_EINVAL;
    }
    if (t.m > INT32_MAX) {
        fp_set_error("tree %d has too many nodes", ti);
        return FP_EUNSUPPORTED;
    }
    for (int64_t v = 0; v < t.m; ++v) {
        if (t.L[v] < 0) {
            if (t.L[v] != -1 || t.R[v] != -1) {
                fp_set_error("tree %d node %lld: leaf must have left = right = -1", ti, (long long)v);
                return FP_EINVAL;
            }
            if (t.Cl[v] < 0 || t.Cl[v] >= C) {
                fp_set_error("tree %d node %lld: leaf class %d out of range", ti, (long long)v, t.Cl[v]);
                return FP_EINVAL;
            }
        } else {
            if (t.L[v] >= t.m || t.R[v] < 0 || t.R[v] >= t.m || t.L[v] == t.R[v] || t.L[v] == v || t.R[v] == v) {
                fp_set_error("tree %d node %lld: bad child ids", ti, (long long)v);
                return FP_EINVAL;
            }
            if (t.Fe[v] < 0 || t.Fe[v] >= F) {
                fp_set_error("tree %d node %lld: feature %d out of range", ti, (long long)v, t.Fe[v]);
                return FP_EINVAL;
            }
        }
    }
    seen.assign((size_t)t.m, 0);
    std::vector<int32_t> stack{0};
    while (!stack.empty()) {
        int32_t v = stack.back();
        stack.pop_back();
        if (seen[v]) {
            fp_set_error("tree %d: node %d reached twice (not a tree)", ti, v);
            return FP_EINVAL;
        }
        seen[v] = 1;
        if (!t.leaf(v)) {
            stack.push_back(t.R[v]);
            stack.push_back(t.L[v]);
        }
    }
    return FP_OK;
}

// Stat rule: is the right child the hot (adjacent) one?
bool hot_is_right(const TreeRef &t, int32_t v) {
    int32_t l = t.L[v], r = t.R[v];
    bool li = !t.leaf(l), ri = !t.leaf(r);
    if (li != ri) return ri;
    if (!t.Card) return false;
    return t.Card[r] > t.Card[l];
}

struct TreeLayout {
    // head: node id per BFS slot (-1 = empty) for slots 0..S+L-1
    std::vector<int32_t> slot_node;
    // deep: node ids in record order
    std::vector<int32_t> deep_nodes;
    std::vector<int32_t> deep_index;  // node id -> record index (-1 if not deep)
};

int layout_tree(const TreeRef &t, int32_t d, int32_t S, int32_t Lk, TreeLayout &out, int32_t ti) {
    out.slot_node.assign((size_t)(S + Lk), -1);
    out.slot_node[0] = 0;
    for (int32_t s = 0; s < S; ++s) {
        int32_t v = out.slot_node[s];
        if (v < 0 || t.leaf(v)) continue;
        out.slot_node[2 * s + 1] = t.L[v];
        out.slot_node[2 * s + 2] = t.R[v];
    }
    out.deep_index.assign((size_t)t.m, -1);
    out.deep_nodes.clear();
    // deep roots: internal nodes at level d+1, in link order; each subtree in
    // hot-first pre-order (explicit stack: hot child pops first)
    std::vector<int32_t> stack;
    for (int32_t j = 0; j < Lk; ++j) {
        int32_t root = out.slot_node[S + j];
        if (root < 0 || t.leaf(root)) continue;
        stack.push_back(root);
        while (!stack.empty()) {
            int32_t v = stack.back();
            stack.pop_back();
            out.deep_index[v] = (int32_t)out.deep_nodes.size();
            out.deep_nodes.push_back(v);
            bool hr = hot_is_right(t, v);
            int32_t hot = hr ? t.R[v] : t.L[v], cold = hr ? t.L[v] : t.R[v];
            if (!t.leaf(cold)) stack.push_back(cold);
            if (!t.leaf(hot)) stack.push_back(hot);
        }
    }
    if ((int64_t)out.deep_nodes.size() >= FP_MAX_DEEP_PER_TREE) {
        fp_set_error("tree %d holds %zu records below the interleaved levels; the record format addresses %d",
                     ti, out.deep_nodes.size(), FP_MAX_DEEP_PER_TREE - 1);
        return FP_EUNSUPPORTED;
    }
    return FP_OK;
}

uint32_t encode_deep(const TreeRef &t, const TreeLayout &lay, int32_t v) {
    int32_t l = t.L[v], r = t.R[v];
    uint32_t meta = (uint32_t)t.Fe[v] << FP_META_FEATURE_SHIFT;
    if (t.leaf(l) && t.leaf(r)) {
        meta |= FP_META_BOTH_LEAF | (uint32_t)t.Cl[l] | ((uint32_t)t.Cl[r] << 9);
        return meta;
    }
    bool hr = hot_is_right(t, v);
    int32_t cold = hr ? l : r;
    if (hr) meta |= FP_META_HOT_RIGHT;
    if (t.leaf(cold)) {
        meta |= FP_META_COLD_LEAF | (uint32_t)t.Cl[cold];
    } else {
        meta |= (uint32_t)lay.deep_index[cold];
    }
    return meta;
}

}  // namespace

extern "C" int fp_pack_forest(const fp_forest_desc *desc, const fp_pack_params *params, fp_packed_forest **out) {
    if (!out) {
        fp_set_error("fp_pack_forest: out is NULL");
        return FP_EINVAL;
    }
    *out = nullptr;
    if (!desc || !desc->tree_node_begin || !desc->left || !desc->right || !desc->feature || !desc->threshold ||
        !desc->leaf_class) {
        fp_set_error("fp_pack_forest: NULL forest array");
        return FP_EINVAL;
    }
    const int32_t T = desc->n_trees, F = desc->n_features, C = desc->n_classes;
    if (T < 1 || T > (1 << 24) || F < 1 || F > FP_MAX_FEATURES || C < 1 || C > FP_MAX_CLASSES) {
        fp_set_error("fp_pack_forest: n_trees %d, n_features %d (1..%d), n_classes %d (1..%d)", T, F,
                     FP_MAX_FEATURES, C, FP_MAX_CLASSES);
        return (F > FP_MAX_FEATURES || C > FP_MAX_CLASSES) ? FP_EUNSUPPORTED : FP_EINVAL;
    }
    if (desc->tree_node_begin[0] != 0) {
        fp_set_error("fp_pack_forest: tree_node_begin[0] must be 0");
        return FP_EINVAL;
    }
    fp_pack_params p = params ? *params : fp_pack_params{0, -1, 0, 0, 0};
    int32_t B = p.bin_size ? p.bin_size : std::min(T, 32);
    int32_t d = p.interleave_depth >= 0 ? p.interleave_depth : 4;
    int32_t W = p.warps_per_cta ? p.warps_per_cta : 8;
    const int32_t P = F | 1;  // shared-memory row stride in floats (odd: no bank conflicts on one feature)
    int32_t R = p.obs_tile;
    if (R == 0) {
        int64_t r = (32 * 1024) / ((int64_t)P * 4);
        r = r / 32 * 32;
        R = (int32_t)std::max<int64_t>(32, std::min<int64_t>(1024, r));
    }
    int64_t pass_budget = p.pass_bytes ? p.pass_bytes : (int64_t)48 << 20;
    if (B < 1 || B > 1024 || d < 0 || d > FP_MAX_DEPTH || W < 1 || W > 32 || R < 32 || R > 2048 || R % 32) {
        fp_set_error("fp_pack_forest: bad params (bin_size %d, interleave_depth %d, obs_tile %d, warps %d)", B, d, R,
                     W);
        return FP_EINVAL;
    }
    if (B > T) B = T;
    const int32_t S = (1 << (d + 1)) - 1, Lk = 1 << (d + 1);
    const int32_t n_bins = (T + B - 1) / B;

    try {
        // ---- validate and lay out every tree
        std::vector<TreeLayout> lays((size_t)T);
        std::vector<uint8_t> seen;
        std::vector<int64_t> deep_count((size_t)T);
        for (int32_t t = 0; t < T; ++t) {
            int64_t b = desc->tree_node_begin[t], e = desc->tree_node_begin[t + 1];
            if (e < b) {
                fp_set_error("fp_pack_forest: tree_node_begin not monotone at tree %d", t);
                return FP_EINVAL;
            }
            TreeRef tr{desc->left + b, desc->right + b, desc->feature + b, desc->leaf_class + b, desc->threshold + b,
                       desc->cardinality ? desc->cardinality + b : nullptr, e - b};
            int rc = validate_tree(tr, F, C, t, seen);
            if (rc) return rc;
            rc = layout_tree(tr, d, S, Lk, lays[t], t);
            if (rc) return rc;
            deep_count[t] = (int64_t)lays[t].deep_nodes.size();
        }

        // ---- section sizes
        FpImageHeader h;
        memset(&h, 0, sizeof h);
        h.magic = FP_IMAGE_MAGIC;
        h.version = FP_IMAGE_VERSION;
        h.n_trees = T; h.n_features = F; h.n_classes = C;
        h.bin_size = B; h.depth = d; h.n_bins = n_bins;
        h.slots = S; h.links = Lk;
        h.obs_tile = R; h.warps_per_cta = W;
        std::vector<FpBin> bins((size_t)n_bins);
        int64_t head_total = 0, phead_total = 0;
        int32_t max_head = 0;
        for (int32_t b = 0; b < n_bins; ++b) {
            FpBin &bn = bins[b];
            memset(&bn, 0, sizeof bn);
            bn.first_tree = b * B;
            bn.width = std::min(B, T - b * B);
            int64_t bytes = align_up((int64_t)S * bn.width * 8 + (int64_t)Lk * bn.width * 4, 16);
            if (head_total + bytes > UINT32_MAX || bytes > 160 * 1024) {
                fp_set_error("fp_pack_forest: interleaved block of %lld bytes per bin is too large; lower "
                             "bin_size or interleave_depth", (long long)bytes);
                return FP_EUNSUPPORTED;
            }
            bn.head_off = (uint32_t)head_total;
            bn.head_bytes = (uint32_t)bytes;
            head_total += bytes;
            max_head = std::max<int32_t>(max_head, (int32_t)bytes);
            int64_t pbytes = align_up((int64_t)(S + Lk) * bn.width * 4, 16);
            bn.phead_off = (uint32_t)phead_total;
            phead_total += pbytes;
        }
        std::vector<int64_t> tree_base((size_t)T + 1, 0);
        for (int32_t t = 0; t < T; ++t) tree_base[t + 1] = tree_base[t] + deep_count[t];
        const int64_t n_deep = tree_base[T];
        if (n_deep > (int64_t)UINT32_MAX) {
            fp_set_error("fp_pack_forest: %lld deep records exceed the 32-bit tree base", (long long)n_deep);
            return FP_EUNSUPPORTED;
        }
        // passes: consecutive bins whose records fit the budget
        std::vector<FpPass> passes;
        {
            int32_t b0 = 0;
            int64_t acc = 0;
            for (int32_t b = 0; b < n_bins; ++b) {
                int64_t bytes = bins[b].head_bytes +
                                8 * (tree_base[bins[b].first_tree + bins[b].width] - tree_base[bins[b].first_tree]);
                if (pass_budget > 0 && b > b0 && acc + bytes > pass_budget) {
                    passes.push_back({b0, b});
                    b0 = b;
                    acc = 0;
                }
                acc += bytes;
            }
            passes.push_back({b0, n_bins});
        }
        h.n_passes = (int32_t)passes.size();
        h.max_head_bytes = max_head;
        h.n_deep = n_deep;
        h.head_bytes_total = head_total;
        h.pass_bytes = pass_budget;

        int64_t off = align_up(sizeof(FpImageHeader), 256);
        h.off_bins = off; off = align_up(off + (int64_t)sizeof(FpBin) * n_bins, 256);
        h.off_passes = off; off = align_up(off + (int64_t)sizeof(FpPass) * h.n_passes, 256);
        h.off_tree_base = off; off = align_up(off + 4 * (int64_t)T, 256);
        h.off_heads = off; off = align_up(off + head_total, 256);
        h.off_deep = off; off = align_up(off + 8 * n_deep, 256);
        h.class_bytes = off;
        h.off_pheads = off; off = align_up(off + phead_total, 256);
        h.off_deep_leaf = off; off = align_up(off + 8 * n_deep, 256);
        h.total_bytes = off;

        auto *pf = new fp_packed_forest;
        pf->hdr = h;
        pf->image.assign((size_t)h.total_bytes, 0);
        uint8_t *img = pf->image.data();
        memcpy(img, &h, sizeof h);
        memcpy(img + h.off_bins, bins.data(), sizeof(FpBin) * bins.size());
        memcpy(img + h.off_passes, passes.data(), sizeof(FpPass) * passes.size());
        uint32_t *tb = reinterpret_cast<uint32_t *>(img + h.off_tree_base);
        for (int32_t t = 0; t < T; ++t) tb[t] = (uint32_t)tree_base[t];

        // ---- heads (interleaved, slot-major) and their parity mirror
        for (int32_t b = 0; b < n_bins; ++b) {
            const FpBin &bn = bins[b];
            uint8_t *blk = img + h.off_heads + bn.head_off;
            uint32_t *link = reinterpret_cast<uint32_t *>(blk + (int64_t)S * bn.width * 8);
            int32_t *phead = reinterpret_cast<int32_t *>(img + h.off_pheads + bn.phead_off);
            for (int32_t k = 0; k < bn.width; ++k) {
                const int32_t t = bn.first_tree + k;
                const int64_t nb = desc->tree_node_begin[t];
                TreeRef tr{desc->left + nb, desc->right + nb, desc->feature + nb, desc->leaf_class + nb,
                           desc->threshold + nb, nullptr, desc->tree_node_begin[t + 1] - nb};
                const TreeLayout &lay = lays[t];
                for (int32_t s = 0; s < S; ++s) {
                    int32_t v = lay.slot_node[s];
                    float thr = 0.0f;
                    uint32_t meta = FP_HEAD_EMPTY;
                    int32_t leaf_id = -1;
                    if (v >= 0 && tr.leaf(v)) {
                        meta = FP_HEAD_LEAF | (uint32_t)tr.Cl[v];
                        leaf_id = v;
                    } else if (v >= 0) {
                        thr = tr.Th[v];
                        meta = (uint32_t)tr.Fe[v];
                    }
                    uint8_t *rec = blk + ((int64_t)s * bn.width + k) * 8;
                    memcpy(rec, &thr, 4);
                    memcpy(rec + 4, &meta, 4);
                    phead[(int64_t)s * bn.width + k] = leaf_id;
                }
                for (int32_t j = 0; j < Lk; ++j) {
                    int32_t v = lay.slot_node[S + j];
                    uint32_t e = FP_HEAD_EMPTY;
                    int32_t leaf_id = -1;
                    if (v >= 0 && tr.leaf(v)) {
                        e = FP_HEAD_LEAF | (uint32_t)tr.Cl[v];
                        leaf_id = v;
                    } else if (v >= 0) {
                        e = (uint32_t)lay.deep_index[v];
                    }
                    link[(int64_t)j * bn.width + k] = e;
                    phead[(int64_t)(S + j) * bn.width + k] = leaf_id;
                }
            }
        }

        // ---- deep records and leaf-id side table
        uint8_t *deep = img + h.off_deep;
        int32_t *dleaf = reinterpret_cast<int32_t *>(img + h.off_deep_leaf);
        for (int32_t t = 0; t < T; ++t) {
            const int64_t nb = desc->tree_node_begin[t];
            TreeRef tr{desc->left + nb, desc->right + nb, desc->feature + nb, desc->leaf_class + nb,
                       desc->threshold + nb, desc->cardinality ? desc->cardinality + nb : nullptr,
                       desc->tree_node_begin[t + 1] - nb};
            const TreeLayout &lay = lays[t];
            for (size_t i = 0; i < lay.deep_nodes.size(); ++i) {
                int32_t v = lay.deep_nodes[i];
                float thr = tr.Th[v];
                uint32_t meta = encode_deep(tr, lay, v);
                int64_t g = tree_base[t] + (int64_t)i;
                memcpy(deep + g * 8, &thr, 4);
                memcpy(deep + g * 8 + 4, &meta, 4);
                dleaf[2 * g] = tr.leaf(tr.L[v]) ? tr.L[v] : -1;
                dleaf[2 * g + 1] = tr.leaf(tr.R[v]) ? tr.R[v] : -1;
            }
        }
        *out = pf;
        return FP_OK;
    } catch (const std::bad_alloc &) {
        fp_set_error("fp_pack_forest: out of host memory");
        return FP_ENOMEM;
    } catch (...) {
        fp_set_error("fp_pack_forest: unexpected failure");
        return FP_EINVAL;
    }
}

extern "C" int fp_packed_info_get(const fp_packed_forest *pf, fp_packed_info *info) {
    if (!pf || !info) {
        fp_set_error("fp_packed_info_get: NULL argument");
        return FP_EINVAL;
    }
    fp_fill_info(&pf->hdr, info);
    return FP_OK;
}

void fp_fill_info(const FpImageHeader *h, fp_packed_info *info) {
    memset(info, 0, sizeof *info);
    info->n_trees = h->n_trees;
    info->n_features = h->n_features;
    info->n_classes = h->n_classes;
    info->bin_size = h->bin_size;
    info->interleave_depth = h->depth;
    info->n_bins = h->n_bins;
    info->obs_tile = h->obs_tile;
    info->warps_per_cta = h->warps_per_cta;
    info->n_deep_records = h->n_deep;
    info->head_bytes = h->head_bytes_total;
    info->deep_bytes = 8 * h->n_deep;
    info->total_bytes = h->class_bytes;
    info->parity_bytes = h->total_bytes - h->class_bytes;
    info->max_head_bytes = h->max_head_bytes;
    info->passes = h->n_passes;
}

extern "C" const void *fp_packed_image(const fp_packed_forest *pf, int64_t *bytes) {
    if (!pf) {
        fp_set_error("fp_packed_image: NULL forest");
        return nullptr;
    }
    if (bytes) *bytes = (int64_t)pf->image.size();
    return pf->image.data();
}

extern "C" void fp_release_packed(fp_packed_forest *pf) { delete pf; }

const FpImageHeader *fp_packed_header(const fp_packed_forest *pf) { return &pf->hdr; }
const uint8_t *fp_packed_bytes(const fp_packed_forest *pf) { return pf->image.data(); }
