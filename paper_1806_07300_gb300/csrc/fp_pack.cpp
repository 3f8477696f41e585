// fp_pack.cpp -- host layout builder: trained forest -> packed image.
//
// Implements the layout of Section III-A of the paper for a GPU that stages
// each bin's interleaved block in shared memory and reads the rest of a tree
// in 32-byte sectors:
//   Bin  (Section III-A, Fig. 2, Fig. 3): trees [bB, (b+1)B) form bin b; the
//        heads of the bin's trees are interleaved node by node
//        (node[slot*stride + k]), so the roots of all trees of a bin are
//        contiguous (Fig. 2: depth 0 = roots only) and the block is staged
//        into shared memory in one piece.  A head is either levels 0..d in
//        implicit breadth-first slots (the paper's interleaved levels; one
//        8-byte node per slot, or, paired, a node and its two children per
//        16-byte slot) or the 2^(d+1)-1 most frequently visited nodes of the
//        tree, ranked;
//   DF-  (Section III-A): leaves are not stored as nodes; a reference to a
//        leaf carries its class (the paper's shared per-class nodes, folded
//        into the reference so no load is spent on them);
//   Stat (Section III-A): below the interleaved levels a tree is cut into
//        super-nodes (one 32-byte sector, one load) of two levels (a node
//        and its two children) laid out depth-first with the child
//        super-node of largest training cardinality immediately after its
//        parent -- the paper's "more likely path adjacent" rule at the
//        granularity of the GPU's memory transaction -- or of three levels
//        (seven nodes, thresholds shortened to key prefixes), whose children
//        sit side by side and whose most frequently reached child is laid
//        out first.
// The image format is described in fp_internal.h.
#include <algorithm>
#include <cmath>
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

// The order key of a threshold: x <= t exactly when key(x) <= thr_key(t),
// with the kernel's key of an observation value (NaN -> 0xFFFFFFFF); a NaN
// threshold gets 0, below every observation key, so every x goes right.
uint32_t thr_key(float t) {
    uint32_t u;
    memcpy(&u, &t, 4);
    if ((u & 0x7FFFFFFFu) > 0x7F800000u) return 0u;
    if (u == 0x80000000u) u = 0u;  // -0 orders as +0
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// A threshold as stored: its order key when the forest compares keys (with
// three-level super-nodes), else its float bits.
uint32_t thr_word(float t, bool keys) {
    if (keys) return thr_key(t);
    uint32_t u;
    memcpy(&u, &t, 4);
    return u;
}

// How a forest stores its thresholds: float bits (two-level super-nodes),
// order keys (three-level, format 1) or remapped order keys V (format 2; the
// map is in fp_internal.h).
struct KeyMap {
    int kind = 0;  // 0 float bits, 1 keys, 2 remapped keys
    uint32_t lo = 0, hi = 0xFFFFFFFFu, shl = 0, flag = 0;
    uint32_t ga = 0xFFFFFFFFu, gb = 0xFFFFFFFFu, gd = 0;  // the collapsed run of keys

    uint32_t gap(uint32_t k) const { return k >= gb ? k - gd : std::min(k, ga); }
    // V of an order key
    uint32_t remap(uint32_t k) const {
        const uint32_t g = gap(k);
        const uint32_t c = g < lo ? lo : (g > hi ? hi : g);
        return flag | ((c - lo) << shl);
    }
    uint32_t word(float t) const {
        if (kind == 0) {
            uint32_t u;
            memcpy(&u, &t, 4);
            return u;
        }
        const uint32_t k = thr_key(t);
        return (kind == 1 || k == 0) ? k : remap(k);  // a NaN threshold stays 0
    }
};

// The remap of format 2 over the thresholds of every internal node of the
// forest: the widest run of keys without a threshold collapsed, then [lo, hi]
// spread over 31 bits below a set top bit, or left as they are when that
// range needs 32 bits.
KeyMap make_remap(const fp_forest_desc *desc) {
    KeyMap km;
    km.kind = 2;
    std::vector<uint32_t> keys;
    const int64_t m = desc->tree_node_begin[desc->n_trees];
    for (int64_t v = 0; v < m; ++v) {
        if (desc->left[v] < 0) continue;
        const uint32_t k = thr_key(desc->threshold[v]);
        if (k != 0) keys.push_back(k);  // 0: NaN
    }
    if (keys.empty()) keys.push_back(0x80000000u);  // no thresholds
    std::sort(keys.begin(), keys.end());
    keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
    uint32_t best = 0;
    size_t at = 0;
    for (size_t i = 1; i < keys.size(); ++i)
        if (keys[i] - keys[i - 1] > best) {
            best = keys[i] - keys[i - 1];
            at = i;
        }
    if (best > 2) {  // a run of at least two keys between adjacent thresholds
        km.ga = keys[at - 1] + 1;
        km.gb = keys[at];
        km.gd = keys[at] - keys[at - 1] - 2;
    }
    const uint32_t lo = keys.front(), top = km.gap(keys.back());
    const uint64_t range = (uint64_t)top + 1 - lo;
    int32_t b = 0;
    while (b < 64 && (range >> b) != 0) ++b;
    if (b <= 31) {
        km.lo = lo;
        km.hi = top + 1;  // top is at most the key of +inf, so no wrap
        km.shl = (uint32_t)(31 - b);
        km.flag = 0x80000000u;
    }
    return km;
}

// bits that hold the values 0 .. n-1 (at least 1)
int32_t bits_for(int32_t n) {
    int32_t b = 1;
    while (b < 31 && ((int64_t)1 << b) < n) ++b;
    return b;
}

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

struct TreeLayout {
    std::vector<int32_t> slot;       // level heads: node id per implicit slot (a leaf = dummy slot)
    std::vector<int32_t> head;       // node id per head rank
    std::vector<uint32_t> head_meta; // unused (kept zero); targets are encoded per bin
    std::vector<int32_t> rank;       // node id -> head rank (-1 outside the head)
    std::vector<int32_t> exits;      // node id behind each exit (leaf or deep root)
    std::vector<int32_t> sn_root;    // root node of each super-node, in layout order
    std::vector<int32_t> sn_index;   // node id -> super-node index (-1 if it roots none)
    std::vector<int32_t> sn_first;   // three-level: super-node index -> its first child's index (0: none)
    std::vector<int32_t> leaf_rank;  // forests with leaf values: node id -> rank among the tree's leaves
    int64_t value_base = -1;         // forests with leaf values: the tree's first value slot
};

// The four exits of the super-node rooted at v: the grandchildren through
// internal children, or the leaf child itself (twice).
void super_exits(const TreeRef &t, int32_t v, int32_t e[4]) {
    const int32_t l = t.L[v], r = t.R[v];
    if (t.leaf(l)) { e[0] = e[1] = l; } else { e[0] = t.L[l]; e[1] = t.R[l]; }
    if (t.leaf(r)) { e[2] = e[3] = r; } else { e[2] = t.L[r]; e[3] = t.R[r]; }
}

// The seven slots and eight exits of the three-level super-node rooted at v;
// a leaf is carried down into every slot and exit below it.
void slots3(const TreeRef &t, int32_t v, int32_t s[7], int32_t e[8]) {
    s[0] = v;
    for (int i = 0; i < 7; ++i) {
        const int32_t u = s[i];
        const int32_t l = t.leaf(u) ? u : t.L[u], r = t.leaf(u) ? u : t.R[u];
        if (i < 3) {
            s[2 * i + 1] = l;
            s[2 * i + 2] = r;
        } else {
            e[2 * (i - 3)] = l;
            e[2 * (i - 3) + 1] = r;
        }
    }
}

int64_t card_of(const TreeRef &t, int32_t v) { return t.Card ? t.Card[v] : 0; }

int finish_super(const TreeRef &t, struct TreeLayout &out, int32_t ti, bool three);

// Head, when select_levels is set: levels 0..d in K = 2^(d+1)-1 implicit
// breadth-first slots (the interleaved levels of the Bin layout).
// Otherwise: the K internal nodes of highest training cardinality (ties:
// shallower, then lower node id) -- the most popular paths of Section III-A,
// kept in fast memory -- which contain every ancestor of their members,
// ranked depth-first, more frequently reached child first (Stat), so the
// first child visited inside the head sits at the next rank.  Below the head
// the tree is cut into super-nodes (a node and its two children: one 32-byte
// sector, one load) laid out depth-first with the child super-node of largest
// cardinality right after its parent (Stat at super-node granularity).
int layout_tree(const TreeRef &t, int32_t K, int32_t d, bool select_levels, bool three, TreeLayout &out,
                int32_t ti) {
    const int32_t m = (int32_t)t.m;
    if (select_levels) {
        // implicit breadth-first slots of levels 0..d; a leaf above level d+1
        // is carried down both sides, so its slot is a dummy and every exit
        // below it names the leaf
        const int32_t S = K;
        out.slot.assign((size_t)S, 0);
        out.exits.assign((size_t)S + 1, 0);
        for (int32_t s = 0; s < S; ++s) {
            const int32_t v = out.slot[s];
            const int32_t kid[2] = {t.leaf(v) ? v : t.L[v], t.leaf(v) ? v : t.R[v]};
            for (int q = 0; q < 2; ++q) {
                const int32_t c = 2 * s + 1 + q;
                if (c < S) out.slot[c] = kid[q];
                else out.exits[c - S] = kid[q];
            }
        }
        out.head.clear();
        return finish_super(t, out, ti, three);
    }
    std::vector<int32_t> depth((size_t)m, 0);
    std::vector<int32_t> order;  // breadth-first
    order.reserve((size_t)m);
    order.push_back(0);
    for (size_t i = 0; i < order.size(); ++i) {
        const int32_t v = order[i];
        if (t.leaf(v)) continue;
        depth[t.L[v]] = depth[v] + 1;
        depth[t.R[v]] = depth[v] + 1;
        order.push_back(t.L[v]);
        order.push_back(t.R[v]);
    }
    std::vector<uint8_t> in_head((size_t)m, 0);
    if (!t.leaf(0)) {
        std::vector<int32_t> cand;
        for (int32_t v : order)
            if (!t.leaf(v) && (!select_levels || depth[v] <= d)) cand.push_back(v);
        if (!select_levels) {
            std::stable_sort(cand.begin(), cand.end(), [&](int32_t a, int32_t b) {
                const int64_t ca = card_of(t, a), cb = card_of(t, b);
                if (ca != cb) return ca > cb;
                if (depth[a] != depth[b]) return depth[a] < depth[b];
                return a < b;
            });
            if ((int64_t)cand.size() > K) cand.resize((size_t)K);
        }
        // members reached from the root through members form the head (with
        // consistent cardinalities that is every member)
        for (int32_t v : cand) in_head[v] = 1;
    }
    // children of v ordered for Stat: larger cardinality first, left on ties
    auto kids_hot_first = [&](int32_t v, int32_t k[2]) {
        const int32_t l = t.L[v], r = t.R[v];
        const bool right_first = card_of(t, r) > card_of(t, l);
        k[0] = right_first ? r : l;
        k[1] = right_first ? l : r;
    };
    out.head.clear();
    out.head_meta.clear();
    out.exits.clear();
    if (t.leaf(0)) {
        // a single-leaf tree: one node whose two targets name one exit holding the leaf
        out.head.push_back(0);
        out.exits.push_back(0);
        out.head_meta.push_back(0);  // targets are fixed up once the bin's nranks is known
        return finish_super(t, out, ti, three);
    }
    std::vector<int32_t> rank((size_t)m, -1);
    std::vector<int32_t> stack{0};
    while (!stack.empty()) {
        const int32_t v = stack.back();
        stack.pop_back();
        rank[v] = (int32_t)out.head.size();
        out.head.push_back(v);
        int32_t k[2];
        kids_hot_first(v, k);
        if (in_head[k[1]]) stack.push_back(k[1]);
        if (in_head[k[0]]) stack.push_back(k[0]);
    }
    // children outside the head become exits, in rank order
    out.head_meta.assign(out.head.size(), 0);
    for (size_t i = 0; i < out.head.size(); ++i) {
        const int32_t v = out.head[i];
        for (int32_t c : {t.L[v], t.R[v]})
            if (t.leaf(c) || !in_head[c]) out.exits.push_back(c);
    }
    if (out.head.size() + out.exits.size() > (size_t)FP_TARGET_MASK + 1) {
        fp_set_error("tree %d: head of %zu nodes and %zu exits exceeds the 11-bit targets", ti, out.head.size(),
                     out.exits.size());
        return FP_EUNSUPPORTED;
    }
    out.rank = rank;
    return finish_super(t, out, ti, three);
}

// Super-nodes below the head, rooted at the internal exits.  Two levels:
// depth-first, the child super-node of largest cardinality right after its
// parent.  Three levels: a super-node's children get consecutive indices in
// exit order (so one offset locates them all), and the children are expanded
// depth-first, most frequently reached first.
int finish_super(const TreeRef &t, TreeLayout &out, int32_t ti, bool three) {
    const int32_t m = (int32_t)t.m;
    out.sn_index.assign((size_t)m, -1);
    out.sn_root.clear();
    out.sn_first.clear();
    std::vector<int32_t> stack;
    if (three) {
        for (int32_t root : out.exits) {
            if (t.leaf(root) || out.sn_index[root] >= 0) continue;
            out.sn_index[root] = (int32_t)out.sn_root.size();
            out.sn_root.push_back(root);
            out.sn_first.push_back(0);
            stack.push_back(root);
            while (!stack.empty()) {
                const int32_t v = stack.back();
                stack.pop_back();
                int32_t sl[7], e[8], kids[8];
                slots3(t, v, sl, e);
                int nk = 0;
                for (int q = 0; q < 8; ++q)
                    if (!t.leaf(e[q])) kids[nk++] = e[q];
                if (nk == 0) continue;
                const int64_t first = (int64_t)out.sn_root.size();
                if (first - out.sn_index[v] > (int64_t)FP_DEEP3_OFFSET_MASK || first + nk >= (int64_t)INT32_MAX) {
                    fp_set_error("tree %d: three-level super-node offsets exceed 24 bits; use deep_levels = 2", ti);
                    return FP_EUNSUPPORTED;
                }
                out.sn_first[out.sn_index[v]] = (int32_t)first;
                for (int q = 0; q < nk; ++q) {
                    out.sn_index[kids[q]] = (int32_t)out.sn_root.size();
                    out.sn_root.push_back(kids[q]);
                    out.sn_first.push_back(0);
                }
                if (t.Card)
                    std::stable_sort(kids, kids + nk, [&](int32_t a, int32_t b) { return t.Card[a] > t.Card[b]; });
                for (int q = nk - 1; q >= 0; --q) stack.push_back(kids[q]);
            }
        }
        return FP_OK;
    }
    for (int32_t root : out.exits) {
        if (t.leaf(root) || out.sn_index[root] >= 0) continue;
        stack.push_back(root);
        while (!stack.empty()) {
            const int32_t v = stack.back();
            stack.pop_back();
            out.sn_index[v] = (int32_t)out.sn_root.size();
            out.sn_root.push_back(v);
            int32_t e[4];
            super_exits(t, v, e);
            int32_t kids[4];
            int nk = 0;
            for (int q = 0; q < 4; ++q)
                if (!t.leaf(e[q])) kids[nk++] = e[q];
            if (t.Card)
                std::stable_sort(kids, kids + nk, [&](int32_t a, int32_t b) { return t.Card[a] > t.Card[b]; });
            for (int q = nk - 1; q >= 0; --q) stack.push_back(kids[q]);
        }
    }
    if ((int64_t)out.sn_root.size() >= (int64_t)FP_REF_LEAF) {
        fp_set_error("tree %d needs more than 2^31 super-nodes", ti);
        return FP_EUNSUPPORTED;
    }
    return FP_OK;
}

// A leaf's class (or, in a forest with leaf values, its value slot), or the
// global index of the super-node rooted at v (base = the tree's first
// super-node).
uint32_t ref_of(const TreeRef &t, const TreeLayout &lay, int32_t v, int64_t base) {
    if (!t.leaf(v)) return (uint32_t)(base + lay.sn_index[v]);
    if (lay.value_base >= 0) return FP_REF_LEAF | (uint32_t)(lay.value_base + lay.leaf_rank[v]);
    return FP_REF_LEAF | (uint32_t)t.Cl[v];
}

void encode_super(const TreeRef &t, const TreeLayout &lay, int32_t v, int64_t base, FpSuper &sn,
                  int32_t leaf_ids[4]) {
    const int32_t l = t.L[v], r = t.R[v];
    sn.w[0] = thr_word(t.Th[v], false);
    sn.w[1] = t.leaf(l) ? 0u : thr_word(t.Th[l], false);
    sn.w[2] = t.leaf(r) ? 0u : thr_word(t.Th[r], false);
    const uint32_t fl = t.leaf(l) ? 0u : (uint32_t)t.Fe[l], fr = t.leaf(r) ? 0u : (uint32_t)t.Fe[r];
    sn.w[3] = (uint32_t)t.Fe[v] | (fl << 10) | (fr << 20);
    int32_t e[4];
    super_exits(t, v, e);
    for (int q = 0; q < 4; ++q) {
        sn.w[4 + q] = ref_of(t, lay, e[q], base);
        leaf_ids[q] = t.leaf(e[q]) ? e[q] : -1;
    }
}

// A three-level super-node (format in fp_internal.h): full keys of the first
// two levels, then per last-level slot its feature, one upper slot's
// feature, its exits' classes and its key prefix; the leaf mask and the
// offset to the first child.  The last level's full keys, the leaf ids and
// (forests with leaf values) the exits' values go to side tables.
void encode_super3(const TreeRef &t, const TreeLayout &lay, int32_t v, int32_t fb, int32_t cb, const float *leaf_value,
                   FpSuper &sn, uint32_t keys[4], int32_t leaf_ids[8], float *vals) {
    int32_t sl[7], e[8];
    slots3(t, v, sl, e);
    auto feat = [&](int32_t u) { return t.leaf(u) ? 0u : (uint32_t)t.Fe[u]; };
    const int32_t sh = 2 * fb + 2 * cb;
    for (int i = 0; i < 7; ++i) {
        const int32_t u = sl[i];
        const uint32_t key = t.leaf(u) ? 0u : thr_key(t.Th[u]);
        if (i < 3) {
            sn.w[i] = key;
            continue;
        }
        keys[i - 3] = key;
        sn.w[i] = (key & ~((1u << sh) - 1u)) | feat(u) | (i < 6 ? feat(sl[i - 3]) << fb : 0u);
    }
    uint32_t mask = 0;
    for (int q = 0; q < 8; ++q) {
        const int32_t c = e[q];
        leaf_ids[q] = -1;
        if (vals) vals[q] = 0.0f;
        if (!t.leaf(c)) continue;
        mask |= 1u << q;
        leaf_ids[q] = c;
        if (cb) sn.w[3 + q / 2] |= (uint32_t)t.Cl[c] << (2 * fb + cb * (q & 1));
        if (vals) vals[q] = leaf_value[c];
    }
    const int32_t first = lay.sn_first[lay.sn_index[v]];
    sn.w[7] = (mask << 24) | (first ? (uint32_t)(first - lay.sn_index[v]) : 0u);
}

// A three-level super-node of format 2 (fp_internal.h): every slot holds its
// feature beside the top bits of its remapped key (and a last-level slot its
// exits' classes between them); the seven full keys, the leaf ids and the
// exits' values go to side tables.
void encode_super3p(const TreeRef &t, const TreeLayout &lay, int32_t v, int32_t fb, int32_t cb, const KeyMap &km,
                    const float *leaf_value, FpSuper &sn, uint32_t keys[8], int32_t leaf_ids[8], float *vals) {
    int32_t sl[7], e[8];
    slots3(t, v, sl, e);
    for (int i = 0; i < 7; ++i) {
        const int32_t u = sl[i];
        const uint32_t key = t.leaf(u) ? 0u : km.word(t.Th[u]);
        const uint32_t low = i < 3 ? (uint32_t)fb : (uint32_t)(fb + 2 * cb);  // bits below the prefix
        keys[i] = key;
        sn.w[i] = (key & ~((1u << low) - 1u)) | (t.leaf(u) ? 0u : (uint32_t)t.Fe[u]);
    }
    keys[7] = 0;
    uint32_t mask = 0;
    for (int q = 0; q < 8; ++q) {
        const int32_t c = e[q];
        leaf_ids[q] = -1;
        if (vals) vals[q] = 0.0f;
        if (!t.leaf(c)) continue;
        mask |= 1u << q;
        leaf_ids[q] = c;
        if (cb) sn.w[3 + q / 2] |= (uint32_t)t.Cl[c] << (fb + cb * (q & 1));
        if (vals) vals[q] = leaf_value[c];
    }
    const int32_t first = lay.sn_first[lay.sn_index[v]];
    sn.w[7] = (mask << 24) | (first ? (uint32_t)(first - lay.sn_index[v]) : 0u);
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
    if (T < 1 || T > (1 << 20) || F < 1 || F > FP_MAX_FEATURES || C < 1 || C > FP_MAX_CLASSES) {
        fp_set_error("fp_pack_forest: n_trees %d, n_features %d (1..%d), n_classes %d (1..%d)", T, F,
                     FP_MAX_FEATURES, C, FP_MAX_CLASSES);
        return (F > FP_MAX_FEATURES || C > FP_MAX_CLASSES) ? FP_EUNSUPPORTED : FP_EINVAL;
    }
    if (desc->tree_node_begin[0] != 0) {
        fp_set_error("fp_pack_forest: tree_node_begin[0] must be 0");
        return FP_EINVAL;
    }
    fp_pack_params p = params ? *params : fp_pack_params{0, -1, 0, 0, 0, 0, 0, 0, 0, 0};
    const int32_t refill = p.refill_lanes ? p.refill_lanes : 32;
    // Defaults.  Rows of at most 384 features: bins of 3 trees with paired
    // level heads 0..9 and tiles of ~96 KiB of rows.  Wider rows (the
    // 784-feature image workload) leave shared memory for few rows, so a bin
    // should hold many trees (more tasks per bin block) with a small head:
    // bins of 32 trees, paired heads 0..3, two bin buffers and tiles of up to
    // ~200 KiB of rows, the launch measured best for such forests.
    const bool wide_rows = F > 384;
    int32_t B = p.bin_size ? p.bin_size : (wide_rows ? 32 : 3);
    const int32_t d = p.interleave_depth >= 0 ? p.interleave_depth : (wide_rows ? 3 : 9);
    // head kind: 0 = default (paired level slots when d is odd, else level slots)
    const int32_t kind = p.head_select ? p.head_select : (d % 2 ? 2 : 1);
    const int32_t W = p.warps_per_cta ? p.warps_per_cta : 32;
    const bool select_levels = kind == 1 || kind == 2;  // level heads: single or paired slots
    const bool paired = kind == 2;
    // three-level super-nodes: feature and class fields beside the key
    // prefixes; format 1 keeps full keys in its first two levels (two feature
    // fields in each last-level word), format 2 prefixes in every slot
    const int32_t fb = bits_for(F), cb = desc->leaf_value ? 0 : (C > 1 ? bits_for(C) : 0);
    const bool fit1 = 2 * fb + 2 * cb <= 24, fit2 = fb + 2 * cb <= 24;
    const bool auto1 = 2 * fb + 2 * cb <= 16, auto2 = fb + 2 * cb <= 20;  // default bounds
    int32_t fmt = 0;  // 0: two-level super-nodes
    if (p.deep_levels == 3)
        fmt = p.deep_format ? p.deep_format : (fit1 ? 1 : 2);
    else if (p.deep_levels == 0)
        fmt = p.deep_format == 1 ? (auto1 ? 1 : 0)
              : p.deep_format == 2 ? (auto2 ? 2 : 0)
                                   : (auto1 ? 1 : (auto2 ? 2 : 0));
    const bool three = fmt != 0;
    int32_t R = p.obs_tile;
    if (R == 0) {  // rows take up to ~96 KiB of shared memory (wide rows: ~200 KiB)
        int64_t r = ((wide_rows ? 200 : 96) * 1024) / ((int64_t)F * 4);
        r = r / 32 * 32;
        R = (int32_t)std::max<int64_t>(32, std::min<int64_t>(1024, r));
    }
    const int64_t pass_budget = p.pass_bytes ? p.pass_bytes : (int64_t)48 << 20;
    if (B < 1 || B > 1024 || d < 0 || d > (select_levels ? FP_MAX_LEVEL_DEPTH : FP_MAX_DEPTH) || W < 1 || W > 32 ||
        R < 32 || R > 2048 || R % 32 ||
        refill < 1 || refill > 32 || p.head_select < 0 || p.head_select > 3 || (paired && d % 2 == 0) ||
        (p.bin_buffers != 0 && p.bin_buffers != 2 && p.bin_buffers != 3) ||
        (p.deep_levels != 0 && p.deep_levels != 2 && p.deep_levels != 3) || p.deep_format < 0 ||
        p.deep_format > 2) {
        fp_set_error("fp_pack_forest: bad params (bin_size %d, interleave_depth %d, obs_tile %d, warps %d, "
                     "refill %d, head_select %d, bin_buffers %d, deep_levels %d, deep_format %d)", B, d, R, W,
                     refill, p.head_select, p.bin_buffers, p.deep_levels, p.deep_format);
        return FP_EINVAL;
    }
    if ((fmt == 1 && !fit1) || (fmt == 2 && !fit2)) {
        fp_set_error("fp_pack_forest: %d features and %d classes leave three-level super-nodes of format %d too "
                     "few key bits; use deep_format = 2 or deep_levels = 2", F, C, fmt);
        return FP_EUNSUPPORTED;
    }
    if (B > T) B = T;
    const int32_t K = (1 << (d + 1)) - 1;
    const int32_t n_bins = (T + B - 1) / B;

    try {
        // ---- validate and lay out every tree
        std::vector<TreeLayout> lays((size_t)T);
        std::vector<uint8_t> seen;
        std::vector<int64_t> deep_count((size_t)T);
        int64_t n_internal = 0, n_values = 0;
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
            rc = layout_tree(tr, K, d, select_levels, three, lays[t], t);
            if (rc) return rc;
            deep_count[t] = (int64_t)lays[t].sn_root.size();
            for (int64_t v = 0; v < tr.m; ++v) n_internal += !tr.leaf((int32_t)v);
            if (desc->leaf_value) {  // value slots: the tree's leaves in node order
                TreeLayout &lay = lays[t];
                lay.value_base = n_values;
                lay.leaf_rank.assign((size_t)tr.m, -1);
                int32_t k = 0;
                for (int64_t v = 0; v < tr.m; ++v) {
                    if (!tr.leaf((int32_t)v)) continue;
                    const float val = desc->leaf_value[b + v];
                    if (!(val - val == 0.0f)) {
                        fp_set_error("fp_pack_forest: tree %d leaf %lld has a non-finite value", t, (long long)v);
                        return FP_EINVAL;
                    }
                    lay.leaf_rank[v] = k++;
                }
                n_values += k;
                if (n_values >= (int64_t)FP_REF_LEAF) {
                    fp_set_error("fp_pack_forest: more than 2^31 leaves");
                    return FP_EUNSUPPORTED;
                }
            }
        }

        // how thresholds are stored (in the heads too)
        KeyMap km;
        if (fmt == 2) km = make_remap(desc);
        else km.kind = three ? 1 : 0;

        // ---- section sizes
        FpImageHeader h;
        memset(&h, 0, sizeof h);
        h.magic = FP_IMAGE_MAGIC;
        h.version = FP_IMAGE_VERSION;
        h.n_trees = T; h.n_features = F; h.n_classes = C;
        h.bin_size = B; h.depth = d; h.n_bins = n_bins;
        h.head_nodes = K;
        h.head_select = kind;
        h.obs_tile = R; h.warps_per_cta = W;
        h.refill_lanes = refill;
        h.bin_buffers = p.bin_buffers ? p.bin_buffers : (wide_rows ? 2 : 3);
        std::vector<FpBin> bins((size_t)n_bins);
        int64_t head_total = 0, phead_total = 0;
        int32_t max_head = 0;
        for (int32_t b = 0; b < n_bins; ++b) {
            FpBin &bn = bins[b];
            memset(&bn, 0, sizeof bn);
            bn.first_tree = b * B;
            bn.width = std::min(B, T - b * B);
            bn.stride = bn.width | 1;
            for (int32_t k = 0; k < bn.width; ++k) {
                bn.nranks = std::max<int32_t>(bn.nranks, (int32_t)(select_levels ? lays[bn.first_tree + k].slot.size()
                                                                                  : lays[bn.first_tree + k].head.size()));
                bn.nexits = std::max<int32_t>(bn.nexits, (int32_t)lays[bn.first_tree + k].exits.size());
            }
            if (paired) bn.nranks = (int32_t)(((int64_t)1 << (d + 1)) - 1) / 3;  // (4^J - 1)/3 paired slots
            if (!select_levels && bn.nranks + bn.nexits > (int32_t)FP_TARGET_MASK + 1) {
                fp_set_error("fp_pack_forest: bin %d needs %d head targets (at most %u); lower interleave_depth", b,
                             bn.nranks + bn.nexits, FP_TARGET_MASK + 1);
                return FP_EUNSUPPORTED;
            }
            const int64_t rec = paired ? 16 : 8;
            const int64_t bytes = align_up((int64_t)bn.nranks * bn.stride * rec + (int64_t)bn.nexits * bn.stride * 4, 16);
            if (head_total + bytes > UINT32_MAX || bytes > 100 * 1024) {
                fp_set_error("fp_pack_forest: interleaved block of %lld bytes per bin is too large; lower "
                             "bin_size or interleave_depth", (long long)bytes);
                return FP_EUNSUPPORTED;
            }
            bn.head_off = (uint32_t)head_total;
            bn.head_bytes = (uint32_t)bytes;
            head_total += bytes;
            max_head = std::max<int32_t>(max_head, (int32_t)bytes);
            bn.phead_off = (uint32_t)phead_total;
            phead_total += align_up((int64_t)bn.nexits * bn.stride * 4, 16);
        }
        std::vector<int64_t> tree_base((size_t)T + 1, 0);
        for (int32_t t = 0; t < T; ++t) tree_base[t + 1] = tree_base[t] + deep_count[t];
        const int64_t n_deep = tree_base[T];
        if (n_deep >= (int64_t)FP_REF_LEAF || (three && 8 * n_deep >= (int64_t)FP_REF_LEAF)) {
            fp_set_error("fp_pack_forest: %lld super-nodes exceed the 31-bit references", (long long)n_deep);
            return FP_EUNSUPPORTED;
        }
        // three-level super-nodes of a forest with leaf values: eight value slots each
        const int64_t values3_base = n_values;
        if (desc->leaf_value && three) {
            n_values += 8 * n_deep;
            if (n_values >= (int64_t)FP_REF_LEAF) {
                fp_set_error("fp_pack_forest: more than 2^31 leaf-value slots; use deep_levels = 2");
                return FP_EUNSUPPORTED;
            }
        }
        // passes: consecutive bins whose records fit the budget
        std::vector<FpPass> passes;
        {
            int32_t b0 = 0;
            int64_t acc = 0;
            for (int32_t b = 0; b < n_bins; ++b) {
                int64_t bytes = bins[b].head_bytes + (int64_t)sizeof(FpSuper) *
                                (tree_base[bins[b].first_tree + bins[b].width] - tree_base[bins[b].first_tree]);
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
        h.n_super = n_deep;
        h.n_internal = n_internal;
        h.head_bytes_total = head_total;
        h.pass_bytes = pass_budget;

        int64_t off = align_up(sizeof(FpImageHeader), 256);
        h.off_bins = off; off = align_up(off + (int64_t)sizeof(FpBin) * n_bins, 256);
        h.off_passes = off; off = align_up(off + (int64_t)sizeof(FpPass) * h.n_passes, 256);
        h.off_tree_base = off; off = align_up(off + 4 * (int64_t)T, 256);
        h.off_heads = off; off = align_up(off + head_total, 256);
        h.off_deep = off; off = align_up(off + (int64_t)sizeof(FpSuper) * n_deep, 256);
        h.deep_levels = three ? 3 : 2;
        h.feature_bits = three ? fb : 0;
        h.class_bits = three ? cb : 0;
        h.deep_format = fmt;
        h.key_lo = km.lo;
        h.key_hi = km.hi;
        h.key_shl = km.shl;
        h.key_flag = km.flag;
        h.key_gap_a = km.ga;
        h.key_gap_b = km.gb;
        h.key_gap_d = km.gd;
        h.off_deep_keys = off; off = align_up(off + (three ? (fmt == 2 ? 32 : 16) * n_deep : 0), 256);
        h.n_values = n_values;
        h.values3_base = values3_base;
        h.off_values = off; off = align_up(off + 4 * n_values, 256);
        h.class_bytes = off;
        h.off_pheads = off; off = align_up(off + phead_total, 256);
        h.off_deep_leaf = off; off = align_up(off + (three ? 32 : 16) * n_deep, 256);
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

        // ---- interleaved blocks (rank-major across the bin's trees) and their parity mirror
        for (int32_t b = 0; b < n_bins; ++b) {
            const FpBin &bn = bins[b];
            uint8_t *blk = img + h.off_heads + bn.head_off;
            uint32_t *exits = reinterpret_cast<uint32_t *>(blk + (int64_t)bn.nranks * bn.stride * (paired ? 16 : 8));
            int32_t *pexits = reinterpret_cast<int32_t *>(img + h.off_pheads + bn.phead_off);
            for (int64_t i = 0; i < (int64_t)bn.nexits * bn.stride; ++i) {
                exits[i] = FP_REF_LEAF | 0x7FFFFFFFu;  // unused entries name no class
                pexits[i] = -1;
            }
            for (int32_t k = 0; k < bn.width; ++k) {
                const int32_t t = bn.first_tree + k;
                const int64_t nb = desc->tree_node_begin[t];
                TreeRef tr{desc->left + nb, desc->right + nb, desc->feature + nb, desc->leaf_class + nb,
                           desc->threshold + nb, nullptr, desc->tree_node_begin[t + 1] - nb};
                const TreeLayout &lay = lays[t];
                if (paired) {
                    // paired slot q of super-level j (q - (4^j - 1)/3 = p) holds the node at
                    // level 2j, position p, and its two children; its four successors are
                    // 4q+1 .. 4q+4, so the walk takes two levels per 16-byte record
                    int64_t q = 0;
                    for (int64_t j = 0; q < bn.nranks; ++j) {
                        const int64_t count = (int64_t)1 << (2 * j);
                        for (int64_t pos = 0; pos < count; ++pos, ++q) {
                            const int64_t s = (((int64_t)1 << (2 * j)) - 1) + pos;  // binary slot of the node
                            const int32_t vv[3] = {lay.slot[s], lay.slot[2 * s + 1], lay.slot[2 * s + 2]};
                            uint32_t w[4] = {0, 0, 0, 0};
                            for (int c = 0; c < 3; ++c) {
                                if (tr.leaf(vv[c])) continue;  // dummy: any outcome lands on the same leaf
                                w[c] = km.word(tr.Th[vv[c]]);
                                w[3] |= (uint32_t)tr.Fe[vv[c]] << (10 * c);
                            }
                            memcpy(blk + (q * bn.stride + k) * 16, w, 16);
                        }
                    }
                    for (size_t e = 0; e < lay.exits.size(); ++e) {
                        const int32_t v = lay.exits[e];
                        exits[(int64_t)e * bn.stride + k] = ref_of(tr, lay, v, tree_base[t]);
                        pexits[(int64_t)e * bn.stride + k] = tr.leaf(v) ? v : -1;
                    }
                    continue;
                }
                if (select_levels) {
                    for (size_t s = 0; s < lay.slot.size(); ++s) {
                        const int32_t v = lay.slot[s];
                        const uint32_t thr = tr.leaf(v) ? 0u : km.word(tr.Th[v]);
                        const uint32_t meta = tr.leaf(v) ? 0u : (uint32_t)tr.Fe[v] << 22;
                        uint8_t *rec = blk + ((int64_t)s * bn.stride + k) * 8;
                        memcpy(rec, &thr, 4);
                        memcpy(rec + 4, &meta, 4);
                    }
                    for (size_t e = 0; e < lay.exits.size(); ++e) {
                        const int32_t v = lay.exits[e];
                        exits[(int64_t)e * bn.stride + k] = ref_of(tr, lay, v, tree_base[t]);
                        pexits[(int64_t)e * bn.stride + k] = tr.leaf(v) ? v : -1;
                    }
                    continue;
                }
                // exit index of each (node, side), in the order layout_tree made them
                size_t next_exit = 0;
                for (size_t i = 0; i < lay.head.size(); ++i) {
                    const int32_t v = lay.head[i];
                    uint32_t thr = 0u;
                    uint32_t meta, tgt[2];
                    if (tr.leaf(v)) {  // single-leaf tree
                        tgt[0] = tgt[1] = (uint32_t)bn.nranks;
                        meta = 0;
                    } else {
                        thr = km.word(tr.Th[v]);
                        meta = (uint32_t)tr.Fe[v] << 22;
                        const int32_t c2[2] = {tr.L[v], tr.R[v]};
                        for (int s2 = 0; s2 < 2; ++s2) {
                            const int32_t c = c2[s2];
                            tgt[s2] = (!tr.leaf(c) && lay.rank[c] >= 0) ? (uint32_t)lay.rank[c]
                                                                         : (uint32_t)(bn.nranks + next_exit++);
                        }
                    }
                    meta |= (tgt[1] << FP_TARGET_BITS) | tgt[0];
                    uint8_t *rec = blk + ((int64_t)i * bn.stride + k) * 8;
                    memcpy(rec, &thr, 4);
                    memcpy(rec + 4, &meta, 4);
                }
                for (size_t e = 0; e < lay.exits.size(); ++e) {
                    const int32_t v = lay.exits[e];
                    exits[(int64_t)e * bn.stride + k] = ref_of(tr, lay, v, tree_base[t]);
                    pexits[(int64_t)e * bn.stride + k] = tr.leaf(v) ? v : -1;
                }
            }
        }

        // ---- leaf values, one slot per leaf
        if (n_values) {
            float *vals = reinterpret_cast<float *>(img + h.off_values);
            for (int32_t t = 0; t < T; ++t) {
                const int64_t nb = desc->tree_node_begin[t];
                const TreeLayout &lay = lays[t];
                for (size_t v = 0; v < lay.leaf_rank.size(); ++v)
                    if (lay.leaf_rank[v] >= 0) vals[lay.value_base + lay.leaf_rank[v]] = desc->leaf_value[nb + v];
            }
        }

        // ---- super-nodes and their leaf-id side table
        FpSuper *deep = reinterpret_cast<FpSuper *>(img + h.off_deep);
        int32_t *dleaf = reinterpret_cast<int32_t *>(img + h.off_deep_leaf);
        for (int32_t t = 0; t < T; ++t) {
            const int64_t nb = desc->tree_node_begin[t];
            TreeRef tr{desc->left + nb, desc->right + nb, desc->feature + nb, desc->leaf_class + nb,
                       desc->threshold + nb, desc->cardinality ? desc->cardinality + nb : nullptr,
                       desc->tree_node_begin[t + 1] - nb};
            const TreeLayout &lay = lays[t];
            for (size_t i = 0; i < lay.sn_root.size(); ++i) {
                const int64_t g = tree_base[t] + (int64_t)i;
                if (three) {
                    float *vals = desc->leaf_value
                                      ? reinterpret_cast<float *>(img + h.off_values) + values3_base + 8 * g
                                      : nullptr;
                    const float *lv = desc->leaf_value ? desc->leaf_value + nb : nullptr;
                    uint32_t *keys = reinterpret_cast<uint32_t *>(img + h.off_deep_keys) + (fmt == 2 ? 8 : 4) * g;
                    if (fmt == 2)
                        encode_super3p(tr, lay, lay.sn_root[i], fb, cb, km, lv, deep[g], keys, dleaf + 8 * g, vals);
                    else
                        encode_super3(tr, lay, lay.sn_root[i], fb, cb, lv, deep[g], keys, dleaf + 8 * g, vals);
                } else {
                    encode_super(tr, lay, lay.sn_root[i], tree_base[t], deep[g], dleaf + 4 * g);
                }
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
    info->head_nodes = h->head_nodes;
    info->head_select = h->head_select;
    info->n_bins = h->n_bins;
    info->obs_tile = h->obs_tile;
    info->warps_per_cta = h->warps_per_cta;
    info->n_super = h->n_super;
    info->n_internal = h->n_internal;
    info->head_bytes = h->head_bytes_total;
    info->deep_bytes = (int64_t)sizeof(FpSuper) * h->n_super;
    info->total_bytes = h->class_bytes;
    info->parity_bytes = h->total_bytes - h->class_bytes;
    info->max_head_bytes = h->max_head_bytes;
    info->passes = h->n_passes;
    info->refill_lanes = h->refill_lanes;
    info->bin_buffers = h->bin_buffers;
    info->deep_levels = h->deep_levels;
    info->deep_format = h->deep_format;
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

// Node cardinalities from leaf counts (Section III-A: the statistics that
// order a tree's nodes may be measured on observations after training).  A
// leaf keeps its count; an internal node gets the sum of its two children,
// children before parents (an explicit post-order stack, so any node
// numbering works); nodes no path reaches get 0.  out_card may alias
// leaf_count.
extern "C" int fp_cardinality_from_leaf_counts(const fp_forest_desc *desc, const int64_t *leaf_count,
                                               int64_t *out_card) {
    if (!desc || !leaf_count || !out_card || !desc->tree_node_begin || !desc->left || !desc->right ||
        !desc->feature || !desc->leaf_class || desc->n_trees < 1 || desc->n_features < 1 || desc->n_classes < 1 ||
        desc->tree_node_begin[0] != 0) {
        fp_set_error("fp_cardinality_from_leaf_counts: bad arguments");
        return FP_EINVAL;
    }
    try {
        std::vector<uint8_t> seen;
        std::vector<std::pair<int32_t, bool>> stack;
        for (int32_t t = 0; t < desc->n_trees; ++t) {
            const int64_t b = desc->tree_node_begin[t], e = desc->tree_node_begin[t + 1];
            if (e < b) {
                fp_set_error("fp_cardinality_from_leaf_counts: tree_node_begin not monotone at tree %d", t);
                return FP_EINVAL;
            }
            TreeRef tr{desc->left + b, desc->right + b, desc->feature + b, desc->leaf_class + b, nullptr, nullptr,
                       e - b};
            int rc = validate_tree(tr, desc->n_features, desc->n_classes, t, seen);
            if (rc) return rc;
            const int64_t *cnt = leaf_count + b;
            int64_t *card = out_card + b;
            stack.assign(1, {0, false});
            while (!stack.empty()) {
                const auto [v, children_done] = stack.back();
                stack.pop_back();
                if (tr.leaf(v)) {
                    card[v] = cnt[v];
                } else if (children_done) {
                    card[v] = card[tr.L[v]] + card[tr.R[v]];
                } else {
                    stack.push_back({v, true});
                    stack.push_back({tr.R[v], false});
                    stack.push_back({tr.L[v], false});
                }
            }
            for (int64_t v = 0; v < tr.m; ++v)
                if (!seen[(size_t)v]) card[v] = 0;
        }
        return FP_OK;
    } catch (const std::bad_alloc &) {
        fp_set_error("fp_cardinality_from_leaf_counts: out of host memory");
        return FP_ENOMEM;
    }
}

// ------------------------------------------------- tree-bin sharding (F3)

// Section III binds bins of trees to processes.  A shard is a contiguous run
// of whole bins; the runs are cut so that each carries about the same
// expected work.  A tree's work is its expected number of internal nodes
// visited per observation -- the sum of its internal nodes' cardinalities over
// the root's (the training statistics of Section III-A) -- or, without
// cardinalities, its internal node count.
extern "C" int fp_shard_trees(const fp_forest_desc *desc, int32_t bin_size, int32_t n_shards, int32_t shard,
                              int32_t *tree_begin, int32_t *tree_end) {
    if (!desc || !desc->tree_node_begin || !desc->left || !tree_begin || !tree_end || desc->n_trees < 1 ||
        bin_size < 1 || n_shards < 1 || shard < 0 || shard >= n_shards || desc->tree_node_begin[0] != 0) {
        fp_set_error("fp_shard_trees: bad arguments");
        return FP_EINVAL;
    }
    const int32_t T = desc->n_trees;
    const int32_t n_bins = (T + bin_size - 1) / bin_size;
    try {
        std::vector<double> bin_work((size_t)n_bins, 0.0);
        for (int32_t t = 0; t < T; ++t) {
            const int64_t b = desc->tree_node_begin[t], e = desc->tree_node_begin[t + 1];
            if (e <= b) {
                fp_set_error("fp_shard_trees: tree %d has no nodes", t);
                return FP_EINVAL;
            }
            double w = 0.0;
            if (desc->cardinality && desc->cardinality[b] > 0) {
                for (int64_t v = b; v < e; ++v)
                    if (desc->left[v] >= 0) w += (double)desc->cardinality[v];
                w /= (double)desc->cardinality[b];
            } else {
                for (int64_t v = b; v < e; ++v) w += desc->left[v] >= 0 ? 1.0 : 0.0;
            }
            bin_work[(size_t)(t / bin_size)] += w;
        }
        // cut k sits at the bin boundary whose prefix of work is closest to k/n of the total
        std::vector<double> prefix((size_t)n_bins + 1, 0.0);
        for (int32_t b = 0; b < n_bins; ++b) prefix[(size_t)b + 1] = prefix[(size_t)b] + bin_work[(size_t)b];
        auto cut = [&](int32_t k) -> int32_t {
            if (k <= 0) return 0;
            if (k >= n_shards) return n_bins;
            const double target = prefix[(size_t)n_bins] * k / n_shards;
            int32_t best = 0;
            for (int32_t b = 1; b <= n_bins; ++b)
                if (std::abs(prefix[(size_t)b] - target) < std::abs(prefix[(size_t)best] - target)) best = b;
            return best;
        };
        // cuts never decrease: each is at or after the previous one
        int32_t lo = 0, hi = 0;
        for (int32_t k = 1; k <= shard + 1; ++k) {
            lo = hi;
            hi = std::max(lo, cut(k));
        }
        *tree_begin = std::min(T, lo * bin_size);
        *tree_end = std::min(T, hi * bin_size);
        return FP_OK;
    } catch (const std::bad_alloc &) {
        fp_set_error("fp_shard_trees: out of host memory");
        return FP_ENOMEM;
    }
}

// A shard's own image: the trees [tree_begin, tree_end) of desc as a forest of
// their own (tree-local node ids, so leaf ids are unchanged).
extern "C" int fp_pack_forest_trees(const fp_forest_desc *desc, const fp_pack_params *params, int32_t tree_begin,
                                    int32_t tree_end, fp_packed_forest **out) {
    if (!out || !desc || !desc->tree_node_begin || tree_begin < 0 || tree_end > desc->n_trees ||
        tree_begin >= tree_end) {
        if (out) *out = nullptr;
        fp_set_error("fp_pack_forest_trees: bad arguments (trees [%d, %d) of %d)", tree_begin, tree_end,
                     desc ? desc->n_trees : 0);
        return FP_EINVAL;
    }
    try {
        const int64_t base = desc->tree_node_begin[tree_begin];
        std::vector<int64_t> nb((size_t)(tree_end - tree_begin) + 1);
        for (int32_t t = tree_begin; t <= tree_end; ++t) nb[(size_t)(t - tree_begin)] = desc->tree_node_begin[t] - base;
        fp_forest_desc sub = *desc;
        sub.n_trees = tree_end - tree_begin;
        sub.tree_node_begin = nb.data();
        sub.left = desc->left ? desc->left + base : nullptr;
        sub.right = desc->right ? desc->right + base : nullptr;
        sub.feature = desc->feature ? desc->feature + base : nullptr;
        sub.threshold = desc->threshold ? desc->threshold + base : nullptr;
        sub.leaf_class = desc->leaf_class ? desc->leaf_class + base : nullptr;
        sub.cardinality = desc->cardinality ? desc->cardinality + base : nullptr;
        sub.leaf_value = desc->leaf_value ? desc->leaf_value + base : nullptr;
        return fp_pack_forest(&sub, params, out);
    } catch (const std::bad_alloc &) {
        *out = nullptr;
        fp_set_error("fp_pack_forest_trees: out of host memory");
        return FP_ENOMEM;
    }
}
