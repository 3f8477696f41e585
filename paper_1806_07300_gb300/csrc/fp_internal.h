// fp_internal.h -- the packed image format shared by the host packer and the
// device code of the library (not part of the public C ABI).
//
// Image = one contiguous blob, sections 256-byte aligned, uploaded verbatim:
//
//   FpImageHeader
//   FpBin    bins[n_bins]        bin b holds trees [first_tree, first_tree+width)
//   FpPass   passes[n_passes]    pass p sweeps bins [bin_begin, bin_end)
//   uint32   tree_base[T]        first super-node of each tree (index into deep)
//   blocks                       per bin, 16-byte aligned, the interleaved block
//                                of the bin's trees (stride = width | 1, odd):
//                                  nranks*stride head nodes (8 B), rank-major:
//                                    node[rank*stride + k] = rank-th head node of tree k
//                                  nexits*stride exit references (4 B):
//                                    exit[e*stride + k]   = e-th exit of tree k
//   deep     FpSuper[]           per tree, its super-nodes in Stat order; the
//                                trees' regions follow one another
//   deep_keys uint32[4] or [8] per super-node (three-level super-nodes
//                                only): the full keys of its last level (slots
//                                3..6; format 1) or of all seven slots and a
//                                zero (format 2)
//   values   float[n_values]     forests with leaf values (see below)
//   --- end of the classification part (class_bytes) ---
//   parity blocks                per bin, int32 leaf id of each exit (or -1),
//                                [nexits][stride] like the exits
//   deep_leaf int32[4] (two-level) or [8] (three-level) per super-node: leaf
//                                id behind each exit, or -1
//
// In a forest with three-level super-nodes every threshold is stored as an
// order key; otherwise thresholds are float bits.  key(v) maps a float to a
// uint32 that orders like the float: +0 for -0, then the sign bit flipped for
// v >= 0 and every bit flipped for v < 0; a NaN observation value maps to
// 0xFFFFFFFF and a NaN threshold to 0.  For every observation value x and
// threshold t, x <= t (go left) exactly when key(x) <= key(t) -- a NaN x or t
// goes right, as the float compare does -- so the kernel converts the rows
// once when it stages them and every compare is an unsigned integer compare.
//
// Super-nodes of format 2 (below) compare remapped keys, which spread the
// forest's own thresholds over the word.  First the widest run of keys that
// holds no threshold key, between adjacent threshold keys ta < tb, is
// collapsed to the single key ta + 1:
//   g(k) = k - (tb - ta - 2)   for k >= tb,     g(k) = min(k, ta + 1) below
// (key_gap_a = ta + 1, key_gap_b = tb, key_gap_d = tb - ta - 2; with no such
// run, 0xFFFFFFFF, 0xFFFFFFFF and 0).  Then, with lo the smallest and top the
// largest threshold key, hi = g(top) + 1 and b = the bit length of hi - lo,
// when b <= 31
//   V(k) = 0x80000000 | ((min(max(g(k), lo), hi) - lo) << (31 - b))
// (key_lo = lo, key_hi = hi, key_shl = 31 - b, key_flag = 0x80000000), else
// V(k) = g(k) (key_lo = 0, key_hi = 0xFFFFFFFF, key_shl = key_flag = 0).  g
// is monotone, one-to-one on the threshold keys, and puts every key inside
// the run strictly between g(ta) and g(tb); the clamp keeps keys below lo
// (above top) below (above) every threshold; the shift is one-to-one.  So x
// <= t exactly when V(key(x)) <= V(key(t)).  A NaN threshold and a dummy slot
// store 0, below every V(key(x)) (remapped, every row value has the top bit
// set), so every x goes right of them.  Rows are staged as V(key(x)) and
// every stored threshold, in the heads too, is V(key(t)).  Short prefixes of
// V distinguish the forest's thresholds far better than prefixes of the key,
// whose top bits spend themselves on the sign and on exponents that no
// threshold of the forest uses (for data of both signs, the run around zero
// between the smallest negative and positive thresholds).
//
// Three kinds of head (the header's head_select, the same for every bin; 1
// and 2 are the level heads, 3 the ranked one):
//
// head_select = 1, levels (the Bin layout of Section III-A): levels 0..d of
// every tree in implicit breadth-first slots, nranks = 2^(d+1) - 1 and
// nexits = 2^(d+1) for every bin.  Slot s has children 2s+1 (left) and 2s+2
// (right); slot nranks + e is exit e.  A leaf above level d+1 fills its slot
// with a dummy node and every exit below it names the leaf, so whichever way
// the dummy compares go the walk ends on that leaf; every walk takes exactly
// d+1 steps.  Head node {float thr; uint32 meta}, meta[31:22] = feature, the
// rest zero.  d <= FP_MAX_LEVEL_DEPTH.
//
// head_select = 2, paired levels: the same levels, slots and exits, stored two
// levels per 16-byte record (d odd): record q of super-level j holds the node
// at level 2j, position p = q - (4^j - 1)/3, and its two children --
// {thr, thr of left child, thr of right child, features [9:0] node,
// [19:10] left child, [29:20] right child} -- and its successors are the
// records 4q+1 .. 4q+4; nranks = (4^J - 1)/3 records for J = (d+1)/2, and
// record index nranks + e is exit e.
//
// head_select = 3, ranked: the K = 2^(d+1) - 1 internal nodes of highest
// training cardinality (ties: shallower, then earlier), a subtree that
// contains the root; for a complete tree these are exactly levels 0..d.
// They are ranked in depth-first order that visits the more frequently
// reached child first.  Head node {float thr; uint32 meta}:
//   [31:22] feature
//   [21:11] right target, [10:0] left target: a target below the bin's
//           nranks is the rank of a head node, otherwise it names
//           exit[target - nranks]
// A tree whose root is a leaf gets one head node whose two targets both name
// an exit holding that leaf.  nranks + nexits <= 2048 (so d <= 9).
//
// A reference (exit entry or super-node exit) is a uint32:
//   bit 31 = 1: a leaf, bits 30..0 = its class (classification forests) or
//               its slot in values[] (forests with leaf values)
//   bit 31 = 0: a super-node, the index into deep[] (so fewer than 2^31)
//
// Forests with leaf values also hold values[n_values] (float) at off_values,
// inside the classification part of the image: one slot per leaf, numbered
// tree by tree in node order, and with three-level super-nodes, from
// values3_base on, eight more per super-node (the value behind each exit).
//
// Super-nodes come in two kinds (the header's deep_levels), 32 bytes each
// (one L2 sector, 32-byte aligned, one load); three-level ones in two formats
// (the header's deep_format):
//
// deep_levels = 2: a node v below the head together with its two children,
// i.e. two levels of the tree resolved by one load:
//   w[0] threshold of v (float)    w[1] threshold of v's left child
//   w[2] threshold of v's right child
//   w[3] features: v [9:0], left child [19:10], right child [29:20]
//   w[4..7] exits: (left,left) (left,right) (right,left) (right,right)
// A child that is a leaf keeps a dummy split and both of its exits name the
// leaf, so either outcome of the dummy compare lands on it.
//
// deep_levels = 3: a node v and the two levels below it -- seven nodes in
// implicit slots (slot i has children 2i+1, 2i+2; a leaf is carried down as
// dummies, like the level heads) and eight exits (exit e is child e & 1 of
// slot 3 + (e >> 1)) -- three levels per load.  With fb = feature_bits and
// cb = class_bits, format 1 (deep_format = 1, 2fb + 2cb <= 24):
//   w[0..2] the full keys of slots 0..2
//   w[3..6] slots 3..6: [fb-1:0] feature, [2fb-1:fb] the feature of slot
//           0, 1, 2 (in w[3], w[4], w[5]; zero in w[6]), [2fb+2cb-1:2fb+cb]
//           class of the right exit and [2fb+cb-1:2fb] of the left one (a
//           leaf exit's class; 0 otherwise), [31:2fb+2cb] the top bits of
//           the slot's key
//   w[7]    [31:24] leaf mask (bit e set: exit e is a leaf),
//           [23:0]  offset from this super-node to the first of its children:
//           the super-nodes rooted at its internal exits are consecutive, in
//           exit order, so exit e continues at this + offset + (number of
//           internal exits before e)
// The first two levels compare full keys; the last compares the key of x
// with a key prefix, and when the prefixes are equal it decides with the full
// key from deep_keys (a 4-byte load, for a small fraction of compares).  A
// dummy slot has key 0 (every observation goes right of it, never a tie).
//
// Format 2 (deep_format = 2, fb + 2cb <= 24): every slot compares a prefix of
// its remapped key V(t), and the feature sits beside it:
//   w[0..2] slots 0..2: [fb-1:0] feature, [31:fb] the top 32 - fb bits of V
//   w[3..6] slots 3..6: [fb-1:0] feature, [fb+cb-1:fb] class of the left exit,
//           [fb+2cb-1:fb+cb] of the right one, [31:fb+2cb] the top bits of V
//   w[7]    as in format 1
// A staged V(key(x)) compared with the whole word decides the split wherever
// its top bits differ from the slot's prefix; where they are equal (rare: the
// forest's thresholds are spread over the prefix range) the slot's full V
// from deep_keys decides.  Dummy slots and NaN thresholds store V = 0, whose
// top bit never equals a remapped row value's.
//
// In a forest with leaf values exit e of super-node g names the value slot
// values3_base + 8g + e.
#pragma once
#include <stdint.h>

#define FP_IMAGE_MAGIC 0x4B435046u /* "FPCK" */
#define FP_IMAGE_VERSION 7u

#define FP_MAX_FEATURES 1024
#define FP_MAX_CLASSES 512
#define FP_REF_LEAF 0x80000000u
#define FP_MAX_DEPTH 9         // ranked heads
#define FP_MAX_LEVEL_DEPTH 11  // level heads
#define FP_TARGET_BITS 11
#define FP_TARGET_MASK 2047u
#define FP_DEEP3_OFFSET_MASK 0xFFFFFFu  // three-level super-nodes: child offset field

struct FpSuper {
    uint32_t w[8];
};

struct FpBin {
    uint32_t head_off;    // bytes from the start of the blocks section
    uint32_t head_bytes;  // head nodes + exits, padded to 16 B
    int32_t first_tree;
    int32_t width;
    uint32_t phead_off;   // bytes from the start of the parity-blocks section
    int32_t stride;       // width | 1
    int32_t nranks;       // head node rows
    int32_t nexits;       // exit rows
};

struct FpPass {
    int32_t bin_begin, bin_end;
};

struct FpImageHeader {
    uint32_t magic, version;
    int32_t n_trees, n_features, n_classes;
    int32_t bin_size, depth, n_bins, n_passes;
    int32_t head_nodes;            // K, head nodes per tree at most
    int32_t head_select;           // 1: levels 0..d in implicit slots, 2: paired slots, 3: ranked
    int32_t obs_tile, warps_per_cta;
    int32_t max_head_bytes;
    int32_t refill_lanes;
    int32_t bin_buffers;           // shared-memory buffers of the bin-block pipeline (2 or 3)
    int64_t n_super;               // super-nodes in the deep section
    int64_t off_bins, off_passes, off_tree_base, off_heads, off_deep;
    int64_t off_pheads, off_deep_leaf;
    int64_t class_bytes;           // end of the classification part
    int64_t total_bytes;           // end of the image (incl. parity tables)
    int64_t head_bytes_total, pass_bytes;
    int64_t n_internal;            // internal nodes of the forest
    int64_t n_values, off_values;  // leaf-value slots (0 for a classification forest)
    int32_t deep_levels;           // 2 or 3 tree levels per super-node
    int32_t feature_bits, class_bits;  // three-level super-nodes: field widths fb, cb
    int32_t deep_format;           // three-level super-nodes: 1 full keys in slots 0..2, 2 prefixes in all
    int64_t off_deep_keys;         // three-level super-nodes: full keys, 4 (format 1) or 8 per super-node
    int64_t values3_base;          // forests with leaf values: first slot of the per-exit values
    uint32_t key_lo, key_hi;       // format 2: the key remap V (above); identity: 0, 0xFFFFFFFF
    uint32_t key_shl, key_flag;
    uint32_t key_gap_a, key_gap_b;  // format 2: the collapsed run of keys (none: 0xFFFFFFFF twice)
    uint32_t key_gap_d, reserved1;
};
