// fp_internal.h -- the packed image format shared by the host packer and the
// device code of the library (not part of the public C ABI).
//
// Image = one contiguous, 256-byte-aligned blob, uploaded verbatim:
//
//   FpImageHeader
//   FpBin    bins[n_bins]        bin b holds trees [first_tree, first_tree+width)
//   FpPass   passes[n_passes]    pass p sweeps bins [bin_begin, bin_end)
//   uint32   tree_base[T]        first deep record of each tree (index into deep)
//   heads                        per bin, 16-byte aligned, one block of
//                                  S*width head records (8 B), slot-major:
//                                    head[s*width + k] = BFS slot s of tree k
//                                  then L*width link entries (4 B), likewise
//                                    link[j*width + k] = slot S+j of tree k
//   deep     uint2 records       per tree, hot-first depth-first order
//   --- end of the classification part (class_bytes) ---
//   parity heads                 per bin, int32 leaf ids mirroring the head
//                                block (S*width, then L*width entries)
//   deep_leaf int2               per deep record: leaf id of the left / right
//                                child when that child is a leaf, else -1
//
// S = 2^(d+1) - 1 implicit breadth-first slots cover levels 0..d (children of
// slot s are 2s+1 and 2s+2); L = 2^(d+1) link entries cover level d+1.
//
// Head record {float thr; uint32 meta}:
//   meta bit 31 = 0: internal node, meta = feature
//   meta bit 31 = 1: leaf, meta & 0x7FFFFFFF = class (0x7FFFFFFF: empty slot)
// Link entry (uint32):
//   bit 31 = 1: leaf, low bits = class (0x7FFFFFFF: empty)
//   bit 31 = 0: tree-local index of the deep record of that node
// Deep record {float thr; uint32 meta}:
//   [31:22] feature
//   [21]    hot child is the right child (the hot child sits at index + 1)
//   [20]    cold child is a leaf: [18:0] = its class
//   [19]    both children are leaves: [8:0] left class, [17:9] right class
//   [18:0]  otherwise: tree-local index of the cold child's record
#pragma once
#include <stdint.h>

#define FP_IMAGE_MAGIC 0x4B435046u /* "FPCK" */
#define FP_IMAGE_VERSION 1u

#define FP_META_FEATURE_SHIFT 22
#define FP_META_HOT_RIGHT (1u << 21)
#define FP_META_COLD_LEAF (1u << 20)
#define FP_META_BOTH_LEAF (1u << 19)
#define FP_META_PAYLOAD_MASK 0x7FFFFu
#define FP_MAX_DEEP_PER_TREE (1 << 19)
#define FP_MAX_FEATURES 1024
#define FP_MAX_CLASSES 512
#define FP_HEAD_LEAF 0x80000000u
#define FP_HEAD_EMPTY 0xFFFFFFFFu
#define FP_MAX_DEPTH 9

struct FpBin {
    uint32_t head_off;    // bytes from the start of the heads section
    uint32_t head_bytes;  // head records + link entries, padded to 16 B
    int32_t first_tree;
    int32_t width;
    uint32_t phead_off;   // bytes from the start of the parity-heads section
    uint32_t pad[3];
};

struct FpPass {
    int32_t bin_begin, bin_end;
};

struct FpImageHeader {
    uint32_t magic, version;
    int32_t n_trees, n_features, n_classes;
    int32_t bin_size, depth, n_bins, n_passes;
    int32_t slots, links;          // S and L
    int32_t obs_tile, warps_per_cta;
    int32_t max_head_bytes;
    int64_t n_deep;
    int64_t off_bins, off_passes, off_tree_base, off_heads, off_deep;
    int64_t off_pheads, off_deep_leaf;
    int64_t class_bytes;           // end of the classification part
    int64_t total_bytes;           // end of the image (incl. parity tables)
    int64_t head_bytes_total, pass_bytes;
};
