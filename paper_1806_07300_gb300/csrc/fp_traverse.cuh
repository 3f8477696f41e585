// fp_traverse.cuh -- the packed-forest traversal kernel (sm_103a).
//
// One work item = (pass, observation tile).  Items are ordered pass-major, so
// at any moment the GPU walks the bins of one pass, whose super-nodes stay
// resident in L2 while every tile of observations goes through them (the GPU
// counterpart of the paper's bins bound to cores, Section III).  For an item
// the CTA:
//   1. stages the tile's rows into shared memory feature-major
//      (x[f * R + r]), so 32 lanes holding 32 consecutive rows read any
//      features from 32 different banks (16-byte loads along a row when the
//      feature count is a multiple of 4, else 4-byte cp.async); for a forest
//      with three-level super-nodes each value is turned into its order key
//      (fp_internal.h) and every compare is an unsigned integer compare,
//      otherwise values and compares stay float;
//   2. streams the bins' interleaved blocks (the heads of their trees,
//      Section III-A Bin) through nbuf (2 or 3) shared-memory buffers with TMA bulk
//      copies (cp.async.bulk) completing on mbarriers: a warp waits only for
//      the block of the bin it is about to claim, and the last warp to finish
//      claiming a bin refills that buffer with the bin nbuf places ahead;
//   3. walks (observation, tree) tasks in two kinds of warp steps:
//        burst -- the warp claims 32 consecutive tasks (32 rows of one tree)
//                 and all lanes walk their paths through the tree's head in
//                 shared memory together, with a branch-free step (level
//                 heads: exactly d+1 steps over implicit slots, or (d+1)/2
//                 steps of two levels when the slots are paired; ranked
//                 heads: until the last lane leaves the head); paths that leave the
//                 head are pushed, compacted with __ballot_sync / __popc,
//                 into the warp's ring of pending tasks;
//        deep  -- every lane holding a task resolves two or three more levels
//                 with one 32-byte super-node load (one L2 sector); a lane
//                 that reaches a leaf votes and takes the next pending task
//                 from the ring.
//      Bursts keep the ring topped up, so lanes stay busy while paths of very
//      different depth diverge -- the GPU form of the paper's round-robin over
//      independent tasks (Section III-B).  Pending and running tasks carry
//      over from one bin to the next, and nothing but the item's end makes a
//      warp wait for another;
//   4. counts votes per (row, class) with shared-memory atomics;
//   5. writes votes and the argmax class (lowest class on ties).  With one
//      pass the tile's votes are complete in shared memory; with several, they
//      are added to a global accumulator and the CTA that finishes a tile's
//      last pass (per-tile counter, no waiting) takes the argmax.
// Parity mode writes the leaf id reached in every (observation, tree)
// instead of voting.  Values mode (forests with real leaf values: regression
// and boosted trees) adds the leaf's value to a float per row instead, and
// writes bias + scale * sum (several passes: summed in global memory, the
// last pass's CTA writes it).
//
// Waits: cp.async.wait_group and __syncthreads are hardware waits; a wait for
// a bin block polls its mbarrier at most spin_limit times (FP_SPIN_LIMIT
// unless a test lowers it), then records FP_ETIMEOUT in the status word and
// makes every warp skip the rest of its work; before exiting, the CTA waits
// (bounded by FP_SPIN_LIMIT polls) for its own bulk copies to land.  A test
// can set `stall` so that bin waits ignore completed copies and run out; the
// copies themselves still complete, so the exit path stays clean.  Every walk
// is bounded too.
#pragma once
#include <stdint.h>

#include "fp_internal.h"

struct TravParams {
    const FpSuper *deep;      // super-nodes
    const uint8_t *heads;     // interleaved blocks
    const FpBin *bins;
    const FpPass *passes;
    const int32_t *pheads;    // parity: leaf id per block exit
    const int32_t *deep_leaf; // parity: 4 leaf ids per super-node
    const float *X;
    int64_t n;
    int64_t n_tiles;
    int64_t n_items;
    int32_t F, C, T, R;
    int32_t n_passes;
    int32_t head_smem;        // bytes reserved for one bin block
    int32_t nbuf;             // bin-block buffers (2 or 3)
    int32_t levels;           // head kind: 0 ranked, 1 level slots (depth+1 steps), 2 paired level slots
    int32_t depth;            // d of the interleaved head
    int32_t refill;           // bursts start when the ring holds at most this many tasks
    uint32_t *out_votes;      // single pass: final votes (may be NULL)
    int32_t *out_class;       // may be NULL
    int32_t *out_leaf;        // parity mode
    uint32_t *acc;            // several passes: vote accumulator
    uint32_t *tile_done;      // several passes: per-tile pass counter
    int32_t *status;          // device status word
    const float *leaf_val;    // forests with leaf values: value of each leaf slot
    uint32_t n_vals;          // slots in leaf_val
    float vscale, vbias;      // out = vbias + vscale * sum of leaf values
    float *out_val;           // values mode: output per row
    float *acc_val;           // values mode, several passes: per-row accumulator
    int32_t spin_limit;       // polls of a bin block's barrier before the wait gives up
    int32_t stall;            // fault injection: bin waits ignore completed copies (0 normally)
    int32_t deep_kind;        // super-nodes: 2 two levels, 3 three levels (format 1), 4 three levels (format 2)
    uint32_t fbits, sh2;      // three levels: feature bits; key-prefix shift of the last level
                              // (2fb + 2cb in format 1, fb + 2cb in format 2)
    uint32_t cbits, fmask, cmask;  // three levels: class bits, feature and class masks
    uint32_t vbase3;          // three levels, values mode: first per-exit value slot
    const uint32_t *deep_keys;  // three levels: full keys, 4 (format 1) or 8 (format 2) per super-node
    uint32_t klo, khi, kshl, kflag;  // format 2: the key remap V of the staged rows
    uint32_t kga, kgb, kgd;          // format 2: its collapsed run of keys
    int64_t n_super;
};

// What a kernel computes per (row, tree) task it finishes.
#define FP_MODE_VOTES 0   // a vote for the leaf's class; then votes and the argmax class
#define FP_MODE_LEAVES 1  // the leaf id (parity mode)
#define FP_MODE_VALUES 2  // the leaf's value, summed per row; then bias + scale * sum

#define FP_ERR_FLAG_DEVICE (-6)
#define FP_ERR_FLAG_TIMEOUT (-5)
#define FP_NBUF 3             // bin-block buffers at most (a launch uses nbuf = 2 or 3)
#define FP_SPIN_LIMIT (1 << 24)
#define FP_RING 64            // pending tasks per warp
#define FP_NO_CLASS (FP_REF_LEAF | 0x7FFFFFFFu)

__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// One super-node: a single 256-bit load (32-byte aligned, one L2 sector).
// The lines are not allocated in L1: few super-nodes are read twice by one
// SM before eviction, and with most of the unified L1/shared array given to
// shared memory, allocating a line per lane for thousands of loads in
// flight throttles the load path (measured: twice the run time once shared
// memory takes more than about 196 KB).  The memory clobber keeps the load
// where it is written, ahead of the work meant to overlap its latency.
__device__ __forceinline__ void ld_super(const FpSuper *p, uint32_t w[8]) {
    asm volatile("ld.global.nc.L1::no_allocate.v8.u32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
                 : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7])
                 : "l"(p)
                 : "memory");
}

__device__ __forceinline__ void report(int32_t *status, int32_t code) { atomicCAS(status, 0, code); }

// The order key of an observation value (fp_internal.h): compares like the
// float against threshold keys; NaN goes above every threshold (right).
__device__ __forceinline__ uint32_t obs_key(float v) {
    uint32_t u = __float_as_uint(v);
    if ((u & 0x7FFFFFFFu) > 0x7F800000u) return 0xFFFFFFFFu;
    if (u == 0x80000000u) u = 0u;
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// The remapped key V of format 2 (fp_internal.h): the run of keys without a
// threshold collapsed, then clamped to the forest's threshold range and
// spread over the 31 bits below a set top bit.
__device__ __forceinline__ uint32_t remap_key(const TravParams &p, uint32_t k) {
    const uint32_t g = k >= p.kgb ? k - p.kgd : min(k, p.kga);
    return p.kflag | ((min(max(g, p.klo), p.khi) - p.klo) << p.kshl);
}

// A staged observation value for super-node kind DK: its float bits (2), its
// order key (3) or its remapped key (4).
template <int DK>
__device__ __forceinline__ uint32_t staged(const TravParams &p, float v) {
    return DK == 2 ? __float_as_uint(v) : (DK == 3 ? obs_key(v) : remap_key(p, obs_key(v)));
}

// x <= t, the split's test (go left): keys compare as unsigned integers,
// otherwise as floats (a NaN x or t goes right either way).
template <bool KEYS>
__device__ __forceinline__ bool goes_left(uint32_t x, uint32_t t) {
    return KEYS ? x <= t : __uint_as_float(x) <= __uint_as_float(t);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// true once the phase of the given parity has completed
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// One thread: copy a bin's block into a buffer with the bulk-copy engine.
__device__ __forceinline__ void stage_block_bulk(const TravParams &p, int b, uint8_t *dst, uint64_t *bar) {
    const FpBin bn = p.bins[b];
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // earlier reads of dst come first
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
                 "r"(bn.head_bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            smem_u32(dst)),
        "l"(p.heads + bn.head_off), "r"(bn.head_bytes), "r"(smem_u32(bar))
        : "memory");
}

// Per-lane state of a running task.
struct LaneTask {
    bool active;
    int r;            // row within the tile
    int t;            // tree
    uint32_t ref;     // current super-node (index into deep)
};

// A finished task: vote, record the leaf id (parity mode) or add the leaf's
// value to the row's sum (cls is then the leaf's value slot).
template <int MODE>
__device__ __forceinline__ void finish(const TravParams &p, uint32_t *svotes, int64_t row0, int r, int t,
                                       uint32_t cls, int32_t leaf_id) {
    if (MODE == FP_MODE_LEAVES) {
        p.out_leaf[(row0 + r) * p.T + t] = leaf_id;
    } else if (MODE == FP_MODE_VALUES) {
        if (cls < p.n_vals)
            atomicAdd(reinterpret_cast<float *>(svotes) + r, __ldg(p.leaf_val + cls));
        else
            report(p.status, FP_ERR_FLAG_DEVICE);
    } else if (cls < (uint32_t)p.C) {
        atomicAdd(&svotes[cls * p.R + r], 1u);  // class-major: a burst's 32 rows hit 32 banks
    } else {
        report(p.status, FP_ERR_FLAG_DEVICE);
    }
}

// Lanes without a task take pending ones from the warp's ring.
__device__ __forceinline__ void pop_tasks(const TravParams &p, const uint2 *ring, int &head, int tail, LaneTask &L,
                                          unsigned lt_mask) {
    const unsigned idle = __ballot_sync(0xffffffffu, !L.active);
    const int npop = min(__popc(idle), tail - head);
    if (npop <= 0) return;
    const int rk = __popc(idle & lt_mask);
    if (!L.active && rk < npop) {
        const uint2 ent = ring[(head + rk) & (FP_RING - 1)];
        L.ref = ent.x;
        L.r = (int)(ent.y & 2047u);
        L.t = (int)(ent.y >> 11);
        L.active = true;
    }
    head += npop;
}

// One deep step, two or three levels of the tree per 32-byte load, in two
// halves: the load is issued first and consumed after the warp has done other
// work (a head burst), so the L2 latency overlaps that work.
__device__ __forceinline__ void deep_issue(const TravParams &p, const LaneTask &L, uint32_t w[8]) {
    ld_super(p.deep + L.ref, w);
}

// Three levels: full keys for the first two, and a key prefix for the last,
// whose tie (rare) is decided by the slot's full key from the side table.
template <int MODE>
__device__ __forceinline__ void deep_finish3(const TravParams &p, const uint32_t *xs, uint32_t *svotes, int64_t row0,
                                             LaneTask &L, const uint32_t w[8]) {
    const uint32_t *xr = xs + L.r;
    const int R = p.R;
    const uint32_t fm = p.fmask, fb = p.fbits, s2 = p.sh2;
    const uint32_t k0 = xr[((w[3] >> fb) & fm) * R];
    const uint32_t d0 = k0 > w[0] ? 1u : 0u;
    const uint32_t n1 = d0 ? w[2] : w[1];
    const uint32_t k1 = xr[(((d0 ? w[5] : w[4]) >> fb) & fm) * R];
    const uint32_t d1 = k1 > n1 ? 1u : 0u;
    const uint32_t j = 2 * d0 + d1;  // last-level slot 3 + j
    const uint32_t n2 = d0 ? (d1 ? w[6] : w[5]) : (d1 ? w[4] : w[3]);
    const uint32_t k2 = xr[(n2 & fm) * R];
    uint32_t d2 = (k2 >> s2) > (n2 >> s2) ? 1u : 0u;
    if ((k2 >> s2) == (n2 >> s2)) d2 = k2 > __ldg(p.deep_keys + 4 * (int64_t)L.ref + j) ? 1u : 0u;
    const uint32_t e = 2 * j + d2;
    const uint32_t mask = w[7] >> 24;
    if ((mask >> e) & 1u) {
        L.active = false;
        int32_t leaf_id = -1;
        if (MODE == FP_MODE_LEAVES) leaf_id = p.deep_leaf[8 * (int64_t)L.ref + e];
        const uint32_t cls =
            MODE == FP_MODE_VALUES ? p.vbase3 + 8 * L.ref + e : (n2 >> (2 * fb + p.cbits * d2)) & p.cmask;
        finish<MODE>(p, svotes, row0, L.r, L.t, cls, leaf_id);
    } else {
        // children sit side by side from the offset on, in exit order
        const uint32_t nref = L.ref + (w[7] & FP_DEEP3_OFFSET_MASK) + __popc(~mask & ((1u << e) - 1u));
        if (nref > L.ref && (int64_t)nref < p.n_super) {  // forward only, so every walk ends
            L.ref = nref;
        } else {
            report(p.status, FP_ERR_FLAG_DEVICE);
            L.active = false;
        }
    }
}

// Three levels, format 2: every slot's word is the top bits of its remapped
// key over its feature (and classes), so comparing the staged V with the
// whole word decides the split wherever their top bits differ.  Where they
// are equal for any of the three slots of the walk (rare), the step is taken
// again with the slots' full keys from the side table.
template <int MODE>
__device__ __forceinline__ void deep_finish3p(const TravParams &p, const uint32_t *xs, uint32_t *svotes,
                                              int64_t row0, LaneTask &L, const uint32_t w[8]) {
    const uint32_t *xr = xs + L.r;
    const int R = p.R;
    const uint32_t fm = p.fmask, fb = p.fbits, s2 = p.sh2;
    const uint32_t k0 = xr[(w[0] & fm) * R];
    uint32_t d0 = k0 > w[0] ? 1u : 0u;
    uint32_t n1 = d0 ? w[2] : w[1];
    const uint32_t k1 = xr[(n1 & fm) * R];
    uint32_t d1 = k1 > n1 ? 1u : 0u;
    uint32_t j = 2 * d0 + d1;  // last-level slot 3 + j
    uint32_t n2 = d0 ? (d1 ? w[6] : w[5]) : (d1 ? w[4] : w[3]);
    uint32_t k2 = xr[(n2 & fm) * R];
    uint32_t d2 = k2 > n2 ? 1u : 0u;
    if ((min(k0 ^ w[0], k1 ^ n1) >> fb) == 0u || ((k2 ^ n2) >> s2) == 0u) {
        const uint32_t *fk = p.deep_keys + 8 * (int64_t)L.ref;
        d0 = k0 > __ldg(fk) ? 1u : 0u;
        n1 = d0 ? w[2] : w[1];
        d1 = xr[(n1 & fm) * R] > __ldg(fk + 1 + d0) ? 1u : 0u;
        j = 2 * d0 + d1;
        n2 = d0 ? (d1 ? w[6] : w[5]) : (d1 ? w[4] : w[3]);
        k2 = xr[(n2 & fm) * R];
        d2 = k2 > __ldg(fk + 3 + j) ? 1u : 0u;
    }
    const uint32_t e = 2 * j + d2;
    const uint32_t mask = w[7] >> 24;
    if ((mask >> e) & 1u) {
        L.active = false;
        int32_t leaf_id = -1;
        if (MODE == FP_MODE_LEAVES) leaf_id = p.deep_leaf[8 * (int64_t)L.ref + e];
        const uint32_t cls =
            MODE == FP_MODE_VALUES ? p.vbase3 + 8 * L.ref + e : (n2 >> (fb + p.cbits * d2)) & p.cmask;
        finish<MODE>(p, svotes, row0, L.r, L.t, cls, leaf_id);
    } else {
        const uint32_t nref = L.ref + (w[7] & FP_DEEP3_OFFSET_MASK) + __popc(~mask & ((1u << e) - 1u));
        if (nref > L.ref && (int64_t)nref < p.n_super) {  // forward only, so every walk ends
            L.ref = nref;
        } else {
            report(p.status, FP_ERR_FLAG_DEVICE);
            L.active = false;
        }
    }
}

// DK: the forest's kind of super-node (p.deep_kind: 2, 3 or 4); a
// compile-time choice, so no kind's step carries another's code.
template <int MODE, int DK>
__device__ __forceinline__ void deep_finish(const TravParams &p, const uint32_t *xs, uint32_t *svotes, int64_t row0,
                                            LaneTask &L, const uint32_t w[8]) {
    if (DK == 3) {
        deep_finish3<MODE>(p, xs, svotes, row0, L, w);
        return;
    }
    if (DK == 4) {
        deep_finish3p<MODE>(p, xs, svotes, row0, L, w);
        return;
    }
    const int R = p.R;
    const uint32_t x0 = xs[(w[3] & 1023u) * R + L.r];
    const uint32_t d0 = goes_left<false>(x0, w[0]) ? 0u : 1u;
    const uint32_t f1 = d0 ? (w[3] >> 20) & 1023u : (w[3] >> 10) & 1023u;
    const uint32_t t1 = d0 ? w[2] : w[1];
    const uint32_t x1 = xs[f1 * R + L.r];
    const uint32_t d1 = goes_left<false>(x1, t1) ? 0u : 1u;
    const uint32_t nref = d0 ? (d1 ? w[7] : w[6]) : (d1 ? w[5] : w[4]);
    if (nref & FP_REF_LEAF) {
        L.active = false;
        int32_t leaf_id = -1;
        if (MODE == FP_MODE_LEAVES) leaf_id = p.deep_leaf[4 * (int64_t)L.ref + 2 * d0 + d1];
        finish<MODE>(p, svotes, row0, L.r, L.t, nref & 0x7FFFFFFFu, leaf_id);
    } else if (nref > L.ref && (int64_t)nref < p.n_super) {  // forward only, so every walk ends
        L.ref = nref;
    } else {
        report(p.status, FP_ERR_FLAG_DEVICE);
        L.active = false;
    }
}

// CTA-wide state shared by the items a CTA runs.
struct CtaShared {
    uint64_t full[FP_NBUF];   // block staged (bulk copy done)
    int task_next[FP_NBUF];   // next unclaimed task of the buffer's bin
    int claim_done[FP_NBUF];  // warps done claiming the buffer's bin
    int issued[FP_NBUF];      // bulk copies issued into the buffer
    int use0[FP_NBUF];        // issued[] when the current item started
    int last;
    int abort;
    long long next_item;
};

__device__ __forceinline__ void cta_init(CtaShared &sh) {
    if (threadIdx.x == 0) {
        for (int i = 0; i < FP_NBUF; ++i) {
            mbar_init(&sh.full[i], 1);
            sh.issued[i] = 0;
        }
        sh.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    }
    __syncthreads();
}

// After an abort, let this CTA's bulk copies land before it exits (bounded).
__device__ __forceinline__ void cta_finish(CtaShared &sh) {
    if (threadIdx.x == 0 && sh.abort) {
        for (int i = 0; i < FP_NBUF; ++i) {
            if (sh.issued[i] == 0) continue;
            const uint32_t parity = (uint32_t)(sh.issued[i] - 1) & 1u;
            for (int spin = 0; spin < FP_SPIN_LIMIT && !mbar_try_wait(&sh.full[i], parity); ++spin) {
            }
        }
    }
}

// One work item (pass, observation tile) of one forest.  Bin bi of the item
// goes through buffer bi % nbuf; the k-th copy ever issued into a buffer
// completes its barrier's phase k, so a wait needs the buffer's copy count
// at the item's start (use0) plus bi / nbuf.  Counting per buffer keeps the
// phases right when items of forests with different nbuf share a CTA.
// HK: the head kind when known at compile time (0 ranked, 1 level slots,
// 2 paired level slots), or -1 to read it from p.levels (the batched kernel,
// whose forests may differ).
template <int MODE, int DK, int HK>
__device__ __forceinline__ void run_item(const TravParams &p, int64_t item, uint8_t *smem, CtaShared &sh) {
    constexpr bool D3 = DK >= 3;  // rows and thresholds are (remapped) order keys
    constexpr bool LEAVES = MODE == FP_MODE_LEAVES, VALUES = MODE == FP_MODE_VALUES;
    const int levels = HK >= 0 ? HK : p.levels;
    const int R = p.R, F = p.F, C = p.C;
    uint32_t *xs = reinterpret_cast<uint32_t *>(smem);  // the tile's rows: (remapped) order keys or float bits
    const int xs_bytes = ((F * R * 4) + 15) & ~15;
    const int nbuf = p.nbuf;
    uint8_t *const hbuf0 = smem + xs_bytes;  // nbuf bin-block buffers, head_smem bytes each
    uint32_t *svotes = reinterpret_cast<uint32_t *>(smem + xs_bytes + nbuf * p.head_smem);
    const int CS = VALUES ? 1 : C;  // counters per row: class votes, or one float sum
    const int vote_bytes = LEAVES ? 0 : ((R * CS * 4) + 15) & ~15;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    uint2 *ring = reinterpret_cast<uint2 *>(smem + xs_bytes + nbuf * p.head_smem + vote_bytes) + warp * FP_RING;
    const unsigned lt_mask = (1u << lane) - 1u;

    // one thread: stage bin b of the pass, the item's bi-th bin
    auto issue = [&](int b, int bi) {
        const int buf = bi % nbuf;
        sh.task_next[buf] = 0;
        sh.claim_done[buf] = 0;
        sh.issued[buf] += 1;
        stage_block_bulk(p, b, hbuf0 + buf * p.head_smem, &sh.full[buf]);
    };

    // A CTA that gave up a wait skips its remaining items; each one records
    // the timeout in its own forest's status, since its outputs stay unwritten
    // (sh.abort is uniform here: it changes only inside the bin loop, and the
    // previous item ended with a CTA barrier).
    if (*(volatile int *)&sh.abort) {
        if (tid == 0) report(p.status, FP_ERR_FLAG_TIMEOUT);
        return;
    }
    const int pass = (int)(item / p.n_tiles);
    const int64_t tile = item - (int64_t)pass * p.n_tiles;
    const int64_t row0 = tile * R;
    const int rows = (int)(p.n - row0 < (int64_t)R ? p.n - row0 : (int64_t)R);
    const FpPass ps = p.passes[pass];
    const int nbins = ps.bin_end - ps.bin_begin;
    const float inv_rows = 1.0f / (float)rows;

    // 1. rows (feature-major, as order keys) -> shared memory; 2. the first
    //    bins' blocks in flight
    const float *src = p.X + row0 * F;
    const bool vec_rows = (F & 3) == 0 && (reinterpret_cast<uintptr_t>(p.X) & 15) == 0;
    {
        if (vec_rows) {
            // lane = row: 16-byte loads along the row, and each store of a
            // warp writes 32 consecutive rows of one feature (32 banks).  The
            // work is cut into units of 32 rows x 16 features, dealt out to
            // all warps, so that a tile of few wide rows (784 features, 64
            // rows) is staged by every warp, not by two
            const int nq = F >> 2;
            const int groups = (rows + 31) >> 5, qblocks = (nq + 3) >> 2;
            for (int u = warp; u < groups * qblocks; u += nwarps) {
                const int g = u % groups, q0 = (u / groups) * 4;
                const int r = g * 32 + lane;
                if (r < rows) {
                    const float4 *rp = reinterpret_cast<const float4 *>(src + (int64_t)r * F);
                    uint32_t *dst = xs + r;
                    if (q0 + 4 <= nq) {
                        float4 v[4];
#pragma unroll
                        for (int k = 0; k < 4; ++k) v[k] = __ldg(rp + q0 + k);
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            uint32_t *d = dst + (4 * (q0 + k)) * R;
                            d[0] = staged<DK>(p, v[k].x);
                            d[R] = staged<DK>(p, v[k].y);
                            d[2 * R] = staged<DK>(p, v[k].z);
                            d[3 * R] = staged<DK>(p, v[k].w);
                        }
                    } else {
                        for (int q = q0; q < nq; ++q) {
                            const float4 v = __ldg(rp + q);
                            uint32_t *d = dst + (4 * q) * R;
                            d[0] = staged<DK>(p, v.x);
                            d[R] = staged<DK>(p, v.y);
                            d[2 * R] = staged<DK>(p, v.z);
                            d[3 * R] = staged<DK>(p, v.w);
                        }
                    }
                }
            }
        } else {
            const int total = rows * F;
            for (int e = tid; e < total; e += blockDim.x) {
                const int r = e / F;
                cp_async4(xs + (e - r * F) * R + r, src + e);
            }
        }
        cp_async_commit();
    }
    if (tid == 0) {
        for (int i = 0; i < FP_NBUF; ++i) sh.use0[i] = sh.issued[i];
        if (!sh.abort)
            for (int i = 0; i < nbuf && i < nbins; ++i) issue(ps.bin_begin + i, i);

    }
    if (!LEAVES)
        for (int i = tid; i < R * CS; i += blockDim.x) svotes[i] = 0;
    cp_async_wait_all();
    if (D3 && !vec_rows) {  // each thread turns the values it copied into keys
        const int total = rows * F;
        for (int e = tid; e < total; e += blockDim.x) {
            const int r = e / F;
            uint32_t *x = xs + (e - r * F) * R + r;
            *x = staged<DK>(p, __uint_as_float(*x));
        }
    }
    __syncthreads();

    LaneTask L;
    L.active = false;
    L.r = 0;
    L.t = 0;
    L.ref = 0;
    int head = 0, tail = 0;  // warp-uniform ring cursors

    const int u0 = sh.use0[0], u1 = sh.use0[1], u2 = sh.use0[2];  // read after the barrier above
    for (int bi = 0; bi < nbins; ++bi) {
        const int buf = bi % nbuf;
        {  // wait until the bin's block has landed
            const int ub = buf == 0 ? u0 : (buf == 1 ? u1 : u2);
            const uint32_t parity = (uint32_t)(ub + bi / nbuf) & 1u;
            bool ok = false;
            for (int spin = 0; spin < p.spin_limit; ++spin) {
                if (*(volatile int *)&sh.abort) break;
                if (mbar_try_wait(&sh.full[buf], parity) && !p.stall) {
                    ok = true;
                    break;
                }
            }
            if (!__all_sync(0xffffffffu, ok)) {
                if (lane == 0 && !*(volatile int *)&sh.abort) {
                    report(p.status, FP_ERR_FLAG_TIMEOUT);
                    *(volatile int *)&sh.abort = 1;
                }
                break;
            }
        }
        const int b = ps.bin_begin + bi;
        const FpBin bn = p.bins[b];
        const int stride = bn.stride, nranks = bn.nranks, nexits = bn.nexits;
        const int ntask = rows * bn.width;
        const uint8_t *blk = hbuf0 + buf * p.head_smem;
        const uint2 *hnode = reinterpret_cast<const uint2 *>(blk);
        const uint32_t *hexit =
            reinterpret_cast<const uint32_t *>(blk + (size_t)nranks * stride * (levels == 2 ? 16 : 8));

        for (;;) {
            uint32_t w[8];
            if (L.active) deep_issue(p, L, w);  // in flight during the burst below
            if (tail - head <= p.refill) {
                // burst: 32 consecutive tasks through the head, all lanes together
                int base = 0;
                if (lane == 0) base = atomicAdd(&sh.task_next[buf], 32);
                base = __shfl_sync(0xffffffffu, base, 0);
                if (base >= ntask) {  // the bin is claimed out: use the load in flight, then move on
                    if (L.active) deep_finish<MODE, DK>(p, xs, svotes, row0, L, w);
                    pop_tasks(p, ring, head, tail, L, lt_mask);
                    break;
                }
                const bool my = lane < ntask - base;
                const int task = base + lane;
                // task / rows by a float reciprocal, corrected to the exact quotient
                int k2 = my ? (int)((float)task * inv_rows) : 0;
                if (my) {
                    k2 -= k2 * rows > task;
                    k2 += (k2 + 1) * rows <= task;
                }
                const int r2 = my ? task - k2 * rows : 0;
                uint32_t hr = 0;  // head rank (or slot), then nranks + exit index
                const uint2 *hn = hnode + k2;  // this lane's tree column of the block
                const uint32_t *xr = xs + r2;  // this lane's row
                if (levels == 2) {
                    // paired slots: a node and its two children per 16-byte record,
                    // successors 4q+1 .. 4q+4; (depth+1)/2 records per walk
                    const uint4 *hq = reinterpret_cast<const uint4 *>(blk) + k2;
#pragma unroll 1  // measured: unrolling the head walk only adds instructions
                    for (int l = 0; l <= p.depth; l += 2) {
                        const uint4 nd = hq[hr * stride];
                        const uint32_t x0 = xr[(nd.w & 1023u) * R];
                        const uint32_t d0 = goes_left<D3>(x0, nd.x) ? 0u : 1u;
                        const uint32_t f1 = d0 ? (nd.w >> 20) & 1023u : (nd.w >> 10) & 1023u;
                        const uint32_t x1 = xr[f1 * R];
                        const uint32_t d1 = goes_left<D3>(x1, d0 ? nd.z : nd.y) ? 0u : 1u;
                        hr = 4 * hr + 1 + 2 * d0 + d1;
                    }
                } else if (levels) {
                    // implicit slots: every walk takes depth+1 steps, children 2s+1, 2s+2
#pragma unroll 1
                    for (int l = 0; l <= p.depth; ++l) {
                        const uint2 nd = hn[hr * stride];
                        const uint32_t xv = xr[(nd.y >> 22) * R];
                        hr = 2 * hr + (goes_left<D3>(xv, nd.x) ? 1u : 2u);
                    }
                }
                bool busy = my && !levels;
                while ((HK <= 0 || levels == 0) && __any_sync(0xffffffffu, busy)) {  // ranked heads only
#pragma unroll
                    for (int u = 0; u < 2; ++u) {  // two steps per vote
                        if (busy) {
                            const uint2 nd = hn[hr * stride];
                            const uint32_t m = nd.y;
                            uint32_t nh = goes_left<D3>(xr[(m >> 22) * R], nd.x)
                                              ? (m & FP_TARGET_MASK)
                                              : ((m >> FP_TARGET_BITS) & FP_TARGET_MASK);
                            busy = nh < (uint32_t)nranks;
                            if (busy && nh <= hr) {  // ranks grow along every path of a valid block
                                report(p.status, FP_ERR_FLAG_DEVICE);
                                busy = false;
                                nh = (uint32_t)(nranks + nexits);
                            }
                            hr = nh;
                        }
                    }
                }
                const uint32_t e = hr - (uint32_t)nranks;
                const uint32_t er = (my && e < (uint32_t)nexits) ? hexit[e * stride + k2] : FP_NO_CLASS;
                const int t2 = bn.first_tree + k2;
                if (my && (er & FP_REF_LEAF)) {
                    int32_t leaf_id = -1;
                    if (LEAVES && e < (uint32_t)nexits) leaf_id = p.pheads[(bn.phead_off >> 2) + e * stride + k2];
                    finish<MODE>(p, svotes, row0, r2, t2, er & 0x7FFFFFFFu, leaf_id);
                }
                const bool push = my && !(er & FP_REF_LEAF);
                const unsigned pm = __ballot_sync(0xffffffffu, push);
                if (push)
                    ring[(tail + __popc(pm & lt_mask)) & (FP_RING - 1)] =
                        make_uint2(er, (uint32_t)r2 | ((uint32_t)t2 << 11));
                tail += __popc(pm);
                __syncwarp();
            }
            if (L.active) deep_finish<MODE, DK>(p, xs, svotes, row0, L, w);
            pop_tasks(p, ring, head, tail, L, lt_mask);
        }
        // this warp reads the bin's block no more; the last warp refills the buffer
        __syncwarp();
        if (lane == 0) {
            const int done = atomicAdd(&sh.claim_done[buf], 1);
            if (done == nwarps - 1 && bi + nbuf < nbins && !*(volatile int *)&sh.abort)
                issue(ps.bin_begin + bi + nbuf, bi + nbuf);
        }
        __syncwarp();
    }
    const bool aborted = *(volatile int *)&sh.abort != 0;
    // drain: the item's last pending and running tasks
    for (; !aborted;) {
        __syncwarp();
        pop_tasks(p, ring, head, tail, L, lt_mask);
        if (!__any_sync(0xffffffffu, L.active)) break;
        if (L.active) {
            uint32_t w[8];
            deep_issue(p, L, w);
            deep_finish<MODE, DK>(p, xs, svotes, row0, L, w);
        }
    }
    __syncthreads();

    // 5. values: bias + scale * the row's sum (several passes: summed in global
    //    memory, the CTA finishing a tile's last pass writes the result)
    if (VALUES && !*(volatile int *)&sh.abort) {
        const float *sv = reinterpret_cast<const float *>(svotes);
        if (p.n_passes == 1) {
            for (int rr = tid; rr < rows; rr += blockDim.x) p.out_val[row0 + rr] = p.vbias + p.vscale * sv[rr];
        } else {
            float *dst = p.acc_val + row0;
            for (int rr = tid; rr < rows; rr += blockDim.x) {
                const float v = sv[rr];
                if (v != 0.0f) atomicAdd(dst + rr, v);
            }
            __threadfence();
            __syncthreads();
            if (tid == 0) sh.last = atomicAdd(p.tile_done + tile, 1u) == (unsigned)(p.n_passes - 1);
            __syncthreads();
            if (sh.last) {
                __threadfence();
                for (int rr = tid; rr < rows; rr += blockDim.x)
                    p.out_val[row0 + rr] = p.vbias + p.vscale * __ldcg(dst + rr);
            }
        }
    }
    // 5. votes and class
    if (MODE == FP_MODE_VOTES && !*(volatile int *)&sh.abort) {
        if (p.n_passes == 1) {
            if (p.out_votes) {  // counters are class-major (svotes[c * R + r]), the output row-major
                uint32_t *dst = p.out_votes + row0 * C;
                for (int i = tid; i < rows * C; i += blockDim.x) {
                    const int rr = i / C;
                    dst[i] = svotes[(i - rr * C) * R + rr];
                }
            }
            if (p.out_class) {
                for (int rr = tid; rr < rows; rr += blockDim.x) {
                    const uint32_t *v = svotes + rr;
                    int best = 0;
                    uint32_t bv = v[0];
                    for (int c = 1; c < C; ++c)
                        if (v[c * R] > bv) { bv = v[c * R]; best = c; }
                    p.out_class[row0 + rr] = best;
                }
            }
        } else {
            uint32_t *dst = p.acc + row0 * C;
            for (int i = tid; i < rows * C; i += blockDim.x) {
                const int rr = i / C;
                const uint32_t v = svotes[(i - rr * C) * R + rr];
                if (v) atomicAdd(dst + i, v);
            }
            if (p.out_class) {
                __threadfence();
                __syncthreads();
                if (tid == 0) sh.last = atomicAdd(p.tile_done + tile, 1u) == (unsigned)(p.n_passes - 1);
                __syncthreads();
                if (sh.last) {
                    __threadfence();
                    for (int rr = tid; rr < rows; rr += blockDim.x) {
                        const uint32_t *v = dst + rr * C;
                        int best = 0;
                        uint32_t bv = __ldcg(v);
                        for (int c = 1; c < C; ++c) {
                            const uint32_t w = __ldcg(v + c);
                            if (w > bv) { bv = w; best = c; }
                        }
                        p.out_class[row0 + rr] = best;
                    }
                }
            }
        }
    }
    __syncthreads();  // the next item reuses shared memory

}

// MINB = 1: one CTA of up to 1024 threads per SM (up to 64 registers a thread);
// MINB = 2: CTAs of up to 768 threads, at most 42 registers a thread, so that
// two 24-warp or three 16-warp CTAs share an SM when shared memory allows:
// more warps to hide the latency of the dependent loads of each walk.
template <int MODE, int MINB, int DK, int HK>
__global__ void __launch_bounds__(MINB == 1 ? 1024 : 768, MINB) fp_traverse_kernel(const TravParams p) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ CtaShared sh;
    cta_init(sh);
    for (int64_t item = blockIdx.x; item < p.n_items; item += gridDim.x) run_item<MODE, DK, HK>(p, item, smem, sh);
    cta_finish(sh);
}

// Several forests and batches in one persistent launch: the work items of
// all batches form one list (batch by batch, pass-major within a batch),
// handed out to CTAs through a global counter so uneven batches balance.
#define FP_MAX_BATCH 32

struct BatchParams {
    int32_t k;
    int64_t item_begin[FP_MAX_BATCH + 1];
    TravParams p[FP_MAX_BATCH];
    unsigned long long *work;  // zeroed before the launch
};

// KIND: 2, 3 or 4 when every forest of the launch has that kind of
// super-node (one walk compiled in), 0 for a mix (all, chosen per item).  HK:
// the head kind when all forests share it (0 ranked, 1, 2), else -1.
template <int KIND, int HK>
__global__ void __launch_bounds__(1024, 1) fp_traverse_batched_kernel(const __grid_constant__ BatchParams bp) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ CtaShared sh;
    cta_init(sh);
    const int64_t total = bp.item_begin[bp.k];
    for (;;) {
        if (threadIdx.x == 0) sh.next_item = (long long)atomicAdd(bp.work, 1ull);
        __syncthreads();
        const int64_t item = sh.next_item;
        __syncthreads();
        if (item >= total) break;
        int j = 0;
        while (j + 1 < bp.k && bp.item_begin[j + 1] <= item) ++j;
        if (KIND == 3 || (KIND == 0 && bp.p[j].deep_kind == 3))
            run_item<FP_MODE_VOTES, 3, HK>(bp.p[j], item - bp.item_begin[j], smem, sh);
        else if (KIND == 4 || (KIND == 0 && bp.p[j].deep_kind == 4))
            run_item<FP_MODE_VOTES, 4, HK>(bp.p[j], item - bp.item_begin[j], smem, sh);
        else
            run_item<FP_MODE_VOTES, 2, HK>(bp.p[j], item - bp.item_begin[j], smem, sh);
    }
    cta_finish(sh);
}
