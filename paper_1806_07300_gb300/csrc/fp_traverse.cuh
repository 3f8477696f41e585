// fp_traverse.cuh -- the packed-forest traversal kernel (sm_103a).
//
// One work item = (pass, observation tile).  Items are ordered pass-major, so
// at any moment the whole GPU walks the bins of one pass, whose records stay
// resident in L2 while every tile of observations goes through them (the
// GPU counterpart of the paper's bins bound to cores, Section III and
// Section IV-D).  Within an item the CTA:
//   1. stages the tile's rows into shared memory with 4-byte cp.async, at an
//      odd row stride so that lanes reading one feature of 32 rows hit 32
//      banks;
//   2. for each bin of the pass, stages the bin's interleaved block (levels
//      0..d of all its trees plus the link row, Section III-A Bin) into shared
//      memory with 16-byte cp.async;
//   3. walks (observation, tree) tasks: the lanes of a warp take consecutive
//      observations of the same tree, walk the interleaved levels in shared
//      memory, then the tree's Stat region in global memory, where the hot
//      child is the next record (Section III-A Stat).  A lane that reaches a
//      leaf takes the warp's next task at once: free lanes are found with
//      __ballot_sync and numbered with __popc, so lanes stay busy while paths
//      of different depth diverge (the GPU form of Section III-B's
//      round-robin over a bin's trees);
//   4. counts votes per (row, class) with shared-memory atomics;
//   5. writes votes and the argmax class (lowest class on ties).  With one
//      pass the tile's votes are complete in shared memory; with several, the
//      tile's votes are added to a global accumulator and the CTA that
//      finishes a tile's last pass (per-tile counter, no waiting) takes the
//      argmax.
// Parity mode writes the leaf id reached in every (observation, tree)
// instead of voting.
//
// Every wait in this kernel is a hardware wait (cp.async.wait_all,
// __syncthreads); there is no spin loop.
#pragma once
#include <stdint.h>

#include "fp_internal.h"

struct TravParams {
    const uint2 *deep;        // deep records
    const uint8_t *heads;     // heads section
    const FpBin *bins;
    const FpPass *passes;
    const uint32_t *tree_base;
    const int32_t *pheads;    // parity heads section
    const int2 *deep_leaf;    // parity: leaf ids per deep record
    const float *X;
    int64_t n;
    int64_t n_tiles;
    int64_t n_items;
    int32_t F, P, C, T, S, Lk, R;
    int32_t n_passes;
    int32_t head_smem;        // bytes reserved for one bin block
    uint32_t *out_votes;      // single pass: final votes (may be NULL)
    int32_t *out_class;       // may be NULL
    int32_t *out_leaf;        // parity mode
    uint32_t *acc;            // several passes: vote accumulator
    uint32_t *tile_done;      // several passes: per-tile pass counter
    int32_t *status;          // device status word
};

#define FP_STATUS_BAD_CLASS 2
#define FP_ERR_FLAG_DEVICE (-6)

__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ uint2 ld_record(const uint2 *p) {
    uint2 v;
    asm volatile("ld.global.nc.v2.u32 {%0, %1}, [%2];\n" : "=r"(v.x), "=r"(v.y) : "l"(p));
    return v;
}

__device__ __forceinline__ void report(int32_t *status, int32_t code) { atomicCAS(status, 0, code); }

template <bool LEAVES>
__global__ void __launch_bounds__(1024) fp_traverse_kernel(const TravParams p) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ int s_task_next;
    __shared__ int s_last;
    const int R = p.R, P = p.P, F = p.F, C = p.C, S = p.S;
    float *xs = reinterpret_cast<float *>(smem);
    const int xs_bytes = ((R * P * 4) + 15) & ~15;
    uint8_t *hbuf = smem + xs_bytes;
    uint32_t *svotes = reinterpret_cast<uint32_t *>(hbuf + p.head_smem);
    const int tid = threadIdx.x, lane = tid & 31;
    const unsigned lt_mask = (1u << lane) - 1u;

    for (int64_t item = blockIdx.x; item < p.n_items; item += gridDim.x) {
        const int pass = (int)(item / p.n_tiles);
        const int64_t tile = item - (int64_t)pass * p.n_tiles;
        const int64_t row0 = tile * R;
        const int rows = (int)(p.n - row0 < (int64_t)R ? p.n - row0 : (int64_t)R);

        // 1. rows -> shared memory (odd stride P)
        {
            const float *src = p.X + row0 * F;
            const int total = rows * F;
            for (int e = tid; e < total; e += blockDim.x) {
                const int r = e / F;
                cp_async4(xs + r * P + (e - r * F), src + e);
            }
        }
        if (!LEAVES)
            for (int i = tid; i < rows * C; i += blockDim.x) svotes[i] = 0;

        const FpPass ps = p.passes[pass];
        for (int b = ps.bin_begin; b < ps.bin_end; ++b) {
            const FpBin bn = p.bins[b];
            // 2. interleaved block -> shared memory
            {
                const uint8_t *src = p.heads + bn.head_off;
                for (int o = tid * 16; o < (int)bn.head_bytes; o += blockDim.x * 16) cp_async16(hbuf + o, src + o);
            }
            if (tid == 0) s_task_next = 0;
            cp_async_wait_all();
            __syncthreads();

            // 3. walk (observation, tree) tasks
            const int width = bn.width;
            const int ntask = rows * width;
            const uint2 *hrec = reinterpret_cast<const uint2 *>(hbuf);
            const uint32_t *hlink = reinterpret_cast<const uint32_t *>(hbuf + (size_t)S * width * 8);
            int pool_next = 0, pool_end = 0;  // warp-uniform local task window
            bool exhausted = false;           // warp-uniform: the bin's tasks are all claimed
            bool active = false;
            int r = 0, k = 0;
            uint32_t idx = 0;
            const uint2 *tdeep = p.deep;
            const float *xrow = xs;
            for (;;) {
                // refill free lanes; a new task first walks the interleaved levels
                while (!exhausted) {
                    const unsigned free_mask = __ballot_sync(0xffffffffu, !active);
                    if (free_mask == 0) break;
                    if (pool_next >= pool_end) {
                        int base = 0;
                        if (lane == 0) base = atomicAdd(&s_task_next, 32);
                        base = __shfl_sync(0xffffffffu, base, 0);
                        if (base >= ntask) {
                            exhausted = true;
                            break;
                        }
                        pool_next = base;
                        pool_end = min(base + 32, ntask);
                    }
                    const int avail = pool_end - pool_next;
                    const int rank = __popc(free_mask & lt_mask);
                    const bool take = !active && rank < avail;
                    const int task = pool_next + rank;
                    pool_next += min(avail, __popc(free_mask));
                    if (!take) continue;
                    k = task / rows;
                    r = task - k * rows;
                    xrow = xs + r * P;
                    const int t = bn.first_tree + k;
                    // interleaved levels 0..d
                    int s = 0;
                    int32_t cls = -1, leaf_id = -1;
                    bool done = false;
                    for (;;) {
                        const uint2 rec = hrec[s * width + k];
                        if (rec.y & FP_HEAD_LEAF) {
                            cls = (int32_t)(rec.y & 0x7FFFFFFFu);
                            if (LEAVES) leaf_id = p.pheads[(bn.phead_off >> 2) + s * width + k];
                            done = true;
                            break;
                        }
                        const float x = xrow[rec.y];
                        s = 2 * s + 1 + (x <= __uint_as_float(rec.x) ? 0 : 1);
                        if (s >= S) {
                            const uint32_t e = hlink[(s - S) * width + k];
                            if (e & FP_HEAD_LEAF) {
                                cls = (int32_t)(e & 0x7FFFFFFFu);
                                if (LEAVES) leaf_id = p.pheads[(bn.phead_off >> 2) + s * width + k];
                                done = true;
                            } else {
                                idx = e;
                                tdeep = p.deep + p.tree_base[t];
                                active = true;
                            }
                            break;
                        }
                    }
                    if (done) {
                        if (LEAVES) {
                            p.out_leaf[(row0 + r) * p.T + t] = leaf_id;
                        } else if ((unsigned)cls < (unsigned)C) {
                            atomicAdd(&svotes[r * C + cls], 1u);
                        } else {
                            report(p.status, FP_ERR_FLAG_DEVICE);
                        }
                    }
                }
                if (__ballot_sync(0xffffffffu, active) == 0) break;
                // one level of the Stat region for every active lane
                if (active) {
                    const uint2 rec = ld_record(tdeep + idx);
                    const uint32_t m = rec.y;
                    const float x = xrow[m >> FP_META_FEATURE_SHIFT];
                    const uint32_t right = x <= __uint_as_float(rec.x) ? 0u : 1u;
                    const uint32_t pay = m & FP_META_PAYLOAD_MASK;
                    int32_t cls = -1;
                    if (m & FP_META_BOTH_LEAF) {
                        cls = (int32_t)(right ? (pay >> 9) : (pay & 511u));
                    } else if (right == ((m >> 21) & 1u)) {
                        idx += 1;
                    } else if (m & FP_META_COLD_LEAF) {
                        cls = (int32_t)pay;
                    } else {
                        idx = pay;
                    }
                    if (cls >= 0) {
                        active = false;
                        if (LEAVES) {
                            const int2 lf = p.deep_leaf[(tdeep - p.deep) + idx];
                            p.out_leaf[(row0 + r) * p.T + bn.first_tree + k] = right ? lf.y : lf.x;
                        } else if (cls < C) {
                            atomicAdd(&svotes[r * C + cls], 1u);
                        } else {
                            report(p.status, FP_ERR_FLAG_DEVICE);
                        }
                    }
                }
            }
            __syncthreads();  // the next bin overwrites the block
        }

        // 5. votes and class
        if (!LEAVES) {
            if (p.n_passes == 1) {
                if (p.out_votes) {
                    uint32_t *dst = p.out_votes + row0 * C;
                    for (int i = tid; i < rows * C; i += blockDim.x) dst[i] = svotes[i];
                }
                if (p.out_class) {
                    for (int rr = tid; rr < rows; rr += blockDim.x) {
                        const uint32_t *v = svotes + rr * C;
                        int best = 0;
                        uint32_t bv = v[0];
                        for (int c = 1; c < C; ++c)
                            if (v[c] > bv) { bv = v[c]; best = c; }
                        p.out_class[row0 + rr] = best;
                    }
                }
            } else {
                uint32_t *dst = p.acc + row0 * C;
                for (int i = tid; i < rows * C; i += blockDim.x) {
                    const uint32_t v = svotes[i];
                    if (v) atomicAdd(dst + i, v);
                }
                if (p.out_class) {
                    __threadfence();
                    __syncthreads();
                    if (tid == 0) s_last = atomicAdd(p.tile_done + tile, 1u) == (unsigned)(p.n_passes - 1);
                    __syncthreads();
                    if (s_last) {
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
}
