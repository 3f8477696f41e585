// fp_plain.cu -- the plain GPU baseline: breadth-first per-tree layout
// (Section III-A, BF, the layout the paper measures against in Section IV-B),
// evaluated the plain way: one thread per (observation, tree), a global
// atomic vote per thread, then a separate argmax kernel; one launch per batch.
//
// Record {float thr; uint32 meta}, 8 bytes, per tree in breadth-first order:
//   meta bit 31 = 1: leaf, meta & 0x7FFFFFFF = class; in a forest with leaf
//                    values the first word holds the leaf's value instead
//                    of a threshold
//   meta bit 31 = 0: [30:21] feature, [20:0] tree-local index of the left
//                    child; the right child follows it (siblings are adjacent
//                    in breadth-first order).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/forest_pack.h"
#include "fp_common.h"

struct fp_plain_forest {
    int device = -1;
    int32_t T = 0, F = 0, C = 0;
    bool values = false;  // leaf records carry values
    uint2 *d_recs = nullptr;
    int64_t *d_tree_off = nullptr;
    int64_t n_recs = 0;
};

namespace {

int plain_fail(cudaError_t e, const char *what) {
    fp_set_error("%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? FP_ENOMEM : FP_ECUDA;
}

__global__ void plain_vote_kernel(const uint2 *__restrict__ recs, const int64_t *__restrict__ tree_off,
                                  const float *__restrict__ X, int64_t n, int32_t T, int32_t F, int32_t C,
                                  int32_t order, uint32_t *__restrict__ votes) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= n * T) return;
    int64_t i;
    int32_t t;
    if (order == FP_PLAIN_OBS_FASTEST) {
        t = (int32_t)(tid / n);
        i = tid - (int64_t)t * n;
    } else {
        i = tid / T;
        t = (int32_t)(tid - i * T);
    }
    const uint2 *tree = recs + tree_off[t];
    const float *x = X + i * F;
    uint32_t node = 0;
    for (;;) {
        const uint2 rec = __ldg(tree + node);
        if (rec.y & 0x80000000u) {
            const uint32_t cls = rec.y & 0x7FFFFFFFu;
            if (cls < (uint32_t)C) atomicAdd(votes + i * C + cls, 1u);
            return;
        }
        const float v = __ldg(x + ((rec.y >> 21) & 1023u));
        node = (rec.y & 0x1FFFFFu) + (v <= __uint_as_float(rec.x) ? 0u : 1u);
    }
}

// Forests with leaf values: thread per (observation, tree), the leaf's value
// added to the row with a global float atomic.
__global__ void plain_value_kernel(const uint2 *__restrict__ recs, const int64_t *__restrict__ tree_off,
                                   const float *__restrict__ X, int64_t n, int32_t T, int32_t F, int32_t order,
                                   float *__restrict__ sum) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= n * T) return;
    int64_t i;
    int32_t t;
    if (order == FP_PLAIN_OBS_FASTEST) {
        t = (int32_t)(tid / n);
        i = tid - (int64_t)t * n;
    } else {
        i = tid / T;
        t = (int32_t)(tid - i * T);
    }
    const uint2 *tree = recs + tree_off[t];
    const float *x = X + i * F;
    uint32_t node = 0;
    for (;;) {
        const uint2 rec = __ldg(tree + node);
        if (rec.y & 0x80000000u) {
            atomicAdd(sum + i, __uint_as_float(rec.x));
            return;
        }
        const float v = __ldg(x + ((rec.y >> 21) & 1023u));
        node = (rec.y & 0x1FFFFFu) + (v <= __uint_as_float(rec.x) ? 0u : 1u);
    }
}

__global__ void plain_value_finish_kernel(float *__restrict__ out, int64_t n, float scale, float bias) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = bias + scale * out[i];
}

__global__ void plain_argmax_kernel(const uint32_t *__restrict__ votes, int64_t n, int32_t C,
                                    int32_t *__restrict__ out_class) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t *v = votes + i * C;
    int best = 0;
    uint32_t bv = v[0];
    for (int c = 1; c < C; ++c)
        if (v[c] > bv) { bv = v[c]; best = c; }
    out_class[i] = best;
}

}  // namespace

extern "C" int fp_plain_build(const fp_forest_desc *desc, void *stream, fp_plain_forest **out) {
    if (!out || !desc || !desc->tree_node_begin || !desc->left || !desc->right || !desc->feature ||
        !desc->threshold || !desc->leaf_class) {
        fp_set_error("fp_plain_build: NULL argument");
        return FP_EINVAL;
    }
    *out = nullptr;
    const int32_t T = desc->n_trees, F = desc->n_features, C = desc->n_classes;
    if (T < 1 || F < 1 || F > 1024 || C < 1 || desc->tree_node_begin[0] != 0) {
        fp_set_error("fp_plain_build: bad forest sizes");
        return FP_EINVAL;
    }
    std::vector<uint2> recs;
    std::vector<int64_t> off((size_t)T + 1, 0);
    try {
        recs.reserve((size_t)desc->tree_node_begin[T]);
        std::vector<int32_t> queue;
        for (int32_t t = 0; t < T; ++t) {
            const int64_t b = desc->tree_node_begin[t], m = desc->tree_node_begin[t + 1] - b;
            if (m < 1 || m > (1 << 21)) {
                fp_set_error("fp_plain_build: tree %d has %lld nodes (1..2^21)", t, (long long)m);
                return m < 1 ? FP_EINVAL : FP_EUNSUPPORTED;
            }
            off[t] = (int64_t)recs.size();
            // breadth-first order: position of node = its index in the queue
            queue.assign(1, 0);
            for (size_t h = 0; h < queue.size(); ++h) {
                const int32_t v = queue[h];
                if (v < 0 || v >= m || queue.size() > (size_t)m) {
                    fp_set_error("fp_plain_build: tree %d is malformed", t);
                    return FP_EINVAL;
                }
                if (desc->left[b + v] >= 0) {
                    queue.push_back(desc->left[b + v]);
                    queue.push_back(desc->right[b + v]);
                }
            }
            size_t child = 1;
            for (size_t h = 0; h < queue.size(); ++h) {
                const int32_t v = queue[h];
                uint2 r;
                if (desc->left[b + v] < 0) {
                    const int32_t c = desc->leaf_class[b + v];
                    if (c < 0 || c >= C) {
                        fp_set_error("fp_plain_build: tree %d leaf %d class %d out of range", t, v, c);
                        return FP_EINVAL;
                    }
                    r.x = 0;
                    if (desc->leaf_value) {
                        const float val = desc->leaf_value[b + v];
                        if (!(val - val == 0.0f)) {
                            fp_set_error("fp_plain_build: tree %d leaf %d has a non-finite value", t, v);
                            return FP_EINVAL;
                        }
                        memcpy(&r.x, &val, 4);
                    }
                    r.y = 0x80000000u | (uint32_t)c;
                } else {
                    const int32_t f = desc->feature[b + v];
                    if (f < 0 || f >= F) {
                        fp_set_error("fp_plain_build: tree %d node %d feature out of range", t, v);
                        return FP_EINVAL;
                    }
                    float th = desc->threshold[b + v];
                    memcpy(&r.x, &th, 4);
                    r.y = ((uint32_t)f << 21) | (uint32_t)child;
                    child += 2;
                }
                recs.push_back(r);
            }
        }
        off[T] = (int64_t)recs.size();
    } catch (const std::bad_alloc &) {
        fp_set_error("fp_plain_build: out of host memory");
        return FP_ENOMEM;
    }
    fp_plain_forest *pf = new (std::nothrow) fp_plain_forest;
    if (!pf) return FP_ENOMEM;
    pf->T = T; pf->F = F; pf->C = C; pf->n_recs = (int64_t)recs.size();
    pf->values = desc->leaf_value != nullptr;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaGetDevice(&pf->device);
    if (e == cudaSuccess) e = cudaMalloc(&pf->d_recs, recs.size() * sizeof(uint2));
    if (e == cudaSuccess) e = cudaMalloc(&pf->d_tree_off, off.size() * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMemcpyAsync(pf->d_recs, recs.data(), recs.size() * sizeof(uint2),
                                              cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(pf->d_tree_off, off.data(), off.size() * sizeof(int64_t),
                                              cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        int rc = plain_fail(e, "fp_plain_build");
        cudaFree(pf->d_recs);
        cudaFree(pf->d_tree_off);
        delete pf;
        return rc;
    }
    *out = pf;
    return FP_OK;
}

extern "C" int fp_plain_predict(const fp_plain_forest *pf, const float *X, int64_t n, int32_t order,
                                uint32_t *out_votes, int32_t *out_class, void *stream) {
    if (!pf || n < 0 || (n > 0 && (!X || !out_votes)) ||
        (order != FP_PLAIN_OBS_FASTEST && order != FP_PLAIN_TREE_FASTEST)) {
        fp_set_error("fp_plain_predict: bad arguments");
        return FP_EINVAL;
    }
    if (pf->values) {
        fp_set_error("fp_plain_predict: the forest has leaf values; use fp_plain_predict_values");
        return FP_EINVAL;
    }
    if (n == 0) return FP_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(out_votes, 0, (size_t)n * pf->C * 4, s);
    if (e != cudaSuccess) return plain_fail(e, "cudaMemsetAsync(votes)");
    const int threads = 256;
    const int64_t work = n * pf->T;
    const int64_t blocks = (work + threads - 1) / threads;
    if (blocks > INT32_MAX) {
        fp_set_error("fp_plain_predict: batch too large for one launch");
        return FP_EUNSUPPORTED;
    }
    plain_vote_kernel<<<(unsigned)blocks, threads, 0, s>>>(pf->d_recs, pf->d_tree_off, X, n, pf->T, pf->F, pf->C,
                                                           order, out_votes);
    e = cudaGetLastError();
    if (e != cudaSuccess) return plain_fail(e, "plain_vote_kernel launch");
    if (out_class) {
        plain_argmax_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(out_votes, n, pf->C, out_class);
        e = cudaGetLastError();
        if (e != cudaSuccess) return plain_fail(e, "plain_argmax_kernel launch");
    }
    return FP_OK;
}

extern "C" int fp_plain_predict_values(const fp_plain_forest *pf, const float *X, int64_t n, int32_t order,
                                       float scale, float bias, float *out, void *stream) {
    if (!pf || n < 0 || (n > 0 && (!X || !out)) ||
        (order != FP_PLAIN_OBS_FASTEST && order != FP_PLAIN_TREE_FASTEST)) {
        fp_set_error("fp_plain_predict_values: bad arguments");
        return FP_EINVAL;
    }
    if (!pf->values) {
        fp_set_error("fp_plain_predict_values: the forest was built without leaf values");
        return FP_EINVAL;
    }
    if (n == 0) return FP_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(out, 0, (size_t)n * 4, s);
    if (e != cudaSuccess) return plain_fail(e, "cudaMemsetAsync(out)");
    const int threads = 256;
    const int64_t blocks = (n * pf->T + threads - 1) / threads;
    if (blocks > INT32_MAX) {
        fp_set_error("fp_plain_predict_values: batch too large for one launch");
        return FP_EUNSUPPORTED;
    }
    plain_value_kernel<<<(unsigned)blocks, threads, 0, s>>>(pf->d_recs, pf->d_tree_off, X, n, pf->T, pf->F, order,
                                                            out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return plain_fail(e, "plain_value_kernel launch");
    plain_value_finish_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(out, n, scale, bias);
    e = cudaGetLastError();
    if (e != cudaSuccess) return plain_fail(e, "plain_value_finish_kernel launch");
    return FP_OK;
}

extern "C" int64_t fp_plain_bytes(const fp_plain_forest *pf) {
    return pf ? pf->n_recs * (int64_t)sizeof(uint2) + (int64_t)(pf->T + 1) * 8 : 0;
}

extern "C" void fp_plain_release(fp_plain_forest *pf) {
    if (!pf) return;
    cudaDeviceSynchronize();
    cudaFree(pf->d_recs);
    cudaFree(pf->d_tree_off);
    delete pf;
}
