// fp_stats.cu -- statistics inferred from observations (Section III-A: the
// leaf cardinalities that order a tree's nodes need not come from training;
// they may be estimated afterwards by classifying many observations).
//
// fp_count_leaves turns the leaf ids that fp_predict_leaves wrote for a
// sample of observations into per-node visit counts of the leaves; summing a
// leaf's count into its ancestors (host side, one pass over the tree) gives
// cardinalities to pack the forest with instead of the training counts.
#include <cuda_runtime.h>

#include "../../include/forest_pack.h"
#include "fp_common.h"

namespace {

__global__ void count_leaves_kernel(const int32_t *__restrict__ leaf, int64_t n, int32_t T,
                                    const int64_t *__restrict__ node_begin, unsigned long long *__restrict__ count,
                                    int32_t *status) {
    const int64_t total = n * T;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t t = (int32_t)(i % T);
        const int32_t v = leaf[i];
        const int64_t b = node_begin[t];
        if (v < 0 || b + v >= node_begin[t + 1]) {  // not a node of tree t
            atomicCAS(status, 0, FP_EDEVICE);
            continue;
        }
        atomicAdd(count + b + v, 1ull);
    }
}

}  // namespace

extern "C" int fp_count_leaves(const int32_t *out_leaf, int64_t n, int32_t n_trees, const int64_t *node_begin,
                               int64_t *leaf_count, int32_t *status, void *stream) {
    if (n < 0 || n_trees < 1 || (n > 0 && (!out_leaf || !node_begin || !leaf_count || !status))) {
        fp_set_error("fp_count_leaves: bad arguments");
        return FP_EINVAL;
    }
    if (n == 0) return FP_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int device = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) {
        count_leaves_kernel<<<sms * 8, 256, 0, s>>>(out_leaf, n, n_trees, node_begin,
                                                   reinterpret_cast<unsigned long long *>(leaf_count), status);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        fp_set_error("fp_count_leaves: %s", cudaGetErrorString(e));
        return FP_ECUDA;
    }
    return FP_OK;
}
