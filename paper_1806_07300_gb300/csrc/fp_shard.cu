// fp_shard.cu -- the last step of tree-bin sharding (Section III binds bins
// of trees to processes): once every process has classified the same rows
// with its own bins and the per-class votes have been summed over processes
// (a collective outside the library), the class of each row is the argmax of
// the summed votes, lowest class on ties.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/forest_pack.h"
#include "fp_common.h"

namespace {

// One thread per row; a row's votes are contiguous, so consecutive threads
// read consecutive rows of C counters.
__global__ void votes_argmax_kernel(const uint32_t *__restrict__ votes, int64_t n, int32_t C,
                                    int32_t *__restrict__ out_class) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t *v = votes + i * C;
        int32_t best = 0;
        uint32_t bv = v[0];
        for (int32_t c = 1; c < C; ++c) {
            const uint32_t x = v[c];
            if (x > bv) {
                bv = x;
                best = c;
            }
        }
        out_class[i] = best;
    }
}

}  // namespace

extern "C" int fp_votes_argmax(const uint32_t *votes, int64_t n, int32_t n_classes, int32_t *out_class,
                               void *stream) {
    if (n < 0 || n_classes < 1 || n_classes > 512 || (n > 0 && (!votes || !out_class))) {
        fp_set_error("fp_votes_argmax: bad arguments");
        return FP_EINVAL;
    }
    if (n == 0) return FP_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int device = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) {
        const int64_t blocks = std::min<int64_t>((n + 255) / 256, (int64_t)sms * 8);
        votes_argmax_kernel<<<(unsigned)blocks, 256, 0, s>>>(votes, n, n_classes, out_class);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        fp_set_error("fp_votes_argmax: %s", cudaGetErrorString(e));
        return FP_ECUDA;
    }
    return FP_OK;
}
