// fp_probe.cu -- bandwidth probes that give the roofline its denominators.
//
// fp_l2_read_probe: every CTA streams a buffer small enough to stay in L2
// with 16-byte loads, `iters` times over; the achieved bytes per second is
// the L2 read bandwidth the traversal kernel can hope for.  No counterpart
// in the paper (whose roofline is a CPU cache model, Section III-A).
#include <cuda_runtime.h>

#include "../../include/forest_pack.h"
#include "fp_common.h"

namespace {

__global__ void l2_read_kernel(const uint4 *__restrict__ buf, int64_t n16, int iters, uint32_t *sink) {
    uint32_t acc = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int it = 0; it < iters; ++it) {
        // each pass starts at a different offset so CTAs do not march in step
        const int64_t shift = ((int64_t)it * 7919 * blockDim.x) % n16;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride) {
            int64_t j = i + shift;
            if (j >= n16) j -= n16;
            uint4 v;
            asm volatile("ld.global.cg.v4.u32 {%0, %1, %2, %3}, [%4];\n"
                         : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                         : "l"(buf + j));
            acc ^= v.x ^ v.y ^ v.z ^ v.w;
        }
    }
    if (acc == 0x9E3779B9u) sink[0] = acc;  // keeps the loads alive
}

}  // namespace

extern "C" int fp_l2_read_probe(const void *buf, int64_t bytes, int32_t iters, void *stream, float *out_ms) {
    if (!buf || bytes < 16 || iters < 1 || !out_ms || ((uintptr_t)buf & 15)) {
        fp_set_error("fp_l2_read_probe: bad arguments");
        return FP_EINVAL;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int device = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    uint32_t *sink = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    if (e == cudaSuccess) e = cudaMallocAsync(&sink, 16, s);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e == cudaSuccess) {
        const int64_t n16 = bytes / 16;
        l2_read_kernel<<<sms * 4, 512, 0, s>>>(static_cast<const uint4 *>(buf), n16, 1, sink);  // warm L2
        cudaEventRecord(a, s);
        l2_read_kernel<<<sms * 4, 512, 0, s>>>(static_cast<const uint4 *>(buf), n16, iters, sink);
        cudaEventRecord(b, s);
        e = cudaEventSynchronize(b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(out_ms, a, b);
    }
    if (sink) cudaFreeAsync(sink, s);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (e != cudaSuccess) {
        fp_set_error("fp_l2_read_probe: %s", cudaGetErrorString(e));
        return FP_ECUDA;
    }
    return FP_OK;
}
