// fp_device.cu -- resident forests and the classification entry points.
//
// fp_upload copies a packed image to the device; fp_predict launches the
// persistent traversal kernel (fp_traverse.cuh) on the caller's stream.  The
// kernel needs scratch memory only when a forest is swept in several passes
// (a vote accumulator when the caller asks for classes only, and one counter
// per observation tile); that scratch comes from a library-owned
// stream-ordered memory pool, so calls on different streams never share it.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/forest_pack.h"
#include "fp_common.h"
#include "fp_internal.h"
#include "fp_traverse.cuh"

struct fp_device_forest {
    int device = -1;
    FpImageHeader hdr{};
    std::vector<FpBin> bins;
    std::vector<FpPass> passes;
    uint8_t *d_image = nullptr;
    int32_t *d_status = nullptr;
    int32_t R = 0;            // observation tile actually launched (fits shared memory)
    int32_t threads = 0;
    int32_t refill = 8;
    int32_t head_smem = 0;
    int32_t nbuf = 3;                          // bin-block buffers
    size_t smem_votes = 0, smem_leaves = 0, smem_values = 0;
    int32_t grid_votes = 0, grid_leaves = 0, grid_values = 0;  // resident CTAs for a persistent launch
    int32_t spin_limit = FP_SPIN_LIMIT;       // fault injection may lower it
    int32_t stall = 0;                        // fault injection: bin waits run out
};

namespace {

std::mutex g_pool_mu;
std::vector<int> g_pool_ready;
std::atomic<int64_t> g_fail_allocs{0};  // fault injection: device allocations still to fail

// true when fault injection takes this allocation
bool injected_alloc_failure(const char *what) {
    int64_t k = g_fail_allocs.load();
    while (k > 0 && !g_fail_allocs.compare_exchange_weak(k, k - 1)) {
    }
    if (k <= 0) return false;
    fp_set_error("%s: injected allocation failure", what);
    return true;
}

int cuda_fail(cudaError_t e, const char *what) {
    fp_set_error("%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? FP_ENOMEM : FP_ECUDA;
}

// Per-call scratch comes from the device's stream-ordered memory pool
// (cudaMallocAsync), which CUDA-graph capture turns into graph memory nodes.
// The first use on a device keeps freed blocks in the pool between calls.
int scratch_alloc(int device, void **out, size_t bytes, cudaStream_t s) {
    {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        if ((int)g_pool_ready.size() <= device) g_pool_ready.resize((size_t)device + 1, 0);
        if (!g_pool_ready[device]) {
            cudaMemPool_t pool;
            cudaError_t e = cudaDeviceGetDefaultMemPool(&pool, device);
            if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetDefaultMemPool");
            uint64_t keep = UINT64_MAX;
            e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemPoolSetAttribute");
            g_pool_ready[device] = 1;
        }
    }
    if (injected_alloc_failure("cudaMallocAsync(scratch)")) return FP_ENOMEM;
    cudaError_t e = cudaMallocAsync(out, bytes, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync(scratch)");
    return FP_OK;
}

// rows tile (feature-major) + nbuf bin blocks + votes + per-warp task rings
size_t smem_bytes(int R, int F, int head_smem, int nbuf, int C, int warps, bool leaves) {
    const size_t xs = ((size_t)R * F * 4 + 15) & ~(size_t)15;
    const size_t votes = leaves ? 0 : (((size_t)R * C * 4 + 15) & ~(size_t)15);
    return xs + (size_t)nbuf * (size_t)head_smem + votes + (size_t)warps * FP_RING * 8;
}

// The kernel variant for a forest and block size: its kind of super-node
// (two levels, three of format 1 or 2), and up to 768 threads run the build
// for several CTAs per SM (<= 42 registers), larger blocks the one-CTA build ...
template <int MODE, int DK, int HK>
void (*traverse_kernel_sized(const fp_device_forest *f))(TravParams) {
    return f->threads <= 768 ? fp_traverse_kernel<MODE, 2, DK, HK> : fp_traverse_kernel<MODE, 1, DK, HK>;
}

// ... and its head kind (compiled in: 0 ranked, 1 level slots, 2 paired).
template <int MODE, int DK>
void (*traverse_kernel_deep(const fp_device_forest *f))(TravParams) {
    switch (f->hdr.head_select) {
        case 1: return traverse_kernel_sized<MODE, DK, 1>(f);
        case 2: return traverse_kernel_sized<MODE, DK, 2>(f);
        default: return traverse_kernel_sized<MODE, DK, 0>(f);
    }
}

// The kernel's super-node kind of a packed header: 2, 3 (format 1) or 4 (format 2).
int deep_kind(const FpImageHeader &h) { return h.deep_levels != 3 ? 2 : (h.deep_format == 2 ? 4 : 3); }

template <int MODE>
void (*traverse_kernel(const fp_device_forest *f))(TravParams) {
    switch (deep_kind(f->hdr)) {
        case 3: return traverse_kernel_deep<MODE, 3>(f);
        case 4: return traverse_kernel_deep<MODE, 4>(f);
        default: return traverse_kernel_deep<MODE, 2>(f);
    }
}

// Every instance of the batched kernel: super-node kind (0 mixed, 2, 3, 4) x
// head kind (-1 mixed, 0 ranked, 1, 2).
template <int KIND>
void add_batched(std::vector<void (*)(BatchParams)> &v) {
    v.push_back(fp_traverse_batched_kernel<KIND, -1>);
    v.push_back(fp_traverse_batched_kernel<KIND, 0>);
    v.push_back(fp_traverse_batched_kernel<KIND, 1>);
    v.push_back(fp_traverse_batched_kernel<KIND, 2>);
}

const std::vector<void (*)(BatchParams)> &batched_kernels() {
    static const std::vector<void (*)(BatchParams)> v = [] {
        std::vector<void (*)(BatchParams)> k;
        add_batched<0>(k);
        add_batched<2>(k);
        add_batched<3>(k);
        add_batched<4>(k);
        return k;
    }();
    return v;
}

// The instance for a launch: index 4 * kind + (head kind + 1) into batched_kernels().
void (*batched_kernel(int kind, int hk))(BatchParams) {
    const int ki = kind >= 2 ? kind - 1 : 0;  // 0 mixed, 1 two levels, 2 format 1, 3 format 2
    return batched_kernels()[(size_t)(4 * ki + (hk + 1))];
}

// The dynamic shared-memory limit is an attribute of the kernel instance,
// which every resident forest of the same kind of super-node, head kind and
// CTA size shares: it is raised to the device's whole budget (a limit, not a
// reservation; each launch asks for its own forest's bytes), so configuring
// one forest never lowers it below another's need.  The grid comes from the
// occupancy at this forest's own bytes.
template <int MODE>
int configure(fp_device_forest *f, size_t smem, size_t budget, int32_t *grid) {
    auto kern = traverse_kernel<MODE>(f);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)budget);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, f->threads, smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    if (per_sm < 1) {
        fp_set_error("traversal kernel does not fit on an SM (%zu bytes of shared memory)", smem);
        return FP_EUNSUPPORTED;
    }
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, f->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    *grid = per_sm * sms;
    return FP_OK;
}

// Fit the observation tile to shared memory and size the persistent grid.
int launch_setup(fp_device_forest *f, int32_t tile, int32_t warps, int32_t refill, int32_t nbuf) {
    if (tile < 32 || tile > 2048 || tile % 32 || warps < 1 || warps > 32 || refill < 1 || refill > 32 ||
        (nbuf != 2 && nbuf != 3)) {
        fp_set_error("launch parameters out of range (obs_tile %d, warps %d, refill %d, bin_buffers %d)", tile, warps,
                     refill, nbuf);
        return FP_EINVAL;
    }
    int max_optin = 0;
    cudaError_t e = cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, f->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    const size_t budget = (size_t)max_optin - 256;  // leaves room for the static shared variables
    const int C = f->hdr.n_classes, F = f->hdr.n_features;
    int R = tile;
    while (R > 32 && smem_bytes(R, F, f->head_smem, nbuf, C, warps, false) > budget) R -= 32;
    if (smem_bytes(R, F, f->head_smem, nbuf, C, warps, false) > budget) {
        fp_set_error("a 32-row tile, the bin-block buffers and the task rings need %zu bytes of shared memory (limit %zu)",
                     smem_bytes(R, F, f->head_smem, nbuf, C, warps, false), budget);
        return FP_EUNSUPPORTED;
    }
    fp_device_forest g = *f;
    g.R = R;
    g.threads = 32 * warps;
    g.refill = refill;
    g.nbuf = nbuf;
    g.smem_votes = smem_bytes(R, F, f->head_smem, nbuf, C, warps, false);
    g.smem_leaves = smem_bytes(R, F, f->head_smem, nbuf, C, warps, true);
    int rc = configure<FP_MODE_VOTES>(&g, g.smem_votes, budget, &g.grid_votes);
    if (rc) return rc;
    rc = configure<FP_MODE_LEAVES>(&g, g.smem_leaves, budget, &g.grid_leaves);
    if (rc) return rc;
    if (f->hdr.n_values > 0) {  // one float per row instead of the class votes
        g.smem_values = smem_bytes(R, F, f->head_smem, nbuf, 1, warps, false);
        rc = configure<FP_MODE_VALUES>(&g, g.smem_values, budget, &g.grid_values);
        if (rc) return rc;
    }
    // the batched kernels may host any resident forest: allow them all of shared memory
    for (auto kern : batched_kernels()) {
        cudaError_t e2 = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)budget);
        if (e2 != cudaSuccess) return cuda_fail(e2, "cudaFuncSetAttribute(batched)");
    }
    f->R = g.R;
    f->threads = g.threads;
    f->refill = g.refill;
    f->nbuf = g.nbuf;
    f->smem_votes = g.smem_votes;
    f->smem_leaves = g.smem_leaves;
    f->grid_votes = g.grid_votes;
    f->grid_leaves = g.grid_leaves;
    f->smem_values = g.smem_values;
    f->grid_values = g.grid_values;
    return FP_OK;
}

TravParams base_params(const fp_device_forest *f, const float *X, int64_t n) {
    TravParams p;
    memset(&p, 0, sizeof p);
    const FpImageHeader &h = f->hdr;
    p.deep = reinterpret_cast<const FpSuper *>(f->d_image + h.off_deep);
    p.heads = f->d_image + h.off_heads;
    p.bins = reinterpret_cast<const FpBin *>(f->d_image + h.off_bins);
    p.passes = reinterpret_cast<const FpPass *>(f->d_image + h.off_passes);
    p.pheads = reinterpret_cast<const int32_t *>(f->d_image + h.off_pheads);
    p.deep_leaf = reinterpret_cast<const int32_t *>(f->d_image + h.off_deep_leaf);
    p.X = X;
    p.n = n;
    p.F = h.n_features;
    p.C = h.n_classes;
    p.T = h.n_trees;
    // A small batch gets smaller tiles, so that its (pass, tile) items still
    // reach every resident CTA; shared memory is laid out for f->R rows and a
    // smaller tile (a multiple of 32) fits in it.
    int32_t R = f->R;
    const int64_t grid = std::max<int64_t>(1, f->grid_votes);
    const int64_t want = (n * std::max<int32_t>(1, h.n_passes) + grid - 1) / grid;  // rows per tile
    if (want < R) R = (int32_t)std::max<int64_t>(32, (want + 31) / 32 * 32);
    p.R = R;
    p.n_tiles = (n + R - 1) / R;
    p.head_smem = f->head_smem;
    p.nbuf = f->nbuf;
    p.levels = h.head_select == 3 ? 0 : h.head_select;  // kernel: 0 ranked, 1 level slots, 2 paired
    p.leaf_val = reinterpret_cast<const float *>(f->d_image + h.off_values);
    p.n_vals = (uint32_t)h.n_values;
    p.depth = h.depth;
    p.refill = f->refill;
    p.status = f->d_status;
    p.spin_limit = f->spin_limit;
    p.stall = f->stall;
    p.n_super = h.n_super;
    p.deep_kind = deep_kind(h);
    if (p.deep_kind >= 3) {
        p.fbits = (uint32_t)h.feature_bits;
        p.cbits = (uint32_t)h.class_bits;
        p.sh2 = (p.deep_kind == 4 ? 1 : 2) * p.fbits + 2 * p.cbits;
        p.klo = h.key_lo;
        p.khi = h.key_hi;
        p.kshl = h.key_shl;
        p.kflag = h.key_flag;
        p.kga = h.key_gap_a;
        p.kgb = h.key_gap_b;
        p.kgd = h.key_gap_d;
        p.fmask = (1u << p.fbits) - 1u;
        p.cmask = (1u << p.cbits) - 1u;
        p.vbase3 = (uint32_t)h.values3_base;
        p.deep_keys = reinterpret_cast<const uint32_t *>(f->d_image + h.off_deep_keys);
    }
    return p;
}

int check_device(const fp_device_forest *f) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != f->device) {
        fp_set_error("forest lives on device %d but device %d is current", f->device, dev);
        return FP_EINVAL;
    }
    return FP_OK;
}

}  // namespace

extern "C" int fp_upload(const fp_packed_forest *pf, void *stream, fp_device_forest **out) {
    if (!out || !pf) {
        fp_set_error("fp_upload: NULL argument");
        return FP_EINVAL;
    }
    *out = nullptr;
    fp_device_forest *f = new (std::nothrow) fp_device_forest;
    if (!f) {
        fp_set_error("fp_upload: out of host memory");
        return FP_ENOMEM;
    }
    const FpImageHeader *h = fp_packed_header(pf);
    f->hdr = *h;
    const uint8_t *img = fp_packed_bytes(pf);
    f->bins.assign(reinterpret_cast<const FpBin *>(img + h->off_bins),
                   reinterpret_cast<const FpBin *>(img + h->off_bins) + h->n_bins);
    f->passes.assign(reinterpret_cast<const FpPass *>(img + h->off_passes),
                     reinterpret_cast<const FpPass *>(img + h->off_passes) + h->n_passes);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int rc = FP_OK;
    cudaError_t e = cudaGetDevice(&f->device);
    if (e != cudaSuccess) { rc = cuda_fail(e, "cudaGetDevice"); goto fail; }
    if (injected_alloc_failure("cudaMalloc(image)")) { rc = FP_ENOMEM; goto fail; }
    e = cudaMalloc(&f->d_image, (size_t)h->total_bytes);
    if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMalloc(image)"); goto fail; }
    e = cudaMalloc(&f->d_status, 256);
    if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMalloc(status)"); goto fail; }
    e = cudaMemsetAsync(f->d_status, 0, 256, s);
    if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMemsetAsync"); goto fail; }
    e = cudaMemcpyAsync(f->d_image, img, (size_t)h->total_bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMemcpyAsync(image)"); goto fail; }
    e = cudaStreamSynchronize(s);  // the caller may free the host image on return
    if (e != cudaSuccess) { rc = cuda_fail(e, "cudaStreamSynchronize"); goto fail; }
    f->head_smem = (h->max_head_bytes + 15) & ~15;
    rc = launch_setup(f, h->obs_tile, h->warps_per_cta, h->refill_lanes, h->bin_buffers);
    if (rc) goto fail;
    *out = f;
    return FP_OK;
fail:
    if (f->d_image) cudaFree(f->d_image);
    if (f->d_status) cudaFree(f->d_status);
    delete f;
    return rc;
}

extern "C" int fp_configure(fp_device_forest *f, const fp_pack_params *params) {
    if (!f || !params) {
        fp_set_error("fp_configure: NULL argument");
        return FP_EINVAL;
    }
    const FpImageHeader &h = f->hdr;
    if ((params->bin_size && params->bin_size != h.bin_size) ||
        (params->interleave_depth > 0 && params->interleave_depth != h.depth) ||
        (params->pass_bytes && params->pass_bytes != h.pass_bytes)) {
        fp_set_error("fp_configure: layout parameters can only change by packing again");
        return FP_EINVAL;
    }
    int rc = check_device(f);
    if (rc) return rc;
    return launch_setup(f, params->obs_tile ? params->obs_tile : f->R,
                        params->warps_per_cta ? params->warps_per_cta : f->threads / 32,
                        params->refill_lanes ? params->refill_lanes : f->refill,
                        params->bin_buffers ? params->bin_buffers : f->nbuf);
}

extern "C" int fp_predict(const fp_device_forest *f, const float *X, int64_t n, uint32_t *out_votes,
                          int32_t *out_class, void *stream) {
    if (!f || n < 0 || (n > 0 && !X)) {
        fp_set_error("fp_predict: bad arguments");
        return FP_EINVAL;
    }
    if (f->hdr.n_values > 0) {
        fp_set_error("fp_predict: the forest has leaf values; use fp_predict_values");
        return FP_EINVAL;
    }
    if (n == 0 || (!out_votes && !out_class)) return FP_OK;
    int rc = check_device(f);
    if (rc) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const FpImageHeader &h = f->hdr;
    TravParams p = base_params(f, X, n);
    p.n_passes = h.n_passes;
    p.n_items = p.n_tiles * h.n_passes;
    p.out_votes = out_votes;
    p.out_class = out_class;
    void *scratch = nullptr;
    cudaError_t e;
    if (h.n_passes > 1) {
        const size_t vote_bytes = out_votes ? 0 : (size_t)n * h.n_classes * 4;
        const size_t cnt_bytes = out_class ? (size_t)p.n_tiles * 4 : 0;
        const size_t bytes = ((vote_bytes + 255) & ~(size_t)255) + cnt_bytes;
        if (bytes) {
            rc = scratch_alloc(f->device, &scratch, bytes, s);
            if (rc) return rc;
            e = cudaMemsetAsync(scratch, 0, bytes, s);
            if (e != cudaSuccess) { cudaFreeAsync(scratch, s); return cuda_fail(e, "cudaMemsetAsync(scratch)"); }
        }
        uint8_t *sc = static_cast<uint8_t *>(scratch);
        p.acc = out_votes ? out_votes : reinterpret_cast<uint32_t *>(sc);
        p.tile_done = reinterpret_cast<uint32_t *>(sc + ((vote_bytes + 255) & ~(size_t)255));
        if (out_votes) {
            e = cudaMemsetAsync(out_votes, 0, (size_t)n * h.n_classes * 4, s);
            if (e != cudaSuccess) {
                if (scratch) cudaFreeAsync(scratch, s);
                return cuda_fail(e, "cudaMemsetAsync(out_votes)");
            }
        }
    }
    const int64_t grid = std::min<int64_t>(p.n_items, f->grid_votes);
    traverse_kernel<FP_MODE_VOTES>(f)<<<(unsigned)grid, f->threads, f->smem_votes, s>>>(p);
    e = cudaGetLastError();
    if (scratch) cudaFreeAsync(scratch, s);
    if (e != cudaSuccess) return cuda_fail(e, "fp_traverse_kernel launch");
    return FP_OK;
}

extern "C" int fp_predict_values(const fp_device_forest *f, const float *X, int64_t n, float scale, float bias,
                                 float *out, void *stream) {
    if (!f || n < 0 || (n > 0 && (!X || !out))) {
        fp_set_error("fp_predict_values: bad arguments");
        return FP_EINVAL;
    }
    if (f->hdr.n_values <= 0) {
        fp_set_error("fp_predict_values: the forest was packed without leaf values");
        return FP_EINVAL;
    }
    if (n == 0) return FP_OK;
    int rc = check_device(f);
    if (rc) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const FpImageHeader &h = f->hdr;
    TravParams p = base_params(f, X, n);
    p.n_passes = h.n_passes;
    p.n_items = p.n_tiles * h.n_passes;
    p.vscale = scale;
    p.vbias = bias;
    p.out_val = out;
    void *scratch = nullptr;
    cudaError_t e;
    if (h.n_passes > 1) {  // a float accumulator per row and a counter per tile
        const size_t acc_bytes = ((size_t)n * 4 + 255) & ~(size_t)255;
        const size_t bytes = acc_bytes + (size_t)p.n_tiles * 4;
        rc = scratch_alloc(f->device, &scratch, bytes, s);
        if (rc) return rc;
        e = cudaMemsetAsync(scratch, 0, bytes, s);
        if (e != cudaSuccess) { cudaFreeAsync(scratch, s); return cuda_fail(e, "cudaMemsetAsync(scratch)"); }
        uint8_t *sc = static_cast<uint8_t *>(scratch);
        p.acc_val = reinterpret_cast<float *>(sc);
        p.tile_done = reinterpret_cast<uint32_t *>(sc + acc_bytes);
    }
    const int64_t grid = std::min<int64_t>(p.n_items, f->grid_values);
    traverse_kernel<FP_MODE_VALUES>(f)<<<(unsigned)grid, f->threads, f->smem_values, s>>>(p);
    e = cudaGetLastError();
    if (scratch) cudaFreeAsync(scratch, s);
    if (e != cudaSuccess) return cuda_fail(e, "fp_traverse_kernel<values> launch");
    return FP_OK;
}

// ---------------------------------------------------------------------------
// fp_predict_noalloc: fp_predict for callers that must not allocate device
// memory.  The scratch that a forest swept in several passes needs (a vote
// accumulator when no votes buffer is given, one counter per observation
// tile when classes are asked for) lives in this fixed array instead of the
// stream-ordered pool.  Every GPU that loads the library holds the array
// until the process exits.
#define FP_NOALLOC_SCRATCH_BYTES (16u << 20)
static __device__ __align__(256) unsigned char fp_noalloc_scratch[FP_NOALLOC_SCRATCH_BYTES];

namespace {
std::mutex g_noalloc_mu;
std::vector<void *> g_noalloc_ptr;  // device address of the array, per device (set up once)

// Host code cannot use the array's name as a device address: look the
// address up once per device, with that device current.
int noalloc_scratch(int device, void **out) {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if ((int)g_noalloc_ptr.size() <= device) g_noalloc_ptr.resize((size_t)device + 1, nullptr);
    if (!g_noalloc_ptr[device]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, fp_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(fp_noalloc_scratch)");
        g_noalloc_ptr[device] = ptr;
    }
    *out = g_noalloc_ptr[device];
    return FP_OK;
}
}  // namespace

extern "C" int fp_predict_noalloc(const fp_device_forest *f, const float *X, int64_t n, uint32_t *out_votes,
                                  int32_t *out_class, void *stream) {
    if (!f || n < 0 || (n > 0 && !X)) {
        fp_set_error("fp_predict_noalloc: bad arguments");
        return FP_EINVAL;
    }
    if (f->hdr.n_values > 0) {
        fp_set_error("fp_predict_noalloc: the forest has leaf values; use fp_predict_values");
        return FP_EINVAL;
    }
    if (n == 0 || (!out_votes && !out_class)) return FP_OK;
    int rc = check_device(f);
    if (rc) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const FpImageHeader &h = f->hdr;
    TravParams p = base_params(f, X, n);
    p.n_passes = h.n_passes;
    p.n_items = p.n_tiles * h.n_passes;
    p.out_votes = out_votes;
    p.out_class = out_class;
    cudaError_t e;
    if (h.n_passes > 1) {
        const size_t vote_bytes = out_votes ? 0 : (size_t)n * h.n_classes * 4;
        const size_t cnt_bytes = out_class ? (size_t)p.n_tiles * 4 : 0;
        const size_t bytes = ((vote_bytes + 255) & ~(size_t)255) + cnt_bytes;
        if (bytes > FP_NOALLOC_SCRATCH_BYTES) {
            fp_set_error("fp_predict_noalloc: %lld rows need %zu bytes of scratch, more than the fixed %u; pass "
                         "out_votes, split the batch, or use fp_predict",
                         (long long)n, bytes, FP_NOALLOC_SCRATCH_BYTES);
            return FP_EINVAL;
        }
        void *scratch = nullptr;
        rc = noalloc_scratch(f->device, &scratch);
        if (rc) return rc;
        if (bytes) {
            e = cudaMemsetAsync(scratch, 0, bytes, s);  // the last call's counts must not leak in
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(noalloc scratch)");
        }
        uint8_t *sc = static_cast<uint8_t *>(scratch);
        p.acc = out_votes ? out_votes : reinterpret_cast<uint32_t *>(sc);
        p.tile_done = reinterpret_cast<uint32_t *>(sc + ((vote_bytes + 255) & ~(size_t)255));
        if (out_votes) {
            e = cudaMemsetAsync(out_votes, 0, (size_t)n * h.n_classes * 4, s);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(out_votes)");
        }
    }
    const int64_t grid = std::min<int64_t>(p.n_items, f->grid_votes);
    traverse_kernel<FP_MODE_VOTES>(f)<<<(unsigned)grid, f->threads, f->smem_votes, s>>>(p);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "fp_traverse_kernel launch");
    return FP_OK;
}

extern "C" int fp_predict_leaves(const fp_device_forest *f, const float *X, int64_t n, int32_t *out_leaf,
                                 void *stream) {
    if (!f || n < 0 || (n > 0 && (!X || !out_leaf))) {
        fp_set_error("fp_predict_leaves: bad arguments");
        return FP_EINVAL;
    }
    if (n == 0) return FP_OK;
    int rc = check_device(f);
    if (rc) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    TravParams p = base_params(f, X, n);
    p.n_passes = f->hdr.n_passes;
    p.n_items = p.n_tiles * f->hdr.n_passes;
    p.out_leaf = out_leaf;
    const int64_t grid = std::min<int64_t>(p.n_items, f->grid_leaves);
    traverse_kernel<FP_MODE_LEAVES>(f)<<<(unsigned)grid, f->threads, f->smem_leaves, s>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "fp_traverse_kernel<leaves> launch");
    return FP_OK;
}

extern "C" int fp_sync_status(const fp_device_forest *f, void *stream) {
    if (!f) {
        fp_set_error("fp_sync_status: NULL forest");
        return FP_EINVAL;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    int32_t word = 0;
    e = cudaMemcpy(&word, f->d_status, 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(status)");
    if (word != 0) {
        e = cudaMemset(f->d_status, 0, 4);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemset(status)");
        fp_set_error("a kernel reported status %d", word);
        return word < 0 ? word : FP_EDEVICE;
    }
    return FP_OK;
}

extern "C" int fp_inject_fault(fp_device_forest *f, int32_t kind, int64_t value) {
    switch (kind) {
    case FP_FAULT_ALLOC:
        if (value < 0) break;
        g_fail_allocs.store(value);
        return FP_OK;
    case FP_FAULT_WAIT_LIMIT:
        if (!f || value < 1 || value > FP_SPIN_LIMIT) break;
        f->spin_limit = (int32_t)value;
        return FP_OK;
    case FP_FAULT_STALL_BIN_COPY:
        if (!f || (value != 0 && value != 1)) break;
        f->stall = (int32_t)value;
        return FP_OK;
    default:
        break;
    }
    fp_set_error("fp_inject_fault: bad kind %d, value %lld or forest", kind, (long long)value);
    return FP_EINVAL;
}

extern "C" int fp_device_info_get(const fp_device_forest *f, fp_packed_info *info) {
    if (!f || !info) {
        fp_set_error("fp_device_info_get: NULL argument");
        return FP_EINVAL;
    }
    fp_fill_info(&f->hdr, info);
    info->obs_tile = f->R;
    info->warps_per_cta = f->threads / 32;
    info->refill_lanes = f->refill;
    info->bin_buffers = f->nbuf;
    return FP_OK;
}

extern "C" void fp_release(fp_device_forest *f) {
    if (!f) return;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != f->device) cudaSetDevice(f->device);
    cudaDeviceSynchronize();
    cudaFree(f->d_image);
    cudaFree(f->d_status);
    if (prev >= 0 && prev != f->device) cudaSetDevice(prev);
    delete f;
}

// One persistent launch over up to FP_MAX_BATCH (forest, batch) pairs.
static int predict_batched_chunk(const fp_device_forest *const *forests, const fp_batch *batches, int32_t k,
                                 cudaStream_t s) {
    int device = -1;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    int max_optin = 0;
    e = cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    const size_t budget = (size_t)max_optin - 256;
    int warps = 1;
    for (int32_t j = 0; j < k; ++j) warps = std::max(warps, forests[j]->threads / 32);

    BatchParams bp;
    memset(&bp, 0, sizeof bp);
    size_t smem = 0;
    size_t scratch_bytes = 256;  // the work counter, then per-batch accumulators and tile counters
    std::vector<size_t> acc_off((size_t)k, 0), cnt_off((size_t)k, 0);
    int32_t m = 0;
    for (int32_t j = 0; j < k; ++j) {
        const fp_device_forest *f = forests[j];
        const fp_batch &bt = batches[j];
        if (bt.n == 0 || (!bt.out_votes && !bt.out_class)) continue;
        const FpImageHeader &h = f->hdr;
        int R = f->R;
        while (R > 32 && smem_bytes(R, h.n_features, f->head_smem, f->nbuf, h.n_classes, warps, false) > budget) R -= 32;
        const size_t need = smem_bytes(R, h.n_features, f->head_smem, f->nbuf, h.n_classes, warps, false);
        if (need > budget) {
            fp_set_error("fp_predict_batched: batch %d does not fit shared memory with %d warps", j, warps);
            return FP_EUNSUPPORTED;
        }
        smem = std::max(smem, need);
        TravParams p = base_params(f, bt.X, bt.n);
        p.R = R;
        p.n_tiles = (bt.n + R - 1) / R;
        p.n_passes = h.n_passes;
        p.n_items = p.n_tiles * h.n_passes;
        p.out_votes = bt.out_votes;
        p.out_class = bt.out_class;
        if (h.n_passes > 1) {
            if (!bt.out_votes) {
                acc_off[j] = scratch_bytes;
                scratch_bytes += ((size_t)bt.n * h.n_classes * 4 + 255) & ~(size_t)255;
            }
            if (bt.out_class) {
                cnt_off[j] = scratch_bytes;
                scratch_bytes += ((size_t)p.n_tiles * 4 + 255) & ~(size_t)255;
            }
        }
        bp.p[m] = p;
        acc_off[m] = acc_off[j];
        cnt_off[m] = cnt_off[j];
        bp.item_begin[m + 1] = bp.item_begin[m] + p.n_items;
        ++m;
    }
    bp.k = m;
    if (m == 0) return FP_OK;
    void *scratch = nullptr;
    int rc = scratch_alloc(device, &scratch, scratch_bytes, s);
    if (rc) return rc;
    uint8_t *sc = static_cast<uint8_t *>(scratch);
    e = cudaMemsetAsync(scratch, 0, scratch_bytes, s);
    for (int32_t j = 0; j < m && e == cudaSuccess; ++j) {
        TravParams &p = bp.p[j];
        if (p.n_passes > 1) {
            p.acc = p.out_votes ? p.out_votes : reinterpret_cast<uint32_t *>(sc + acc_off[j]);
            if (p.out_class) p.tile_done = reinterpret_cast<uint32_t *>(sc + cnt_off[j]);
            if (p.out_votes) e = cudaMemsetAsync(p.out_votes, 0, (size_t)p.n * p.C * 4, s);
        }
    }
    bp.work = reinterpret_cast<unsigned long long *>(sc);
    // one walk compiled in when every forest has the same kind of super-node,
    // and the head kind when every forest has the same one
    int dk = bp.p[0].deep_kind, hk = bp.p[0].levels;
    for (int32_t j = 0; j < m; ++j) {
        if (bp.p[j].deep_kind != dk) dk = 0;
        if (bp.p[j].levels != hk) hk = -1;
    }
    void (*kern)(BatchParams) = batched_kernel(dk, hk);
    int per_sm = 0, sms = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * warps, smem);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) {
        const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(bp.item_begin[m], (int64_t)per_sm * sms));
        kern<<<(unsigned)grid, 32 * warps, smem, s>>>(bp);
        e = cudaGetLastError();
    }
    cudaFreeAsync(scratch, s);
    if (e != cudaSuccess) return cuda_fail(e, "fp_predict_batched");
    return FP_OK;
}

extern "C" int fp_predict_batched(const fp_device_forest *const *forests, const fp_batch *batches, int32_t k,
                                  void *stream) {
    if (k < 0 || (k > 0 && (!forests || !batches))) {
        fp_set_error("fp_predict_batched: bad arguments");
        return FP_EINVAL;
    }
    for (int32_t i = 0; i < k; ++i) {
        if (!forests[i] || batches[i].n < 0 || (batches[i].n > 0 && !batches[i].X)) {
            fp_set_error("fp_predict_batched: bad batch %d", i);
            return FP_EINVAL;
        }
        if (forests[i]->hdr.n_values > 0) {
            fp_set_error("fp_predict_batched: forest %d has leaf values; use fp_predict_values", i);
            return FP_EINVAL;
        }
        int rc = check_device(forests[i]);
        if (rc) return rc;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    for (int32_t i = 0; i < k; i += FP_MAX_BATCH) {
        int rc = predict_batched_chunk(forests + i, batches + i, std::min<int32_t>(FP_MAX_BATCH, k - i), s);
        if (rc) return rc;
    }
    return FP_OK;
}

// ------------------------------------------------- host buffers, pipelined

namespace {

std::mutex g_copy_mu;
// per device, created on first use, kept for the process: [0] the copy
// stream, [1] a second stream for every other chunk's kernel
std::vector<cudaStream_t> g_lib_stream[2];

int lib_stream(int device, int which, cudaStream_t *out) {
    std::lock_guard<std::mutex> lk(g_copy_mu);
    std::vector<cudaStream_t> &v = g_lib_stream[which];
    if ((int)v.size() <= device) v.resize((size_t)device + 1, nullptr);
    if (!v[device]) {
        cudaError_t e = cudaStreamCreateWithFlags(&v[device], cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            v[device] = nullptr;
            return cuda_fail(e, which ? "cudaStreamCreateWithFlags(compute)" : "cudaStreamCreateWithFlags(copy)");
        }
    }
    *out = v[device];
    return FP_OK;
}

// Rows from host memory through the device in chunks (eight by default):
// chunk c's rows are copied in on the library's copy stream into one of two
// device buffers while earlier chunks are classified; the chunks of buffer 0
// are classified on the caller's stream and those of buffer 1 on a second
// library stream, so that a chunk's kernel starts on the SMs that the
// previous chunk's kernel has left, instead of after its last CTA; each
// chunk's outputs are copied back on its kernel's stream.  The caller's
// stream waits for the second one before the buffers are released, so all
// the work is ordered before whatever the caller enqueues next.  out_bytes:
// bytes of output per row (one region per output); run(Xd, rows, outs,
// stream) launches the chunk's classification on `stream`.
template <class Run>
int pipeline_host(const fp_device_forest *f, const float *X_host, int64_t n, int64_t chunk_rows,
                  const int64_t out_bytes[2], void *const out_host[2], cudaStream_t s, const char *what, Run run) {
    const int64_t F = f->hdr.n_features;
    const int64_t chunk = std::min<int64_t>(n, chunk_rows > 0 ? chunk_rows : std::max<int64_t>(65536, (n + 7) / 8));
    const int nbuf = n > chunk ? 2 : 1;
    auto align = [](int64_t b) { return (b + 255) & ~(int64_t)255; };
    const int64_t in_b = align(chunk * F * 4), o0 = align(chunk * out_bytes[0]), o1 = align(chunk * out_bytes[1]);
    const int64_t per_buf = in_b + o0 + o1;
    cudaStream_t cs = nullptr, s2 = nullptr;
    int rc = lib_stream(f->device, 0, &cs);
    if (rc == FP_OK && nbuf == 2) rc = lib_stream(f->device, 1, &s2);
    if (rc) return rc;
    void *block = nullptr;
    rc = scratch_alloc(f->device, &block, (size_t)(nbuf * per_buf), s);
    if (rc) return rc;
    cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};  // ready, in[2], free[2], s2 done
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 6 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev[0], s);  // the block is allocated; earlier work on s is ordered
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev[0], 0);
    if (e == cudaSuccess && s2) e = cudaStreamWaitEvent(s2, ev[0], 0);
    bool s2_used = false;
    uint8_t *base = static_cast<uint8_t *>(block);
    for (int64_t c = 0, r0 = 0; e == cudaSuccess && rc == FP_OK && r0 < n; ++c, r0 += chunk) {
        const int b = (int)(c % nbuf);
        cudaStream_t ks = b == 0 ? s : s2;  // the chunk's kernel and output copies
        s2_used |= b == 1;
        const int64_t rows = std::min<int64_t>(chunk, n - r0);
        uint8_t *buf = base + b * per_buf;
        if (c >= nbuf) e = cudaStreamWaitEvent(cs, ev[3 + b], 0);  // chunk c-2 is done with the buffer
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(buf, X_host + r0 * F, (size_t)(rows * F * 4), cudaMemcpyHostToDevice, cs);
        if (e == cudaSuccess) e = cudaEventRecord(ev[1 + b], cs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ks, ev[1 + b], 0);
        if (e != cudaSuccess) break;
        void *outs[2] = {out_host[0] ? buf + in_b : nullptr, out_host[1] ? buf + in_b + o0 : nullptr};
        rc = run(reinterpret_cast<const float *>(buf), rows, outs, ks);
        for (int k = 0; k < 2 && rc == FP_OK && e == cudaSuccess; ++k)
            if (out_host[k])
                e = cudaMemcpyAsync(static_cast<uint8_t *>(out_host[k]) + r0 * out_bytes[k], outs[k],
                                    (size_t)(rows * out_bytes[k]), cudaMemcpyDeviceToHost, ks);
        if (e == cudaSuccess) e = cudaEventRecord(ev[3 + b], ks);
    }
    if (s2_used) {  // the caller's stream covers the second stream's work, errors or not
        cudaError_t e2 = cudaEventRecord(ev[5], s2);
        if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(s, ev[5], 0);
        if (e2 != cudaSuccess) cudaStreamSynchronize(s2);
        if (e == cudaSuccess) e = e2;
    }
    if (e != cudaSuccess || rc != FP_OK) cudaStreamSynchronize(cs);  // nothing of the copy stream outlives the block
    cudaFreeAsync(block, s);
    for (int i = 0; i < 6; ++i)
        if (ev[i]) cudaEventDestroy(ev[i]);
    if (e != cudaSuccess) return cuda_fail(e, what);
    return rc;
}

}  // namespace

extern "C" int fp_predict_host(const fp_device_forest *f, const float *X_host, int64_t n, uint32_t *out_votes_host,
                               int32_t *out_class_host, int64_t chunk_rows, void *stream) {
    if (!f || n < 0 || chunk_rows < 0 || (n > 0 && !X_host)) {
        fp_set_error("fp_predict_host: bad arguments");
        return FP_EINVAL;
    }
    if (f->hdr.n_values > 0) {
        fp_set_error("fp_predict_host: the forest has leaf values; use fp_predict_values_host");
        return FP_EINVAL;
    }
    if (n == 0 || (!out_votes_host && !out_class_host)) return FP_OK;
    int rc = check_device(f);
    if (rc) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int64_t ob[2] = {4 * (int64_t)f->hdr.n_classes, 4};
    void *const oh[2] = {out_votes_host, out_class_host};
    return pipeline_host(f, X_host, n, chunk_rows, ob, oh, s, "fp_predict_host",
                         [&](const float *Xd, int64_t rows, void *const outs[2], cudaStream_t ks) {
                             return fp_predict(f, Xd, rows, static_cast<uint32_t *>(outs[0]),
                                               static_cast<int32_t *>(outs[1]), ks);
                         });
}

extern "C" int fp_predict_values_host(const fp_device_forest *f, const float *X_host, int64_t n, float scale,
                                      float bias, float *out_host, int64_t chunk_rows, void *stream) {
    if (!f || n < 0 || chunk_rows < 0 || (n > 0 && (!X_host || !out_host))) {
        fp_set_error("fp_predict_values_host: bad arguments");
        return FP_EINVAL;
    }
    if (f->hdr.n_values <= 0) {
        fp_set_error("fp_predict_values_host: the forest was packed without leaf values");
        return FP_EINVAL;
    }
    if (n == 0) return FP_OK;
    int rc = check_device(f);
    if (rc) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int64_t ob[2] = {4, 0};
    void *const oh[2] = {out_host, nullptr};
    return pipeline_host(f, X_host, n, chunk_rows, ob, oh, s, "fp_predict_values_host",
                         [&](const float *Xd, int64_t rows, void *const outs[2], cudaStream_t ks) {
                             return fp_predict_values(f, Xd, rows, scale, bias, static_cast<float *>(outs[0]), ks);
                         });
}

// ------------------------------------------- statistics from observations

// Section III-A: the cardinalities that order a tree's nodes (Stat) may be
// measured on observations instead of taken from training.  The rows go
// through fp_predict_leaves in chunks (the leaf ids of one chunk sit in
// scratch), fp_count_leaves adds them up per node on the device, and the
// counts come back to the host, where each internal node becomes the sum of
// its children (fp_cardinality_from_leaf_counts).
extern "C" int fp_infer_cardinality(const fp_device_forest *f, const fp_forest_desc *desc, const float *X, int64_t n,
                                    int64_t chunk_rows, int64_t *out_card, void *stream) {
    if (!f || !desc || !out_card || n < 0 || chunk_rows < 0 || (n > 0 && !X) || !desc->tree_node_begin) {
        fp_set_error("fp_infer_cardinality: bad arguments");
        return FP_EINVAL;
    }
    const FpImageHeader &h = f->hdr;
    if (desc->n_trees != h.n_trees || desc->n_features != h.n_features || desc->n_classes != h.n_classes) {
        fp_set_error("fp_infer_cardinality: the descriptor (%d trees, %d features, %d classes) is not the forest's "
                     "(%d, %d, %d)", desc->n_trees, desc->n_features, desc->n_classes, h.n_trees, h.n_features,
                     h.n_classes);
        return FP_EINVAL;
    }
    int64_t n_internal = 0;
    const int64_t total = desc->tree_node_begin[desc->n_trees];
    if (desc->left)
        for (int64_t v = 0; v < total; ++v) n_internal += desc->left[v] >= 0;
    if (!desc->left || n_internal != h.n_internal) {
        fp_set_error("fp_infer_cardinality: the descriptor's internal nodes do not match the packed forest's");
        return FP_EINVAL;
    }
    int rc = check_device(f);
    if (rc) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int64_t T = h.n_trees;
    const int64_t chunk = std::max<int64_t>(
        1, std::min<int64_t>(n, chunk_rows > 0 ? chunk_rows : std::max<int64_t>(1, (256 << 20) / (4 * T))));
    auto align = [](int64_t b) { return (b + 255) & ~(int64_t)255; };
    const int64_t cnt_b = align(total * 8), nb_b = align((T + 1) * 8), st_b = 256;
    const int64_t leaf_b = n > 0 ? align(chunk * T * 4) : 0;
    void *block = nullptr;
    rc = scratch_alloc(f->device, &block, (size_t)(cnt_b + nb_b + st_b + leaf_b), s);
    if (rc) return rc;
    uint8_t *base = static_cast<uint8_t *>(block);
    int64_t *d_cnt = reinterpret_cast<int64_t *>(base);
    int64_t *d_nb = reinterpret_cast<int64_t *>(base + cnt_b);
    int32_t *d_st = reinterpret_cast<int32_t *>(base + cnt_b + nb_b);
    int32_t *d_leaf = reinterpret_cast<int32_t *>(base + cnt_b + nb_b + st_b);
    int32_t st = 0;
    cudaError_t e = cudaMemsetAsync(block, 0, (size_t)(cnt_b + nb_b + st_b), s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_nb, desc->tree_node_begin, (size_t)(T + 1) * 8, cudaMemcpyHostToDevice, s);
    for (int64_t r0 = 0; e == cudaSuccess && rc == FP_OK && r0 < n; r0 += chunk) {
        const int64_t rows = std::min<int64_t>(chunk, n - r0);
        rc = fp_predict_leaves(f, X + r0 * h.n_features, rows, d_leaf, stream);
        if (rc == FP_OK) rc = fp_count_leaves(d_leaf, rows, (int32_t)T, d_nb, d_cnt, d_st, stream);
    }
    if (e == cudaSuccess && rc == FP_OK)
        e = cudaMemcpyAsync(out_card, d_cnt, (size_t)total * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && rc == FP_OK) e = cudaMemcpyAsync(&st, d_st, 4, cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(block, s);
    const cudaError_t es = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = es;
    if (rc != FP_OK) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "fp_infer_cardinality");
    if (st != 0) {
        fp_set_error("fp_infer_cardinality: a leaf id was not a node of its tree");
        return FP_EDEVICE;
    }
    rc = fp_sync_status(f, stream);  // an error the traversal kernel recorded
    if (rc) return rc;
    return fp_cardinality_from_leaf_counts(desc, out_card, out_card);
}
