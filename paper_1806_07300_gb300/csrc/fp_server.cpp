// fp_server.cpp -- the serving runtime: continuous batching of classification
// requests over resident packed forests.
//
// Requests (rows of one forest, in host memory) are queued from any thread.
// A batcher thread takes whatever has arrived, up to max_rows rows in
// arrival order, groups it by forest and issues one persistent launch over
// all the groups (fp_predict_batched), so requests of different forests and
// sizes share a launch.  Each launch uses one of `slots` slots -- a CUDA
// stream, an event, a page-locked staging buffer and a device buffer -- so up
// to `slots` launches are in flight and overlap on the device; a launch is
// admitted once a slot is free and the device reports enough free memory
// (plus a margin), else it waits for launches in flight to finish.  A
// completion thread polls each launch's event in order (bounded: 60 s),
// copies every request's classes (and votes) into the caller's buffers and
// wakes its waiters.  Latency runs from submit to completion.  A slot goes
// back into service only once everything queued on it has finished; a slot
// whose work did not finish within the limit is retired (its buffers may
// still be in use), and with no slot left in service requests are answered
// with FP_ETIMEOUT.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "../../include/forest_pack.h"
#include "fp_common.h"

using fp_clock = std::chrono::steady_clock;

struct fp_request {
    fp_server *srv;
    int32_t forest;
    const float *X;
    int64_t n;
    int32_t *out_class;
    uint32_t *out_votes;
    fp_clock::time_point t_submit, t_done;
    int status = FP_OK;
    bool done = false;
};

namespace {

struct Entry {          // one request of a launch: where its results land in the staging buffer
    fp_request *req;
    size_t class_off;   // int32 [n]
    size_t votes_off;   // uint32 [n][C], or SIZE_MAX
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    uint8_t *pin = nullptr;  // page-locked: the launch's rows, then its results
    size_t pin_cap = 0;
    uint8_t *dev = nullptr;  // device: the rows, then the results
    size_t dev_cap = 0;
    std::vector<Entry> entries;
    int status = FP_OK;
    bool retired = false;  // work on it outlived the completion poll; never reused
};

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

struct fp_server {
    int32_t device = 0;
    int64_t max_rows = 0, mem_margin = 0;
    int32_t return_votes = 0;
    double max_wait_s = 0;
    std::vector<const fp_device_forest *> forests;
    std::vector<int32_t> F, C;
    std::mutex mu;
    std::condition_variable cv_queue, cv_slot, cv_done;
    std::deque<fp_request *> queue;
    std::vector<int> free_slots;
    std::deque<int> inflight;
    std::vector<Slot> slot;
    std::thread batcher, completer;
    bool started = false, stopping = false, batcher_done = false, joined = false;
    int64_t launches = 0, rejected_for_memory = 0;
    int64_t free_override = -1;  // reported free device bytes for tests (-1: ask the device)
    double launch_timeout_s = 60.0;  // completion poll per launch
    int32_t live_slots = 0;          // slots not retired
};

namespace {

// Free device bytes as the admission test sees them.
size_t free_bytes(fp_server *s) {
    int64_t ov;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        ov = s->free_override;
    }
    if (ov >= 0) return (size_t)ov;
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return 0;
    return fr;
}

// Stage, copy, classify and copy back one batch on slot `sl`; always records
// the slot's event after whatever was queued.  Returns an FP_ status.
int launch(fp_server *s, Slot &sl, const std::vector<std::vector<fp_request *>> &groups,
           const std::vector<int32_t> &gforest) {
    const size_t k = groups.size();
    std::vector<int64_t> rows(k, 0);
    size_t in_bytes = 0, out_bytes = 0;
    for (size_t g = 0; g < k; ++g) {
        for (fp_request *r : groups[g]) rows[g] += r->n;
        const int32_t f = gforest[g];
        in_bytes += align256((size_t)rows[g] * s->F[f] * 4);
        out_bytes += align256((size_t)rows[g] * 4) + (s->return_votes ? align256((size_t)rows[g] * s->C[f] * 4) : 0);
    }
    const size_t need = in_bytes + out_bytes;
    cudaError_t e = cudaSuccess;
    if (sl.pin_cap < need) {  // the slot is idle, so its old buffers are unused
        const size_t cap = std::max(need, 2 * sl.pin_cap + ((size_t)1 << 20));
        if (sl.pin) cudaFreeHost(sl.pin);
        sl.pin = nullptr;
        sl.pin_cap = 0;
        e = cudaHostAlloc(reinterpret_cast<void **>(&sl.pin), cap, cudaHostAllocDefault);
        if (e != cudaSuccess) {
            sl.pin = nullptr;
            fp_set_error("fp_server: cudaHostAlloc(%zu): %s", cap, cudaGetErrorString(e));
            return FP_ENOMEM;
        }
        sl.pin_cap = cap;
    }
    if (sl.dev_cap < need) {  // stream-ordered, so no device-wide synchronisation
        const size_t cap = std::max(need, 2 * sl.dev_cap + ((size_t)1 << 20));
        if (sl.dev) cudaFreeAsync(sl.dev, sl.stream);
        sl.dev = nullptr;
        sl.dev_cap = 0;
        e = cudaMallocAsync(reinterpret_cast<void **>(&sl.dev), cap, sl.stream);
        if (e != cudaSuccess) {
            sl.dev = nullptr;
            cudaEventRecord(sl.ev, sl.stream);
            fp_set_error("fp_server: cudaMallocAsync(%zu): %s", cap, cudaGetErrorString(e));
            return FP_ENOMEM;
        }
        sl.dev_cap = cap;
    }
    // gather the rows group by group, and lay out the results after them
    std::vector<fp_batch> batches(k);
    std::vector<const fp_device_forest *> fl(k);
    sl.entries.clear();
    size_t in_off = 0, out_off = in_bytes;
    for (size_t g = 0; g < k; ++g) {
        const int32_t f = gforest[g];
        const size_t row_bytes = (size_t)s->F[f] * 4;
        size_t o = in_off;
        for (fp_request *r : groups[g]) {
            memcpy(sl.pin + o, r->X, (size_t)r->n * row_bytes);
            o += (size_t)r->n * row_bytes;
        }
        const size_t cls_off = out_off;
        const size_t votes_off = s->return_votes ? cls_off + align256((size_t)rows[g] * 4) : SIZE_MAX;
        int64_t r0 = 0;
        for (fp_request *r : groups[g]) {
            sl.entries.push_back({r, cls_off + (size_t)r0 * 4,
                                  s->return_votes ? votes_off + (size_t)r0 * s->C[f] * 4 : SIZE_MAX});
            r0 += r->n;
        }
        batches[g].X = reinterpret_cast<const float *>(sl.dev + in_off);
        batches[g].n = rows[g];
        batches[g].out_class = reinterpret_cast<int32_t *>(sl.dev + cls_off);
        batches[g].out_votes = s->return_votes ? reinterpret_cast<uint32_t *>(sl.dev + votes_off) : nullptr;
        fl[g] = s->forests[f];
        in_off += align256((size_t)rows[g] * row_bytes);
        out_off += align256((size_t)rows[g] * 4) + (s->return_votes ? align256((size_t)rows[g] * s->C[f] * 4) : 0);
    }
    int rc = FP_OK;
    e = cudaMemcpyAsync(sl.dev, sl.pin, in_bytes, cudaMemcpyHostToDevice, sl.stream);
    if (e != cudaSuccess) {
        fp_set_error("fp_server: cudaMemcpyAsync(rows): %s", cudaGetErrorString(e));
        rc = FP_ECUDA;
    }
    if (rc == FP_OK) rc = fp_predict_batched(fl.data(), batches.data(), (int32_t)k, sl.stream);
    if (rc == FP_OK) {
        e = cudaMemcpyAsync(sl.pin + in_bytes, sl.dev + in_bytes, out_bytes, cudaMemcpyDeviceToHost, sl.stream);
        if (e != cudaSuccess) {
            fp_set_error("fp_server: cudaMemcpyAsync(results): %s", cudaGetErrorString(e));
            rc = FP_ECUDA;
        }
    }
    cudaEventRecord(sl.ev, sl.stream);
    return rc;
}

void batch_loop(fp_server *s) {
    cudaSetDevice(s->device);
    for (;;) {
        std::vector<fp_request *> batch;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_queue.wait(lk, [&] { return s->stopping || !s->queue.empty(); });
            if (s->queue.empty()) break;  // stopping, and every queued request taken
            if (s->max_wait_s > 0) {      // let a small batch grow until the oldest request has waited enough
                const auto deadline = s->queue.front()->t_submit +
                                      std::chrono::duration_cast<fp_clock::duration>(
                                          std::chrono::duration<double>(s->max_wait_s));
                for (;;) {
                    int64_t q = 0;
                    for (fp_request *r : s->queue) q += r->n;
                    if (q >= s->max_rows || s->stopping ||
                        s->cv_queue.wait_until(lk, deadline) == std::cv_status::timeout)
                        break;
                }
            }
            int64_t rows = 0;
            while (!s->queue.empty() && (batch.empty() || rows + s->queue.front()->n <= s->max_rows)) {
                rows += s->queue.front()->n;
                batch.push_back(s->queue.front());
                s->queue.pop_front();
            }
        }
        // group by forest, keeping arrival order within a forest
        std::vector<int32_t> gforest;
        std::vector<std::vector<fp_request *>> groups;
        size_t need = 0;
        for (fp_request *r : batch) {
            size_t g = 0;
            while (g < gforest.size() && gforest[g] != r->forest) ++g;
            if (g == gforest.size()) {
                gforest.push_back(r->forest);
                groups.emplace_back();
            }
            groups[g].push_back(r);
            need += (size_t)r->n * 4 * (s->F[r->forest] + 1 + (s->return_votes ? s->C[r->forest] : 0));
        }
        // admission: enough free device memory, else wait for launches in flight
        while (free_bytes(s) < need + (size_t)s->mem_margin) {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->inflight.empty()) break;
            ++s->rejected_for_memory;
            s->cv_slot.wait_for(lk, std::chrono::milliseconds(1));
        }
        int si = -1;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_slot.wait(lk, [&] { return !s->free_slots.empty() || s->live_slots == 0; });
            if (!s->free_slots.empty()) {
                si = s->free_slots.back();
                s->free_slots.pop_back();
            } else {  // every slot retired: nothing can run this batch
                const auto t = fp_clock::now();
                for (fp_request *r : batch) {
                    r->status = FP_ETIMEOUT;
                    r->t_done = t;
                    r->done = true;
                }
            }
        }
        if (si < 0) {
            s->cv_done.notify_all();
            continue;
        }
        Slot &sl = s->slot[si];
        sl.status = launch(s, sl, groups, gforest);
        if (sl.status != FP_OK) {  // answer the batch's requests with the error
            sl.entries.clear();
            for (fp_request *r : batch) sl.entries.push_back({r, 0, SIZE_MAX});
        }
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->inflight.push_back(si);
            if (sl.status == FP_OK) ++s->launches;
        }
        s->cv_slot.notify_all();
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->batcher_done = true;
    }
    s->cv_slot.notify_all();
}

void complete_loop(fp_server *s) {
    cudaSetDevice(s->device);
    for (;;) {
        int si;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_slot.wait(lk, [&] { return !s->inflight.empty() || s->batcher_done; });
            if (s->inflight.empty()) break;
            si = s->inflight.front();
        }
        Slot &sl = s->slot[si];
        int st = sl.status;
        const auto limit = std::chrono::duration_cast<fp_clock::duration>(
            std::chrono::duration<double>(s->launch_timeout_s));
        // bounded poll of the slot's event: 1 = done, 0 = not done by the deadline, -1 = CUDA error
        auto poll = [&](fp_clock::time_point deadline) {
            for (;;) {
                const cudaError_t q = cudaEventQuery(sl.ev);
                if (q == cudaSuccess) return 1;
                if (q != cudaErrorNotReady) return -1;
                if (fp_clock::now() > deadline) return 0;
                std::this_thread::sleep_for(std::chrono::microseconds(20));
            }
        };
        int idle = 0;
        if (st == FP_OK) {
            idle = poll(fp_clock::now() + limit);
            if (idle != 1) st = idle < 0 ? FP_ECUDA : FP_ETIMEOUT;
        } else {  // a failed launch may have queued work before it failed: let it drain, bounded
            idle = poll(fp_clock::now() + limit);
        }
        if (st == FP_ETIMEOUT && idle == 0) idle = poll(fp_clock::now());  // one last look
        const auto t = fp_clock::now();
        if (st == FP_OK) {
            for (const Entry &en : sl.entries) {
                fp_request *r = en.req;
                if (r->out_class) memcpy(r->out_class, sl.pin + en.class_off, (size_t)r->n * 4);
                if (r->out_votes && en.votes_off != SIZE_MAX)
                    memcpy(r->out_votes, sl.pin + en.votes_off, (size_t)r->n * s->C[r->forest] * 4);
            }
        }
        {
            std::lock_guard<std::mutex> lk(s->mu);
            for (const Entry &en : sl.entries) {
                en.req->status = st;
                en.req->t_done = t;
                en.req->done = true;
            }
            sl.entries.clear();
            s->inflight.pop_front();
            if (idle == 1) {
                s->free_slots.push_back(si);
            } else {  // its copies or kernel may still touch its buffers
                sl.retired = true;
                --s->live_slots;
            }
        }
        s->cv_done.notify_all();
        s->cv_slot.notify_all();
    }
}

void join_threads(fp_server *s) {
    if (!s->started || s->joined) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
    }
    s->cv_queue.notify_all();
    s->cv_slot.notify_all();
    s->batcher.join();
    s->completer.join();
    s->joined = true;
}

}  // namespace

extern "C" int fp_server_create(int32_t device, int32_t slots, int64_t max_rows, int64_t mem_margin,
                                int32_t return_votes, double max_wait_s, fp_server **out) {
    if (!out || slots < 1 || slots > 64 || max_rows < 1 || mem_margin < 0 || max_wait_s < 0) {
        fp_set_error("fp_server_create: bad arguments");
        return FP_EINVAL;
    }
    *out = nullptr;
    fp_server *s = new (std::nothrow) fp_server;
    if (!s) {
        fp_set_error("fp_server_create: out of host memory");
        return FP_ENOMEM;
    }
    s->device = device;
    s->max_rows = max_rows;
    s->mem_margin = mem_margin;
    s->return_votes = return_votes ? 1 : 0;
    s->max_wait_s = max_wait_s;
    s->slot.resize((size_t)slots);
    cudaError_t e = cudaSetDevice(device);
    for (int i = 0; i < slots && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&s->slot[i].stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->slot[i].ev, cudaEventDisableTiming);
        s->free_slots.push_back(slots - 1 - i);
    }
    s->live_slots = slots;
    if (e != cudaSuccess) {
        fp_set_error("fp_server_create: %s", cudaGetErrorString(e));
        fp_server_release(s);
        return FP_ECUDA;
    }
    *out = s;
    return FP_OK;
}

extern "C" int fp_server_add_forest(fp_server *s, const fp_device_forest *forest, int32_t *out_id) {
    if (!s || !forest || !out_id || s->started) {
        fp_set_error("fp_server_add_forest: bad arguments (forests are added before fp_server_start)");
        return FP_EINVAL;
    }
    fp_packed_info info;
    int rc = fp_device_info_get(forest, &info);
    if (rc) return rc;
    s->forests.push_back(forest);
    s->F.push_back(info.n_features);
    s->C.push_back(info.n_classes);
    *out_id = (int32_t)s->forests.size() - 1;
    return FP_OK;
}

extern "C" int fp_server_start(fp_server *s) {
    if (!s || s->started) {
        fp_set_error("fp_server_start: bad arguments or already started");
        return FP_EINVAL;
    }
    s->started = true;
    try {
        s->batcher = std::thread(batch_loop, s);
        s->completer = std::thread(complete_loop, s);
    } catch (...) {
        fp_set_error("fp_server_start: cannot start threads");
        if (s->batcher.joinable()) {
            {
                std::lock_guard<std::mutex> lk(s->mu);
                s->stopping = true;
                s->batcher_done = true;
            }
            s->cv_queue.notify_all();
            s->batcher.join();
        }
        s->joined = true;
        return FP_ENOMEM;
    }
    return FP_OK;
}

extern "C" int fp_server_submit(fp_server *s, int32_t forest_id, const float *X_host, int64_t n,
                                int32_t *out_class_host, uint32_t *out_votes_host, fp_request **out) {
    if (!s || !out || forest_id < 0 || forest_id >= (int32_t)s->forests.size() || n < 1 || !X_host ||
        (!out_class_host && !out_votes_host) || (out_votes_host && !s->return_votes)) {
        fp_set_error("fp_server_submit: bad arguments");
        return FP_EINVAL;
    }
    fp_request *r = new (std::nothrow) fp_request;
    if (!r) {
        fp_set_error("fp_server_submit: out of host memory");
        return FP_ENOMEM;
    }
    r->srv = s;
    r->forest = forest_id;
    r->X = X_host;
    r->n = n;
    r->out_class = out_class_host;
    r->out_votes = out_votes_host;
    r->t_submit = fp_clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (!s->started || s->stopping) {
            delete r;
            fp_set_error("fp_server_submit: the server is not running");
            return FP_EINVAL;
        }
        s->queue.push_back(r);
    }
    s->cv_queue.notify_one();
    *out = r;
    return FP_OK;
}

extern "C" int fp_request_wait(fp_request *r, double timeout_s) {
    if (!r) {
        fp_set_error("fp_request_wait: NULL request");
        return FP_EINVAL;
    }
    fp_server *s = r->srv;
    std::unique_lock<std::mutex> lk(s->mu);
    if (timeout_s < 0) {
        s->cv_done.wait(lk, [&] { return r->done; });
    } else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return r->done; })) {
        return FP_ETIMEOUT;
    }
    return r->status;
}

extern "C" double fp_request_latency(const fp_request *r) {
    if (!r) return -1.0;
    std::lock_guard<std::mutex> lk(r->srv->mu);
    if (!r->done) return -1.0;
    return std::chrono::duration<double>(r->t_done - r->t_submit).count();
}

extern "C" void fp_request_release(fp_request *r) {
    if (!r) return;
    {
        std::unique_lock<std::mutex> lk(r->srv->mu);  // a request is freed only once answered
        r->srv->cv_done.wait(lk, [&] { return r->done; });
    }
    delete r;
}

extern "C" int fp_server_stop(fp_server *s) {
    if (!s) {
        fp_set_error("fp_server_stop: NULL server");
        return FP_EINVAL;
    }
    join_threads(s);
    return FP_OK;
}

extern "C" int fp_server_stats(const fp_server *s, int64_t *launches, int64_t *rejected_for_memory) {
    if (!s) {
        fp_set_error("fp_server_stats: NULL server");
        return FP_EINVAL;
    }
    std::lock_guard<std::mutex> lk(const_cast<fp_server *>(s)->mu);
    if (launches) *launches = s->launches;
    if (rejected_for_memory) *rejected_for_memory = s->rejected_for_memory;
    return FP_OK;
}

extern "C" int fp_server_set_free_bytes(fp_server *s, int64_t free_bytes) {
    if (!s) {
        fp_set_error("fp_server_set_free_bytes: NULL server");
        return FP_EINVAL;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    s->free_override = free_bytes < 0 ? -1 : free_bytes;
    return FP_OK;
}

extern "C" int fp_server_set_launch_timeout(fp_server *s, double seconds) {
    if (!s || !(seconds >= 0)) {
        fp_set_error("fp_server_set_launch_timeout: bad arguments");
        return FP_EINVAL;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    s->launch_timeout_s = seconds;
    return FP_OK;
}

extern "C" int fp_server_slots_in_service(const fp_server *s, int32_t *out) {
    if (!s || !out) {
        fp_set_error("fp_server_slots_in_service: bad arguments");
        return FP_EINVAL;
    }
    std::lock_guard<std::mutex> lk(const_cast<fp_server *>(s)->mu);
    *out = s->live_slots;
    return FP_OK;
}

extern "C" void fp_server_release(fp_server *s) {
    if (!s) return;
    join_threads(s);
    cudaSetDevice(s->device);
    for (Slot &sl : s->slot) {
        bool idle = true;
        if (sl.retired && sl.ev) {  // its work outlived the completion poll: wait once more, bounded
            const auto deadline = fp_clock::now() + std::chrono::duration_cast<fp_clock::duration>(
                                                        std::chrono::duration<double>(s->launch_timeout_s));
            cudaError_t q;
            while ((q = cudaEventQuery(sl.ev)) == cudaErrorNotReady && fp_clock::now() <= deadline)
                std::this_thread::sleep_for(std::chrono::microseconds(100));
            idle = q == cudaSuccess;
        } else if (sl.stream) {
            cudaStreamSynchronize(sl.stream);  // idle already: every launch on it completed
        }
        if (idle) {  // else the buffers stay allocated: work that never finished may still use them
            if (sl.dev) cudaFree(sl.dev);
            if (sl.pin) cudaFreeHost(sl.pin);
        }
        if (sl.ev) cudaEventDestroy(sl.ev);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    delete s;
}
