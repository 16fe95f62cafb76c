// Serving loop of the bsort library: continuous batching of sort requests.
//
// Requests (a device buffer of n keys, dtype, direction) are submitted from
// any host thread and queue in arrival order.  A scheduler thread owns
// `num_slots` slots -- a CUDA stream, a handle and a workspace each -- and
// admits the oldest waiting request whenever a slot is free and the HBM
// budget (payload + the workspace a standalone sort of that request needs,
// summed over requests in flight) has room.  A slot takes several small
// requests at once while their keys stay under `batch_keys`.  Requests in
// different slots overlap on the device.  Completion is observed with an
// event per slot; each completion carries host steady-clock timestamps of
// submit, admission and completion.  The sorts themselves are the library's
// plain sort (bsort_keys_ws), so a request gives the same bytes alone and in
// the mix.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "bsort.h"
#include "bsort_device.cuh"
#include "bsort_handle.h"

namespace {

uint64_t now_ns() {
    return static_cast<uint64_t>(
        std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
            .count());
}

int key_bytes(bsort_dtype dt) {
    static const int b[] = {1, 1, 2, 2, 2, 4, 4, 4, 8, 8, 8, 2};
    const int i = static_cast<int>(dt);
    return i >= 0 && i <= 11 ? b[i] : 0;
}

struct Request {
    void *keys;
    size_t n;
    bsort_dtype dt;
    int desc;
    uint64_t tag;
    uint64_t t_submit, t_admit;
    size_t footprint;
    bsort_status launch;  // status of the host call that enqueued the sort
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bsort_handle *handle = nullptr;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    uint32_t *err = nullptr;  // pinned host: device error word of each request in the batch
    std::vector<Request> batch;
    bool busy = false;
};

}  // namespace

struct bsort_server {
    bsort_server_config cfg;
    int device = 0;
    std::vector<Slot> slots;
    std::mutex mu;  // queue, completions, counters
    std::condition_variable cv;
    std::deque<Request> pending;
    std::deque<bsort_completion> done;
    size_t in_flight_bytes = 0;
    size_t peak_bytes = 0;
    uint64_t submitted = 0, completed = 0, batches = 0;
    std::atomic<uint64_t> launches{0};
    int max_concurrent = 0;
    std::atomic<bool> stop{false};
    std::atomic<bool> paused{false};
    std::atomic<int> fatal{0};
    std::thread thread;

    void run();
    bool step();
};

bool bsort_server::step() {
    bool progress = false;
    // retire finished slots
    for (size_t i = 0; i < slots.size(); ++i) {
        Slot &s = slots[i];
        if (!s.busy) continue;
        const cudaError_t q = cudaEventQuery(s.done);
        if (q == cudaErrorNotReady) continue;
        const uint64_t t = now_ns();
        std::lock_guard<std::mutex> lk(mu);
        for (size_t j = 0; j < s.batch.size(); ++j) {
            const Request &r = s.batch[j];
            bsort_completion c;
            c.tag = r.tag;
            c.status = r.launch != BSORT_OK              ? r.launch
                       : q != cudaSuccess                  ? BSORT_ERR_CUDA
                       : (s.err[j] & bsort::kErrCapacity) ? BSORT_ERR_CAPACITY
                       : (s.err[j] & bsort::kErrTimeout)  ? BSORT_ERR_TIMEOUT
                       : s.err[j]                         ? BSORT_ERR_INTERNAL
                                                          : BSORT_OK;
            c.slot = static_cast<int32_t>(i);
            c.t_submit_ns = r.t_submit;
            c.t_admit_ns = r.t_admit;
            c.t_done_ns = t;
            done.push_back(c);
            in_flight_bytes -= r.footprint;
            ++completed;
        }
        s.batch.clear();
        s.busy = false;
        progress = true;
    }
    // admit waiting requests, oldest first
    for (size_t i = 0; i < slots.size() && !paused.load(); ++i) {
        Slot &s = slots[i];
        if (s.busy) continue;
        std::unique_lock<std::mutex> lk(mu);
        size_t keys_in_batch = 0;
        while (!pending.empty() && static_cast<int>(s.batch.size()) < cfg.max_batch) {
            Request &r = pending.front();
            if (in_flight_bytes + r.footprint > cfg.hbm_budget_bytes && in_flight_bytes > 0) break;
            if (!s.batch.empty() && keys_in_batch + r.n > cfg.batch_keys) break;
            r.t_admit = now_ns();
            in_flight_bytes += r.footprint;
            if (in_flight_bytes > peak_bytes) peak_bytes = in_flight_bytes;
            keys_in_batch += r.n;
            s.batch.push_back(r);
            pending.pop_front();
        }
        lk.unlock();
        if (s.batch.empty()) break;  // nothing admissible: later slots would see the same head
        for (size_t j = 0; j < s.batch.size(); ++j) {
            Request &r = s.batch[j];
            s.err[j] = 0;
            s.handle->last_ctl = nullptr;
            r.launch = bsort_keys_ws(s.handle, r.keys, r.n, r.dt, r.desc, static_cast<bsort_mode>(cfg.mode), s.ws,
                                     s.ws_bytes, s.stream);
            if (r.launch == BSORT_ERR_CUDA) fatal.store(r.launch);
            launches += static_cast<uint64_t>(s.handle->rec.launches);
            // the next request of the batch reuses the workspace (and its error word): copy this one's out
            if (s.handle->last_ctl)
                cudaMemcpyAsync(&s.err[j], &s.handle->last_ctl->error, 4, cudaMemcpyDeviceToHost, s.stream);
        }
        cudaEventRecord(s.done, s.stream);
        s.busy = true;
        ++batches;
        int busy = 0;
        for (const Slot &x : slots) busy += x.busy;
        if (busy > max_concurrent) max_concurrent = busy;
        progress = true;
    }
    return progress;
}

void bsort_server::run() {
    cudaSetDevice(device);
    while (!stop.load()) {
        if (!step()) {
            std::unique_lock<std::mutex> lk(mu);
            cv.wait_for(lk, std::chrono::microseconds(20));
        }
    }
}

extern "C" {

bsort_status bsort_server_create(const bsort_server_config *cfg, bsort_server **out) {
    if (!cfg || !out || cfg->num_slots < 1 || cfg->num_slots > 64 || cfg->max_request_keys < 2 ||
        cfg->max_batch < 1 || cfg->max_batch > 4096 ||
        (cfg->mode != BSORT_MODE_PINGPONG && cfg->mode != BSORT_MODE_INPLACE))
        return BSORT_ERR_INVALID_ARG;
    bsort_server *s = new (std::nothrow) bsort_server();
    if (!s) return BSORT_ERR_NO_MEMORY;
    s->cfg = *cfg;
    cudaGetDevice(&s->device);
    // workspace of the widest request any dtype can make
    size_t ws = 0;
    for (int dt = 0; dt <= 11; ++dt) {
        size_t b = 0;
        if (bsort_workspace_bytes(cfg->max_request_keys, static_cast<bsort_dtype>(dt),
                                  static_cast<bsort_mode>(cfg->mode), &b) ==
                BSORT_OK &&
            b > ws)
            ws = b;
    }
    s->slots.resize(cfg->num_slots);
    for (Slot &sl : s->slots) {
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
            bsort_handle_create(&sl.handle) != BSORT_OK || cudaMalloc(&sl.ws, ws) != cudaSuccess ||
            cudaMallocHost(&sl.err, sizeof(uint32_t) * cfg->max_batch) != cudaSuccess) {
            bsort_server_destroy(s);
            (void)cudaGetLastError();
            return BSORT_ERR_NO_MEMORY;
        }
        sl.ws_bytes = ws;
    }
    s->thread = std::thread([s] { s->run(); });
    *out = s;
    return BSORT_OK;
}

bsort_status bsort_server_submit(bsort_server *s, void *keys, size_t n, bsort_dtype dt, int descending,
                                 uint64_t tag) {
    if (!s) return BSORT_ERR_INVALID_ARG;
    const int b = key_bytes(dt);
    if (!b) return BSORT_ERR_INVALID_ARG;
    if (n > s->cfg.max_request_keys) return BSORT_ERR_UNSUPPORTED;
    if (n > 1 && !keys) return BSORT_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(keys) % b) return BSORT_ERR_MISALIGNED;
    if (s->fatal.load()) return static_cast<bsort_status>(s->fatal.load());
    size_t ws = 0;
    bsort_workspace_bytes(n, dt, static_cast<bsort_mode>(s->cfg.mode), &ws);
    Request r{keys, n, dt, descending, tag, now_ns(), 0, n * static_cast<size_t>(b) + ws, BSORT_OK};
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->pending.push_back(r);
        ++s->submitted;
    }
    s->cv.notify_one();
    return BSORT_OK;
}

bsort_status bsort_server_poll(bsort_server *s, bsort_completion *out, size_t max, size_t *count) {
    if (!s || !count || (max && !out)) return BSORT_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    size_t k = 0;
    while (k < max && !s->done.empty()) {
        out[k++] = s->done.front();
        s->done.pop_front();
    }
    *count = k;
    return static_cast<bsort_status>(s->fatal.load());
}

bsort_status bsort_server_stats(bsort_server *s, bsort_server_info *out) {
    if (!s || !out) return BSORT_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->batches = s->batches;
    out->pending = s->pending.size();
    out->in_flight_bytes = s->in_flight_bytes;
    out->peak_in_flight_bytes = s->peak_bytes;
    out->max_concurrent_slots = s->max_concurrent;
    out->slot_workspace_bytes = s->slots.empty() ? 0 : s->slots[0].ws_bytes;
    out->launches = s->launches.load();
    return BSORT_OK;
}

bsort_status bsort_server_drain(bsort_server *s, double timeout_s) {
    if (!s) return BSORT_ERR_INVALID_ARG;
    const uint64_t t_end = now_ns() + static_cast<uint64_t>(timeout_s * 1e9);
    for (;;) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if (s->completed == s->submitted) return static_cast<bsort_status>(s->fatal.load());
        }
        if (now_ns() > t_end) return BSORT_ERR_TIMEOUT;
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

bsort_status bsort_server_pause(bsort_server *s, int paused) {
    if (!s) return BSORT_ERR_INVALID_ARG;
    s->paused.store(paused != 0);
    s->cv.notify_one();
    return BSORT_OK;
}

bsort_status bsort_server_destroy(bsort_server *s) {
    if (!s) return BSORT_ERR_INVALID_ARG;
    s->stop.store(true);
    s->cv.notify_one();
    if (s->thread.joinable()) s->thread.join();
    for (Slot &sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.ws) cudaFree(sl.ws);
        if (sl.err) cudaFreeHost(sl.err);
        if (sl.handle) bsort_handle_destroy(sl.handle);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    delete s;
    return BSORT_OK;
}

}  // extern "C"
