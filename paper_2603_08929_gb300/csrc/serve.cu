// Serving loop of the bsort library: continuous batching of sort requests,
// on one or several GPUs.
//
// A server owns lanes, one per entry of its device list (an entry is a CUDA
// device; the same device may appear twice, which splits its slots and
// budget in two).  Each lane has `num_slots` slots -- a CUDA stream, a
// handle and workspaces each -- and its own HBM budget.  A submitted request
// (a device buffer of n keys, dtype, direction) joins the queue of the
// least-loaded lane of the buffer's device (in-flight plus queued bytes over
// the budget); `bsort_server_pick_device` tells a caller which device to put
// its next request on.  A scheduler thread admits each lane's oldest waiting
// request whenever one of the lane's slots is free and the lane's budget
// (payload + the workspace a standalone sort of the request needs, summed
// over its requests in flight) has room.  A slot takes several small
// requests at once while their keys stay under `batch_keys`; requests of one
// 4- or 8-byte dtype and direction in a slot are sorted together: their
// keys are gathered into the slot's staging buffer, one segmented sort (one
// launch sequence for all of them) sorts each request's segment, and the
// keys go back to their buffers.  Other requests take the plain sort.  Both
// give every request the same bytes alone and in the mix (a segment is
// sorted exactly as a plain array).  Completion is observed with an event
// per slot; each completion carries host steady-clock timestamps of submit,
// admission and completion.
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
    static const int b[] = {1, 1, 2, 2, 2, 4, 4, 4, 8, 8, 8, 2, 16, 16};
    const int i = static_cast<int>(dt);
    return i >= 0 && i <= 13 ? b[i] : 0;
}

// Requests one segmented sort gathers (descriptor passed by value).
constexpr int kMaxGroup = 16;

struct GroupDesc {
    void *keys[kMaxGroup];
    uint64_t off[kMaxGroup + 1];  // segment starts in the staging buffer, then the total
    uint32_t *err[kMaxGroup];     // pinned host words receiving the sort's device error word
    int count;
};

// Copies the group's requests into the staging buffer (key by key, words of
// W bytes) and writes the segment offsets for the segmented sort.
template <typename W>
__global__ void k_group_gather(GroupDesc g, W *__restrict__ stage, uint64_t *__restrict__ d_off) {
    const int r = blockIdx.y;
    if (blockIdx.x == 0 && threadIdx.x <= static_cast<unsigned>(g.count) && r == 0) d_off[threadIdx.x] = g.off[threadIdx.x];
    const W *src = static_cast<const W *>(g.keys[r]);
    const uint64_t a = g.off[r], n = g.off[r + 1] - a;
    for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<uint64_t>(gridDim.x) * blockDim.x)
        stage[a + i] = src[i];
}

// Copies the sorted segments back and hands each request the error word.
template <typename W>
__global__ void k_group_scatter(GroupDesc g, const W *__restrict__ stage, const uint32_t *ctl_err) {
    const int r = blockIdx.y;
    W *dst = static_cast<W *>(g.keys[r]);
    const uint64_t a = g.off[r], n = g.off[r + 1] - a;
    for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<uint64_t>(gridDim.x) * blockDim.x)
        dst[i] = stage[a + i];
    if (blockIdx.x == 0 && threadIdx.x == 0) *g.err[r] = ctl_err ? *ctl_err : 0u;
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
    int lane;
};

struct Slot {
    int lane = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bsort_handle *handle = nullptr;
    void *ws = nullptr;  // plain sorts
    size_t ws_bytes = 0;
    void *stage = nullptr;  // grouped requests: gathered keys
    uint64_t *d_off = nullptr;
    void *seg_ws = nullptr;
    size_t seg_ws_bytes = 0;
    uint32_t *err = nullptr;  // pinned host: device error word of each request in the batch
    std::vector<Request> batch;
    bool busy = false;
};

struct Lane {
    int device = 0;
    size_t budget = 0;
    size_t in_flight = 0, peak = 0, queued = 0;
    uint64_t admitted = 0, completed = 0;
    std::deque<Request> pending;
};

}  // namespace

struct bsort_server {
    bsort_server_config cfg;
    std::vector<Lane> lanes;
    std::vector<Slot> slots;  // lane l owns slots [l * num_slots, (l + 1) * num_slots)
    std::mutex mu;            // queues, completions, counters
    std::condition_variable cv;
    std::deque<bsort_completion> done;
    size_t in_flight_bytes = 0;
    size_t peak_bytes = 0;
    size_t pending_count = 0;
    uint64_t submitted = 0, completed = 0, batches = 0, grouped = 0;
    std::atomic<uint64_t> launches{0};
    int max_concurrent = 0;
    std::atomic<bool> stop{false};
    std::atomic<bool> paused{false};
    std::atomic<int> fatal{0};
    std::thread thread;

    void run();
    bool step();
    void launch(Slot &s);
    int pick_lane(int device) const;  // caller holds mu; -1: no lane on that device
};

int bsort_server::pick_lane(int device) const {
    int best = -1;
    double best_load = 0;
    for (size_t l = 0; l < lanes.size(); ++l) {
        const Lane &ln = lanes[l];
        if (device >= 0 && ln.device != device) continue;
        const double load = static_cast<double>(ln.in_flight + ln.queued) / static_cast<double>(ln.budget);
        if (best < 0 || load < best_load) {
            best = static_cast<int>(l);
            best_load = load;
        }
    }
    return best;
}

// Enqueues a slot's batch on its stream: requests of one 4/8-byte dtype and
// direction go through one segmented sort (in groups of up to kMaxGroup),
// the rest through the plain sort.
void bsort_server::launch(Slot &s) {
    std::vector<char> used(s.batch.size(), 0);
    for (size_t j = 0; j < s.batch.size(); ++j) {
        if (used[j]) continue;
        const Request &r0 = s.batch[j];
        const int b = key_bytes(r0.dt);
        std::vector<size_t> grp{j};
        if ((b == 4 || b == 8) && r0.n > 1 && s.stage) {
            size_t keys = r0.n;
            for (size_t k = j + 1; k < s.batch.size() && grp.size() < static_cast<size_t>(kMaxGroup); ++k)
                if (!used[k] && s.batch[k].dt == r0.dt && s.batch[k].desc == r0.desc && s.batch[k].n > 1 &&
                    keys + s.batch[k].n <= cfg.batch_keys) {
                    grp.push_back(k);
                    keys += s.batch[k].n;
                }
        }
        if (grp.size() >= 2) {
            GroupDesc g;
            g.count = static_cast<int>(grp.size());
            uint64_t total = 0, longest = 0;
            for (int q = 0; q < g.count; ++q) {
                Request &r = s.batch[grp[q]];
                g.keys[q] = r.keys;
                g.off[q] = total;
                g.err[q] = &s.err[grp[q]];
                s.err[grp[q]] = 0;
                total += r.n;
                longest = r.n > longest ? r.n : longest;
                used[grp[q]] = 1;
            }
            g.off[g.count] = total;
            const dim3 grid(static_cast<unsigned>((longest + 1023) / 1024 < 64 ? (longest + 1023) / 1024 : 64),
                            static_cast<unsigned>(g.count));
            if (b == 4) k_group_gather<uint32_t><<<grid, 256, 0, s.stream>>>(g, static_cast<uint32_t *>(s.stage), s.d_off);
            else k_group_gather<uint64_t><<<grid, 256, 0, s.stream>>>(g, static_cast<uint64_t *>(s.stage), s.d_off);
            s.handle->last_ctl = nullptr;
            const bsort_status st = bsort_keys_segmented_ws(s.handle, s.stage, total, s.d_off, g.count, r0.dt, r0.desc,
                                                            s.seg_ws, s.seg_ws_bytes, s.stream);
            const uint32_t *ctl_err = s.handle->last_ctl ? &s.handle->last_ctl->error : nullptr;
            if (b == 4) k_group_scatter<uint32_t><<<grid, 256, 0, s.stream>>>(g, static_cast<const uint32_t *>(s.stage), ctl_err);
            else k_group_scatter<uint64_t><<<grid, 256, 0, s.stream>>>(g, static_cast<const uint64_t *>(s.stage), ctl_err);
            for (int q = 0; q < g.count; ++q) s.batch[grp[q]].launch = st;
            if (st == BSORT_ERR_CUDA || cudaGetLastError() != cudaSuccess) fatal.store(BSORT_ERR_CUDA);
            launches += static_cast<uint64_t>(s.handle->rec.launches) + 2;
            ++grouped;
            continue;
        }
        Request &r = s.batch[j];
        used[j] = 1;
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
}

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
        Lane &ln = lanes[s.lane];
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
            c.lane = s.lane;
            c.pad = 0;
            c.t_submit_ns = r.t_submit;
            c.t_admit_ns = r.t_admit;
            c.t_done_ns = t;
            done.push_back(c);
            in_flight_bytes -= r.footprint;
            ln.in_flight -= r.footprint;
            ++ln.completed;
            ++completed;
        }
        s.batch.clear();
        s.busy = false;
        progress = true;
    }
    // admit each lane's waiting requests, oldest first
    const int per = cfg.num_slots;
    for (size_t i = 0; i < slots.size() && !paused.load(); ++i) {
        Slot &s = slots[i];
        if (s.busy) continue;
        Lane &ln = lanes[s.lane];
        std::unique_lock<std::mutex> lk(mu);
        size_t keys_in_batch = 0;
        while (!ln.pending.empty() && static_cast<int>(s.batch.size()) < cfg.max_batch) {
            Request &r = ln.pending.front();
            if (ln.in_flight + r.footprint > ln.budget && ln.in_flight > 0) break;
            if (!s.batch.empty() && keys_in_batch + r.n > cfg.batch_keys) break;
            r.t_admit = now_ns();
            ln.in_flight += r.footprint;
            ln.queued -= r.footprint;
            if (ln.in_flight > ln.peak) ln.peak = ln.in_flight;
            in_flight_bytes += r.footprint;
            if (in_flight_bytes > peak_bytes) peak_bytes = in_flight_bytes;
            keys_in_batch += r.n;
            ++ln.admitted;
            --pending_count;
            s.batch.push_back(r);
            ln.pending.pop_front();
        }
        lk.unlock();
        if (s.batch.empty()) {  // nothing admissible on this lane: skip its other slots
            i = (i / per + 1) * per - 1;
            continue;
        }
        cudaSetDevice(ln.device);
        launch(s);
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
    while (!stop.load()) {
        if (!step()) {
            std::unique_lock<std::mutex> lk(mu);
            cv.wait_for(lk, std::chrono::microseconds(20));
        }
    }
}

namespace {
bool config_ok(const bsort_server_config *cfg) {
    return cfg && cfg->num_slots >= 1 && cfg->num_slots <= 64 && cfg->max_request_keys >= 2 && cfg->max_batch >= 1 &&
           cfg->max_batch <= 4096 && cfg->hbm_budget_bytes > 0 &&
           (cfg->mode == BSORT_MODE_PINGPONG || cfg->mode == BSORT_MODE_INPLACE);
}
}  // namespace

extern "C" {

bsort_status bsort_server_create_multi(const bsort_server_config *cfg, const int32_t *devices, int32_t num_devices,
                                       bsort_server **out) {
    if (!config_ok(cfg) || !out || !devices || num_devices < 1 || num_devices > BSORT_SERVER_MAX_LANES)
        return BSORT_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) return BSORT_ERR_CUDA;
    for (int l = 0; l < num_devices; ++l)
        if (devices[l] < 0 || devices[l] >= ndev) return BSORT_ERR_INVALID_ARG;
    int prev = 0;
    cudaGetDevice(&prev);
    bsort_server *s = new (std::nothrow) bsort_server();
    if (!s) return BSORT_ERR_NO_MEMORY;
    s->cfg = *cfg;
    // workspace of the widest request any dtype can make; grouped sorts: the
    // segmented workspace and staging of batch_keys keys (8-byte keys at most)
    size_t ws = 0, seg_ws = 0;
    const size_t gkeys = cfg->batch_keys;
    for (int dt = 0; dt <= 11; ++dt) {  // the dtypes the loop serves
        size_t b = 0;
        if (bsort_workspace_bytes(cfg->max_request_keys, static_cast<bsort_dtype>(dt),
                                  static_cast<bsort_mode>(cfg->mode), &b) == BSORT_OK &&
            b > ws)
            ws = b;
        if (key_bytes(static_cast<bsort_dtype>(dt)) >= 4 &&
            bsort_segmented_workspace_bytes(gkeys, kMaxGroup, static_cast<bsort_dtype>(dt), &b) == BSORT_OK &&
            b > seg_ws)
            seg_ws = b;
    }
    const bool group = cfg->max_batch >= 2 && gkeys >= 2;
    s->lanes.resize(num_devices);
    s->slots.resize(static_cast<size_t>(num_devices) * cfg->num_slots);
    bool ok = true;
    for (int l = 0; l < num_devices && ok; ++l) {
        s->lanes[l].device = devices[l];
        s->lanes[l].budget = cfg->hbm_budget_bytes;
        if (cudaSetDevice(devices[l]) != cudaSuccess) ok = false;
        for (int k = 0; k < cfg->num_slots && ok; ++k) {
            Slot &sl = s->slots[static_cast<size_t>(l) * cfg->num_slots + k];
            sl.lane = l;
            ok = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) == cudaSuccess &&
                 bsort_handle_create(&sl.handle) == BSORT_OK && cudaMalloc(&sl.ws, ws) == cudaSuccess &&
                 cudaMallocHost(&sl.err, sizeof(uint32_t) * cfg->max_batch) == cudaSuccess;
            if (ok && group)
                ok = cudaMalloc(&sl.stage, gkeys * 8) == cudaSuccess &&
                     cudaMalloc(&sl.d_off, sizeof(uint64_t) * (kMaxGroup + 1)) == cudaSuccess &&
                     cudaMalloc(&sl.seg_ws, seg_ws) == cudaSuccess;
            sl.ws_bytes = ws;
            sl.seg_ws_bytes = group ? seg_ws : 0;
        }
    }
    cudaSetDevice(prev);
    if (!ok) {
        bsort_server_destroy(s);
        (void)cudaGetLastError();
        return BSORT_ERR_NO_MEMORY;
    }
    s->thread = std::thread([s] { s->run(); });
    *out = s;
    return BSORT_OK;
}

bsort_status bsort_server_create(const bsort_server_config *cfg, bsort_server **out) {
    if (!config_ok(cfg) || !out) return BSORT_ERR_INVALID_ARG;
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess) return BSORT_ERR_CUDA;
    const int32_t dev = d;
    return bsort_server_create_multi(cfg, &dev, 1, out);
}

bsort_status bsort_server_pick_device(bsort_server *s, int32_t *device) {
    if (!s || !device) return BSORT_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    *device = s->lanes[s->pick_lane(-1)].device;
    return BSORT_OK;
}

bsort_status bsort_server_submit(bsort_server *s, void *keys, size_t n, bsort_dtype dt, int descending,
                                 uint64_t tag) {
    if (!s) return BSORT_ERR_INVALID_ARG;
    const int b = key_bytes(dt);
    if (!b) return BSORT_ERR_INVALID_ARG;
    if (b > 8 || n > s->cfg.max_request_keys) return BSORT_ERR_UNSUPPORTED;  // keys of up to 8 bytes
    if (n > 1 && !keys) return BSORT_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(keys) % b) return BSORT_ERR_MISALIGNED;
    if (s->fatal.load()) return static_cast<bsort_status>(s->fatal.load());
    int device = s->lanes[0].device;
    if (keys) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, keys) != cudaSuccess) {
            (void)cudaGetLastError();
            return BSORT_ERR_INVALID_ARG;
        }
        if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return BSORT_ERR_INVALID_ARG;
        device = at.device;
    }
    size_t ws = 0;
    bsort_workspace_bytes(n, dt, static_cast<bsort_mode>(s->cfg.mode), &ws);
    Request r{keys, n, dt, descending, tag, now_ns(), 0, n * static_cast<size_t>(b) + ws, BSORT_OK, 0};
    {
        std::lock_guard<std::mutex> lk(s->mu);
        const int l = s->pick_lane(device);
        if (l < 0) return BSORT_ERR_INVALID_ARG;  // the buffer is on a device the server does not serve
        r.lane = l;
        s->lanes[l].pending.push_back(r);
        s->lanes[l].queued += r.footprint;
        ++s->pending_count;
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
    out->pending = s->pending_count;
    out->in_flight_bytes = s->in_flight_bytes;
    out->peak_in_flight_bytes = s->peak_bytes;
    out->max_concurrent_slots = s->max_concurrent;
    out->num_lanes = static_cast<int32_t>(s->lanes.size());
    out->slot_workspace_bytes =
        s->slots.empty() ? 0 : s->slots[0].ws_bytes + s->slots[0].seg_ws_bytes + (s->slots[0].stage ? s->cfg.batch_keys * 8 : 0);
    out->launches = s->launches.load();
    out->grouped_sorts = s->grouped;
    return BSORT_OK;
}

bsort_status bsort_server_lane_stats(bsort_server *s, int32_t lane, bsort_server_lane_info *out) {
    if (!s || !out || lane < 0 || lane >= static_cast<int32_t>(s->lanes.size())) return BSORT_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    const Lane &ln = s->lanes[lane];
    out->device = ln.device;
    out->num_slots = s->cfg.num_slots;
    out->budget_bytes = ln.budget;
    out->in_flight_bytes = ln.in_flight;
    out->peak_in_flight_bytes = ln.peak;
    out->queued_bytes = ln.queued;
    out->admitted = ln.admitted;
    out->completed = ln.completed;
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
    int prev = 0;
    cudaGetDevice(&prev);
    for (Slot &sl : s->slots) {
        if (!s->lanes.empty()) cudaSetDevice(s->lanes[sl.lane].device);
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.ws) cudaFree(sl.ws);
        if (sl.stage) cudaFree(sl.stage);
        if (sl.d_off) cudaFree(sl.d_off);
        if (sl.seg_ws) cudaFree(sl.seg_ws);
        if (sl.err) cudaFreeHost(sl.err);
        if (sl.handle) bsort_handle_destroy(sl.handle);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    cudaSetDevice(prev);
    delete s;
    return BSORT_OK;
}

}  // extern "C"
