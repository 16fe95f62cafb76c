// C ABI of the bsort library: argument checks, workspace planning, handles,
// and dispatch to the counting path (1/2-byte keys) or the MSD path (4/8-byte
// keys).  Every step of the sort runs in the library's own kernels.
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <mutex>
#include <new>

#include "bsort_handle.h"
#include "bsort_launch.h"

using namespace bsort;

namespace {

struct DtypeInfo {
    int bytes;
    int kind;  // 0 unsigned, 1 signed, 2 float
};

bool dtype_info(bsort_dtype dt, DtypeInfo *out) {
    // bfloat16 takes the binary16 codec: the transform depends only on the
    // width and the kind (sign-magnitude), not on the exponent/mantissa split
    static const DtypeInfo table[] = {{1, 0}, {1, 1}, {2, 0}, {2, 1}, {2, 2}, {4, 0}, {4, 1},
                                      {4, 2}, {8, 0}, {8, 1}, {8, 2}, {2, 2}, {16, 0}, {16, 1}};
    const int i = static_cast<int>(dt);
    if (i < 0 || i > 13) return false;
    *out = table[i];
    return true;
}

// Constants of encode(x) = x ^ (msb(x) ? f1 : f0) and its inverse (Sec. III:
// the sign pass of Algs. 3/4 runs in the inverted direction; negative floats
// run in the inverted direction on exponent and mantissa).
Codec codec_for(const DtypeInfo &di, int descending) {
    if (di.bytes == 16) {  // integers: one xor, f0/d0 the low word and f1/d1 the high word
        const uint64_t dm = descending ? ~0ull : 0ull;
        Codec c;
        c.f0 = c.d0 = dm;
        c.f1 = c.d1 = dm ^ (di.kind == 1 ? 1ull << 63 : 0ull);
        return c;
    }
    const int w = di.bytes * 8;
    const uint64_t all = w == 64 ? ~0ull : ((1ull << w) - 1);
    const uint64_t sb = 1ull << (w - 1);
    const uint64_t dm = descending ? all : 0;
    Codec c;
    if (di.kind == 0) {
        c.f0 = c.f1 = dm;
        c.d0 = c.d1 = dm;
    } else if (di.kind == 1) {
        c.f0 = c.f1 = sb ^ dm;
        c.d0 = c.d1 = sb ^ dm;
    } else if (!descending) {
        c.f0 = sb;   // non-negative: flip the sign bit
        c.f1 = all;  // negative: flip every bit
        c.d1 = sb;   // encoded msb 1 <- non-negative
        c.d0 = all;  // encoded msb 0 <- negative
    } else {
        c.f0 = sb ^ all;
        c.f1 = 0;
        c.d1 = 0;
        c.d0 = sb ^ all;
    }
    return c;
}

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

struct MsdLayout {
    size_t alt, ctl, buckets0, buckets1, chunks0, chunks1, hist, cand, cor, bbase, units, fb_units, fills, total;
    uint32_t max_buckets, max_chunks, max_units, max_fills;
    // in-place mode (alt is empty then)
    bool inplace;
    size_t ip_big, ip_stripes, ip_ncnt, ip_rem, ip_part, ip_ovf, ip_state, lists_end;
    uint32_t max_big, max_stripes, max_slots;
    // stable key-value sort: value bytes (0: keys only), and whether the
    // values are positions made by the sort (then vals0 holds their parity-0
    // buffer; otherwise the caller's values are that buffer)
    int kv_bytes;
    bool kv_pos;
    size_t vals0, vals1;
};

MsdLayout msd_layout(size_t n, int key_bytes, size_t nseg = 0, bool inplace = false, const Tuning &tune = Tuning(),
                     int kv_bytes = 0, bool kv_pos = false) {
    const MsdShape s = msd_shape(key_bytes, tune, inplace, kv_bytes, n);
    MsdLayout L;
    // finish units hold at least merge_cap / 4 keys unless merged, and merged
    // groups reach merge_cap unless a run ends: the unit count per level is
    // bounded by n over the smaller of unit_cap and 5/4 merge_cap
    const uint64_t unit_floor = s.unit_cap < 5ull * s.merge_cap / 4 ? s.unit_cap : 5ull * s.merge_cap / 4;
    const uint64_t per_t = n / unit_floor + 1;
    L.max_buckets = static_cast<uint32_t>(n / (s.unit_cap + 1) + 2);
    // a bucket of len keys spans ceil((len + misalignment) / chunk) <= 1 + (len + 16) / chunk chunks
    L.max_chunks = static_cast<uint32_t>(L.max_buckets + (n + 16ull * L.max_buckets) / s.chunk + 2);
    // wide digits are classified in pages of 256: a run of merged small
    // buckets also ends at a page boundary (one more unit per page and parent)
    const uint64_t page_units = static_cast<uint64_t>(s.bins / kBins - 1) * s.levels * L.max_buckets;
    L.max_units = static_cast<uint32_t>((4 + 2 * static_cast<uint64_t>(s.levels)) * per_t + 16 + nseg + page_units);
    L.max_fills = static_cast<uint32_t>(n / kFillPiece + per_t + 16);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = align_up(off + bytes);
        return at;
    };
    L.inplace = inplace;
    L.alt = take(inplace ? 0 : n * key_bytes);
    L.kv_bytes = kv_bytes;
    L.kv_pos = kv_pos;
    L.vals0 = take(kv_pos ? n * kv_bytes : 0);
    L.vals1 = take(kv_bytes ? n * kv_bytes : 0);
    L.ctl = take(sizeof(Ctl));
    L.buckets0 = take(sizeof(Bucket) * L.max_buckets);
    L.buckets1 = take(sizeof(Bucket) * L.max_buckets);
    L.chunks0 = take(sizeof(Chunk) * L.max_chunks);
    L.chunks1 = take(sizeof(Chunk) * L.max_chunks);
    L.hist = take(sizeof(uint32_t) * s.bins * static_cast<size_t>(L.max_chunks));
    const size_t and_words = key_bytes > 8 ? 2 : 1;  // per chunk
    L.cand = take(sizeof(uint64_t) * and_words * L.max_chunks);
    L.cor = take(sizeof(uint64_t) * and_words * L.max_chunks);
    L.bbase = take(sizeof(uint32_t) * s.bins * static_cast<size_t>(L.max_buckets));
    L.units = take(sizeof(Unit) * L.max_units);
    L.fb_units = take(sizeof(Unit) * L.max_units);
    L.fills = take(sizeof(Fill) * L.max_fills);
    L.lists_end = off;
    L.max_big = L.max_stripes = L.max_slots = 0;
    L.ip_big = L.ip_stripes = L.ip_ncnt = L.ip_rem = L.ip_part = L.ip_ovf = L.ip_state = 0;
    if (inplace) {
        // a level's big buckets are disjoint and longer than the shared-memory capacity
        const uint64_t blk = kIpBlockBytes / key_bytes;
        const uint64_t cap = kIpSmemCapBytes / key_bytes;
        const uint64_t stripe = kIpStripeBytes / key_bytes;
        L.max_big = static_cast<uint32_t>(n / (cap + 1) + 1);
        L.max_stripes = static_cast<uint32_t>(n / stripe + L.max_big + 1);
        L.max_slots = static_cast<uint32_t>(n / blk + L.max_big + 1);
        L.ip_big = take(sizeof(IpBig) * L.max_big);
        L.ip_stripes = take(sizeof(IpStripe) * L.max_stripes);
        L.ip_ncnt = take(sizeof(uint32_t) * kBins * static_cast<size_t>(L.max_big));
        L.ip_rem = take(static_cast<size_t>(kBins) * L.max_stripes);
        L.ip_part = take(static_cast<size_t>(kIpBlockBytes) * kBins * L.max_stripes);
        L.ip_ovf = take(static_cast<size_t>(kIpBlockBytes) * kBins * L.max_big);
        L.ip_state = take(sizeof(uint32_t) * static_cast<size_t>(L.max_slots));
    }
    L.total = off;
    return L;
}

constexpr uint32_t kMaxGrid16 = 160;

uint32_t grid16_for(size_t n) {
    uint64_t g = (n + 65535) / 65536;
    if (g < 1) g = 1;
    if (g > kMaxGrid16) g = kMaxGrid16;
    return static_cast<uint32_t>(g);
}

struct CountLayout {
    size_t hist, rstart, rval, nruns, btot, bnnz, partial, total;
};

CountLayout count_layout(size_t n, int key_bytes) {
    CountLayout L;
    const size_t bins = key_bytes == 1 ? 256 : 65536;
    size_t off = 0;
    L.hist = off;
    off = align_up(off + bins * 8);
    L.rstart = off;
    off = align_up(off + (bins + 1) * 8);
    L.rval = off;
    off = align_up(off + bins * 4);
    L.nruns = off;
    off = align_up(off + 4);
    L.btot = off;
    off = align_up(off + 256 * 8);
    L.bnnz = off;
    off = align_up(off + 256 * 4);
    L.partial = off;
    if (key_bytes == 2) off = align_up(off + static_cast<size_t>(grid16_for(n)) * 65536 * 4);
    L.total = off;
    return L;
}

int num_sms_of(int device) {
    static std::atomic<int> cache[64];
    if (device < 0 || device >= 64) return 148;
    int v = cache[device].load(std::memory_order_relaxed);
    if (!v) {
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || v <= 0) v = 148;
        cache[device].store(v, std::memory_order_relaxed);
    }
    return v;
}

std::mutex g_default_mu;
bsort_handle *g_default[64] = {nullptr};

bsort_handle *default_handle(int device) {
    if (device < 0 || device >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_default_mu);
    if (!g_default[device]) {
        g_default[device] = new (std::nothrow) bsort_handle();
        if (g_default[device]) g_default[device]->device = device;
    }
    return g_default[device];
}

bsort_status ensure_events(bsort_handle *h) {
    if (h->events) return BSORT_OK;
    for (int i = 0; i < BSORT_PROFILE_MAX; ++i) {
        if (cudaEventCreate(&h->rec.rec[i].a) != cudaSuccess || cudaEventCreate(&h->rec.rec[i].b) != cudaSuccess)
            return BSORT_ERR_CUDA;
    }
    if (cudaMalloc(&h->prof_ctl, sizeof(Ctl) * BSORT_PROFILE_MAX_CALLS) != cudaSuccess) return BSORT_ERR_NO_MEMORY;
    h->events = true;
    return BSORT_OK;
}

bsort_status check_args(const void *keys, size_t n, bsort_dtype dt, DtypeInfo *di) {
    if (!dtype_info(dt, di)) return BSORT_ERR_INVALID_ARG;
    if (n <= 1) return BSORT_OK;
    if (!keys) return BSORT_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(keys) % di->bytes) return BSORT_ERR_MISALIGNED;
    if (di->bytes >= 4 && n >= (1ull << 32)) return BSORT_ERR_UNSUPPORTED;
    return BSORT_OK;
}

Work make_work(const MsdLayout &L, char *ws, void *keys, size_t n, const DtypeInfo &di, const Codec &codec,
               const Tuning &tune = Tuning()) {
    const MsdShape s = msd_shape(di.bytes, tune, L.inplace, L.kv_bytes, n);
    Work wk;
    wk.ctl = reinterpret_cast<Ctl *>(ws + L.ctl);
    wk.buckets[0] = reinterpret_cast<Bucket *>(ws + L.buckets0);
    wk.buckets[1] = reinterpret_cast<Bucket *>(ws + L.buckets1);
    wk.chunks[0] = reinterpret_cast<Chunk *>(ws + L.chunks0);
    wk.chunks[1] = reinterpret_cast<Chunk *>(ws + L.chunks1);
    wk.hist = reinterpret_cast<uint32_t *>(ws + L.hist);
    wk.chunk_and = reinterpret_cast<uint64_t *>(ws + L.cand);
    wk.chunk_or = reinterpret_cast<uint64_t *>(ws + L.cor);
    wk.bucket_base = reinterpret_cast<uint32_t *>(ws + L.bbase);
    wk.units = reinterpret_cast<Unit *>(ws + L.units);
    wk.fb_units = reinterpret_cast<Unit *>(ws + L.fb_units);
    wk.fills = reinterpret_cast<Fill *>(ws + L.fills);
    wk.keys = keys;
    wk.alt = ws + L.alt;
    wk.n = n;
    wk.codec = codec;
    wk.max_buckets = L.max_buckets;
    wk.max_chunks = L.max_chunks;
    wk.max_units = L.max_units;
    wk.max_fills = L.max_fills;
    wk.chunk_keys = s.chunk;
    wk.unit_cap = s.unit_cap;
    wk.merge_cap = s.merge_cap;
    wk.w = di.bytes * 8;
    wk.radix_bits = s.radix_bits;
    wk.bins = s.bins;
    wk.levels = s.levels;
    wk.stop_level = s.levels;
    wk.keys_vec_ok = (reinterpret_cast<uintptr_t>(keys) & 15) == 0;
    wk.inplace = L.inplace;
    wk.kv = L.kv_bytes;
    wk.kv_positions = L.kv_pos;
    wk.vals = L.kv_pos ? static_cast<void *>(ws + L.vals0) : nullptr;  // else the caller's values
    wk.vals_alt = L.kv_bytes ? static_cast<void *>(ws + L.vals1) : nullptr;
    wk.out_vals = nullptr;
    wk.out_idx = nullptr;
    wk.ip_big = L.inplace ? reinterpret_cast<IpBig *>(ws + L.ip_big) : nullptr;
    wk.ip_stripes = L.inplace ? reinterpret_cast<IpStripe *>(ws + L.ip_stripes) : nullptr;
    wk.ip_ncnt = L.inplace ? reinterpret_cast<uint32_t *>(ws + L.ip_ncnt) : nullptr;
    wk.ip_rem = L.inplace ? reinterpret_cast<uint8_t *>(ws + L.ip_rem) : nullptr;
    wk.ip_part = L.inplace ? static_cast<void *>(ws + L.ip_part) : nullptr;
    wk.ip_ovf = L.inplace ? static_cast<void *>(ws + L.ip_ovf) : nullptr;
    wk.ip_state = L.inplace ? reinterpret_cast<uint32_t *>(ws + L.ip_state) : nullptr;
    wk.max_big = L.max_big;
    wk.max_stripes = L.max_stripes;
    wk.max_slots = L.max_slots;
    if (L.inplace) wk.alt = nullptr;
    return wk;
}

void begin_call(bsort_handle *h, cudaStream_t st) {
    h->rec.enabled = h->profiling;
    h->rec.launches = 0;
    h->rec.stream = st;
    h->rec.active = h->profiling && h->events && h->rec.calls < BSORT_PROFILE_MAX_CALLS;
}

void end_call(bsort_handle *h, cudaStream_t st, size_t n, int key_bytes, int val_bytes = 0, int out_bytes = 0) {
    if (h->rec.active) {
        const int c = h->rec.calls;
        h->prof_path[c] = h->last_path;
        h->prof_key_bytes[c] = key_bytes;
        h->prof_n[c] = n;
        h->prof_val_bytes[c] = val_bytes;
        h->prof_out_bytes[c] = out_bytes;
        if (h->last_ctl) cudaMemcpyAsync(h->prof_ctl + c, h->last_ctl, sizeof(Ctl), cudaMemcpyDeviceToDevice, st);
        ++h->rec.calls;
    }
}

// The handle's MSD tuning for 4- and 8-byte keys; 16-byte keys run the
// library defaults.
const Tuning &tune_of(const bsort_handle *h, int key_bytes) {
    static const Tuning defaults;
    return key_bytes == 16 ? defaults : h->tune[key_bytes == 8];
}

bsort_status run_sort(bsort_handle *h, void *keys, size_t n, const DtypeInfo &di, int descending,
                      void *workspace, size_t ws_bytes, cudaStream_t st, bool inplace = false,
                      const Tuning *tune_override = nullptr) {
    (void)cudaGetLastError();  // clear a stale non-sticky error
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return BSORT_ERR_CUDA;
    const int sms = num_sms_of(dev);
    if (h->profiling) {
        const bsort_status es = ensure_events(h);
        if (es != BSORT_OK) return es;
    }
    begin_call(h, st);
    const Codec codec = codec_for(di, descending);
    char *ws = static_cast<char *>(workspace);
    h->last_stream = st;
    h->last_n = n;
    h->last_key_bytes = di.bytes;
    if (di.bytes <= 2) {
        const CountLayout L = count_layout(n, di.bytes);
        if (ws_bytes < L.total) return BSORT_ERR_WORKSPACE_TOO_SMALL;
        CountWork cw;
        cw.keys = keys;
        cw.n = n;
        cw.codec = codec;
        cw.hist = reinterpret_cast<unsigned long long *>(ws + L.hist);
        cw.rstart = reinterpret_cast<unsigned long long *>(ws + L.rstart);
        cw.rval = reinterpret_cast<uint32_t *>(ws + L.rval);
        cw.nruns = reinterpret_cast<uint32_t *>(ws + L.nruns);
        cw.btot = reinterpret_cast<unsigned long long *>(ws + L.btot);
        cw.bnnz = reinterpret_cast<uint32_t *>(ws + L.bnnz);
        cw.partial = reinterpret_cast<uint32_t *>(ws + L.partial);
        // one wave: at most one 128 KB-shared-memory CTA per SM (the partials are sized for grid16_for(n))
        cw.grid16 = std::min<uint32_t>(grid16_for(n), static_cast<uint32_t>(sms));
        if (di.bytes == 1) launch_count8(cw, st, h->rec, sms);
        else launch_count16(cw, st, h->rec, sms);
        h->last_path = 1;
        h->last_ctl = nullptr;
        h->last_inplace = inplace;  // the counting path writes the keys from counts: in place either way
        h->last_fixed_aux = L.total;
    } else {
        if (inplace && di.bytes > 8) return BSORT_ERR_UNSUPPORTED;
        const Tuning &tune = tune_override ? *tune_override : tune_of(h, di.bytes);
        const MsdLayout L = msd_layout(n, di.bytes, 0, inplace, tune);
        if (ws_bytes < L.total) return BSORT_ERR_WORKSPACE_TOO_SMALL;
        h->last_inplace = inplace;
        h->last_fixed_aux = inplace ? L.lists_end - L.ctl : L.total;
        Work wk = make_work(L, ws, keys, n, di, codec, tune);
        if (h->stop_levels > 0 && h->stop_levels < wk.levels) wk.stop_level = h->stop_levels;
        if (di.bytes == 4) launch_msd<uint32_t>(wk, st, h->rec, sms);
        else if (di.bytes == 8) launch_msd<uint64_t>(wk, st, h->rec, sms);
        else launch_msd<u128>(wk, st, h->rec, sms);
        h->last_path = 2;
        h->last_ctl = wk.ctl;
    }
    end_call(h, st, n, di.bytes);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? BSORT_OK : BSORT_ERR_CUDA;
}

bsort_status check_segmented(const void *keys, size_t n, const uint64_t *d_offsets, size_t nseg, bsort_dtype dt,
                             DtypeInfo *di) {
    if (!dtype_info(dt, di)) return BSORT_ERR_INVALID_ARG;
    if (di->bytes < 4) return BSORT_ERR_UNSUPPORTED;  // the segmented form takes 4- and 8-byte keys only
    if (nseg == 0 || n == 0) return BSORT_OK;
    if (!keys || !d_offsets) return BSORT_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(keys) % di->bytes || reinterpret_cast<uintptr_t>(d_offsets) % 8)
        return BSORT_ERR_MISALIGNED;
    if (n >= (1ull << 32) || nseg >= (1ull << 31)) return BSORT_ERR_UNSUPPORTED;
    return BSORT_OK;
}

// Enqueues the segmented sort (offsets checked on the device).
bsort_status run_segmented(bsort_handle *h, void *keys, size_t n, const uint64_t *d_offsets, size_t nseg,
                           const DtypeInfo &di, int descending, void *workspace, size_t ws_bytes, cudaStream_t st,
                           bool record) {
    (void)cudaGetLastError();
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return BSORT_ERR_CUDA;
    const int sms = num_sms_of(dev);
    if (record && h->profiling) {
        const bsort_status es = ensure_events(h);
        if (es != BSORT_OK) return es;
    }
    begin_call(h, st);
    if (!record) h->rec.active = false;
    const Tuning &tune = tune_of(h, di.bytes);
    const MsdLayout L = msd_layout(n, di.bytes, nseg, false, tune);
    if (ws_bytes < L.total) return BSORT_ERR_WORKSPACE_TOO_SMALL;
    const Work wk = make_work(L, static_cast<char *>(workspace), keys, n, di, codec_for(di, descending), tune);
    if (di.bytes == 4) launch_msd_segmented<uint32_t>(wk, d_offsets, static_cast<uint32_t>(nseg), st, h->rec, sms);
    else if (di.bytes == 8) launch_msd_segmented<uint64_t>(wk, d_offsets, static_cast<uint32_t>(nseg), st, h->rec, sms);
    else launch_msd_segmented<u128>(wk, d_offsets, static_cast<uint32_t>(nseg), st, h->rec, sms);
    h->last_path = 2;
    h->last_ctl = wk.ctl;
    h->last_stream = st;
    h->last_n = n;
    h->last_key_bytes = di.bytes;
    if (record) end_call(h, st, n, di.bytes);
    return cudaGetLastError() == cudaSuccess ? BSORT_OK : BSORT_ERR_CUDA;
}

bsort_status grow(void **buf, size_t *have, size_t need) {
    if (*have >= need && *buf) return BSORT_OK;
    if (*buf) {
        cudaFree(*buf);  // synchronises the device
        *buf = nullptr;
        *have = 0;
    }
    if (cudaMalloc(buf, need ? need : 256) != cudaSuccess) {
        (void)cudaGetLastError();
        *buf = nullptr;
        return BSORT_ERR_NO_MEMORY;
    }
    *have = need ? need : 256;
    return BSORT_OK;
}

size_t workspace_for(size_t n, const DtypeInfo &di, bool inplace = false, const Tuning &tune = Tuning()) {
    return di.bytes <= 2 ? count_layout(n, di.bytes).total : msd_layout(n, di.bytes, 0, inplace, tune).total;
}

// Key-value sorting workspace of 4- and 8-byte keys (the value-carrying MSD
// path): the MSD workspace with carry_bytes-wide value buffers (positions:
// both parities, else the alternate one), then the gather target of values
// that follow positions.
struct PairsKvLayout {
    MsdLayout msd;
    size_t tmp, total;
};

PairsKvLayout pairs_kv_layout(size_t n, int key_bytes, int carry_bytes, bool positions, size_t gather_bytes) {
    PairsKvLayout P;
    P.msd = msd_layout(n, key_bytes, 0, false, Tuning(), carry_bytes, positions);
    P.tmp = P.msd.total;
    P.total = align_up(P.tmp + gather_bytes * n);
    return P;
}

// Workspace of a key-value sort of n keys of key_bytes, for every form of
// request (values carried, positions, positions then a gather of 8-byte
// values).  1- and 2-byte keys: their 32-bit order codes (n words) ahead of
// the workspace of a 4-byte key-value sort.
size_t pairs_workspace_for(size_t n, int key_bytes) {
    if (key_bytes <= 2) return std::max(count_layout(n, key_bytes).total, align_up(4 * n) + pairs_workspace_for(n, 4));
    size_t b = msd_layout(n, key_bytes).total;  // keys alone (no values, no positions asked for)
    b = std::max(b, pairs_kv_layout(n, key_bytes, 4, false, 0).total);
    b = std::max(b, pairs_kv_layout(n, key_bytes, 8, false, 0).total);
    b = std::max(b, pairs_kv_layout(n, key_bytes, 4, true, 8).total);
    return b;
}

bool to_tuning(const bsort_tuning *in, int key_bytes, Tuning *out) {
    Tuning t;
    if (in) {
        t.radix_bits = in->radix_bits;
        t.unit_keys = in->unit_keys;
        t.merge_keys = in->merge_keys;
        t.chunk_tiles = in->chunk_tiles;
    }
    if (!tuning_valid(key_bytes, t)) return false;
    *out = t;
    return true;
}

// Stable key-value sort of 4- or 8-byte keys by the value-carrying MSD
// path.  Values of 4 or 8 bytes travel with their keys when no positions are
// asked for; otherwise 32-bit input positions travel (made when a key is
// first read), the int64 positions are written beside the sorted keys, and
// the values (any width) follow by one gather along the positions.
bsort_status run_pairs_kv(bsort_handle *h, void *keys, void *values, size_t value_bytes, int64_t *indices, size_t n,
                          const DtypeInfo &di, int descending, void *workspace, cudaStream_t st) {
    (void)cudaGetLastError();
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return BSORT_ERR_CUDA;
    const int sms = num_sms_of(dev);
    if (h->profiling) {
        const bsort_status es = ensure_events(h);
        if (es != BSORT_OK) return es;
    }
    begin_call(h, st);
    const bool carry = values && !indices && (value_bytes == 4 || value_bytes == 8);
    const int cb = carry ? static_cast<int>(value_bytes) : 4;
    const bool gather = !carry && values;
    const PairsKvLayout P = pairs_kv_layout(n, di.bytes, cb, !carry, gather ? value_bytes : 0);
    char *ws = static_cast<char *>(workspace);
    Work wk = make_work(P.msd, ws, keys, n, di, codec_for(di, descending));
    if (carry) {
        wk.vals = values;
        wk.out_vals = values;
    } else {
        wk.out_idx = indices;
        wk.out_vals = gather ? wk.vals : nullptr;
    }
    if (di.bytes == 4) {
        if (cb == 4) launch_msd_kv<uint32_t, uint32_t>(wk, st, h->rec, sms);
        else launch_msd_kv<uint32_t, uint64_t>(wk, st, h->rec, sms);
    } else {
        if (cb == 4) launch_msd_kv<uint64_t, uint32_t>(wk, st, h->rec, sms);
        else launch_msd_kv<uint64_t, uint64_t>(wk, st, h->rec, sms);
    }
    h->last_stream = st;
    h->last_n = n;
    h->last_key_bytes = di.bytes;
    h->last_path = 3;
    h->last_ctl = wk.ctl;
    h->last_inplace = false;
    h->last_fixed_aux = P.total;
    // value bytes written per output element: the carried values, or int64
    // positions (plus the 32-bit ones kept for the gather)
    const int out_bytes = carry ? cb : (indices ? 8 : 0) + (gather ? 4 : 0);
    if (gather) {
        h->rec.begin(BSORT_K_FILL, -1);
        launch_gather(values, static_cast<int>(value_bytes), static_cast<const uint32_t *>(wk.vals), n, ws + P.tmp,
                      wk.ctl, st, sms);
        h->rec.end();
        if (cudaMemcpyAsync(values, ws + P.tmp, value_bytes * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return BSORT_ERR_CUDA;
    }
    end_call(h, st, n, di.bytes, cb, out_bytes);
    return cudaGetLastError() == cudaSuccess ? BSORT_OK : BSORT_ERR_CUDA;
}

}  // namespace

extern "C" {

const char *bsort_status_string(bsort_status status) {
    switch (status) {
    case BSORT_OK: return "BSORT_OK";
    case BSORT_ERR_INVALID_ARG: return "BSORT_ERR_INVALID_ARG: invalid argument";
    case BSORT_ERR_UNSUPPORTED: return "BSORT_ERR_UNSUPPORTED: request the library does not support";
    case BSORT_ERR_MISALIGNED: return "BSORT_ERR_MISALIGNED: pointer not aligned to the key size";
    case BSORT_ERR_NO_MEMORY: return "BSORT_ERR_NO_MEMORY: device allocation failed";
    case BSORT_ERR_WORKSPACE_TOO_SMALL: return "BSORT_ERR_WORKSPACE_TOO_SMALL: workspace smaller than required";
    case BSORT_ERR_CUDA: return "BSORT_ERR_CUDA: a CUDA runtime call failed";
    case BSORT_ERR_TIMEOUT: return "BSORT_ERR_TIMEOUT: a bounded device wait expired";
    case BSORT_ERR_CAPACITY: return "BSORT_ERR_CAPACITY: a device work list outgrew its plan";
    case BSORT_ERR_INTERNAL: return "BSORT_ERR_INTERNAL: a device-side bounds check refused a store";
    }
    return "BSORT_ERR_UNKNOWN";
}

bsort_status bsort_workspace_bytes(size_t n, bsort_dtype dt, bsort_mode mode, size_t *bytes) {
    DtypeInfo di;
    if (!bytes || !dtype_info(dt, &di)) return BSORT_ERR_INVALID_ARG;
    if (mode != BSORT_MODE_PINGPONG && mode != BSORT_MODE_INPLACE) return BSORT_ERR_INVALID_ARG;
    if (mode == BSORT_MODE_INPLACE && di.bytes > 8) return BSORT_ERR_UNSUPPORTED;
    *bytes = workspace_for(n, di, mode == BSORT_MODE_INPLACE);
    return BSORT_OK;
}

bsort_status bsort_handle_create(bsort_handle **handle) {
    if (!handle) return BSORT_ERR_INVALID_ARG;
    *handle = new (std::nothrow) bsort_handle();
    if (!*handle) return BSORT_ERR_NO_MEMORY;
    int dev = 0;
    cudaGetDevice(&dev);
    (*handle)->device = dev;
    return BSORT_OK;
}

bsort_status bsort_handle_destroy(bsort_handle *handle) {
    if (!handle) return BSORT_ERR_INVALID_ARG;
    for (int d = 0; d < 64; ++d)
        if (g_default[d] == handle) return BSORT_ERR_INVALID_ARG;  // default handles live until exit
    if (handle->events) {
        for (int i = 0; i < BSORT_PROFILE_MAX; ++i) {
            cudaEventDestroy(handle->rec.rec[i].a);
            cudaEventDestroy(handle->rec.rec[i].b);
        }
        cudaFree(handle->prof_ctl);
    }
    delete handle;
    return BSORT_OK;
}

bsort_status bsort_keys_ws(bsort_handle *handle, void *keys, size_t n, bsort_dtype dt, int descending,
                           bsort_mode mode, void *workspace, size_t ws_bytes, void *stream) {
    if (!handle) return BSORT_ERR_INVALID_ARG;
    DtypeInfo di;
    const bsort_status st = check_args(keys, n, dt, &di);
    if (st != BSORT_OK) return st;
    if (mode != BSORT_MODE_PINGPONG && mode != BSORT_MODE_INPLACE) return BSORT_ERR_INVALID_ARG;
    if (n <= 1) return BSORT_OK;
    if (!workspace) return BSORT_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(workspace) % kAlign) return BSORT_ERR_MISALIGNED;
    std::lock_guard<std::mutex> lk(handle->mu);
    return run_sort(handle, keys, n, di, descending, workspace, ws_bytes, static_cast<cudaStream_t>(stream),
                    mode == BSORT_MODE_INPLACE);
}

bsort_status bsort_pairs_workspace_bytes(size_t n, bsort_dtype dt, size_t *bytes) {
    DtypeInfo di;
    if (!bytes || !dtype_info(dt, &di)) return BSORT_ERR_INVALID_ARG;
    if (di.bytes > 8) return BSORT_ERR_UNSUPPORTED;
    *bytes = pairs_workspace_for(n, di.bytes);
    return BSORT_OK;
}

bsort_status bsort_pairs_workspace_bytes_tuned(size_t n, bsort_dtype dt, const bsort_tuning *tuning8, size_t *bytes) {
    DtypeInfo di;
    if (!bytes || !dtype_info(dt, &di)) return BSORT_ERR_INVALID_ARG;
    if (di.bytes > 8) return BSORT_ERR_UNSUPPORTED;
    Tuning t;
    if (!to_tuning(tuning8, 8, &t)) return BSORT_ERR_INVALID_ARG;  // (validated; the key-value levels have a fixed shape)
    *bytes = pairs_workspace_for(n, di.bytes);
    return BSORT_OK;
}

bsort_status bsort_pairs_ws(bsort_handle *handle, void *keys, void *values, size_t value_bytes, int64_t *indices,
                            size_t n, bsort_dtype dt, int descending, void *workspace, size_t ws_bytes,
                            void *stream) {
    if (!handle) return BSORT_ERR_INVALID_ARG;
    DtypeInfo di;
    if (!dtype_info(dt, &di)) return BSORT_ERR_INVALID_ARG;
    if (values && value_bytes != 1 && value_bytes != 2 && value_bytes != 4 && value_bytes != 8)
        return BSORT_ERR_INVALID_ARG;
    if (n >= (1ull << 32) || di.bytes > 8) return BSORT_ERR_UNSUPPORTED;  // positions travel in 32 bits
    if (n == 0) return BSORT_OK;
    if (!keys) return BSORT_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(keys) % di.bytes || (values && reinterpret_cast<uintptr_t>(values) % value_bytes) ||
        reinterpret_cast<uintptr_t>(indices) % 8)
        return BSORT_ERR_MISALIGNED;
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> lk(handle->mu);
    if (n == 1) {  // one element: position 0, nothing moves
        handle->rec.launches = 0;
        if (indices && cudaMemsetAsync(indices, 0, 8, st) != cudaSuccess) return BSORT_ERR_CUDA;
        return BSORT_OK;
    }
    if (!workspace) return BSORT_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(workspace) % kAlign) return BSORT_ERR_MISALIGNED;
    if (ws_bytes < pairs_workspace_for(n, di.bytes)) return BSORT_ERR_WORKSPACE_TOO_SMALL;
    if (!values && !indices) {  // equal keys are bit-identical: the keys-only sort gives the same keys
        const Tuning defaults;
        return run_sort(handle, keys, n, di, descending, workspace, ws_bytes, st, false, &defaults);
    }
    if (di.bytes >= 4) return run_pairs_kv(handle, keys, values, value_bytes, indices, n, di, descending, workspace, st);
    // 1- and 2-byte keys: their order codes as 32-bit words, sorted as
    // unsigned keys carrying the values (or positions), then narrowed back
    (void)cudaGetLastError();
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return BSORT_ERR_CUDA;
    const int sms = num_sms_of(dev);
    const Codec codec = codec_for(di, descending);
    uint32_t *wide = static_cast<uint32_t *>(workspace);
    launch_widen(keys, di.bytes, n, codec, wide, st, sms);
    DtypeInfo word;
    dtype_info(BSORT_U32, &word);
    const bsort_status s = run_pairs_kv(handle, wide, values, value_bytes, indices, n, word, 0,
                                        static_cast<char *>(workspace) + align_up(4 * n), st);
    if (s != BSORT_OK) return s;
    launch_narrow(wide, di.bytes, n, codec, keys, st, sms);
    handle->rec.launches += 2;
    return cudaGetLastError() == cudaSuccess ? BSORT_OK : BSORT_ERR_CUDA;
}

bsort_status bsort_keys(void *keys, size_t n, bsort_dtype dt, int descending, void *stream) {
    DtypeInfo di;
    const bsort_status st = check_args(keys, n, dt, &di);
    if (st != BSORT_OK) return st;
    if (n <= 1) return BSORT_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return BSORT_ERR_CUDA;
    bsort_handle *h = default_handle(dev);
    if (!h) return BSORT_ERR_NO_MEMORY;
    std::lock_guard<std::mutex> lk(h->mu);
    const bsort_status gs = grow(&h->ws, &h->ws_bytes, workspace_for(n, di));
    if (gs != BSORT_OK) return gs;
    return run_sort(h, keys, n, di, descending, h->ws, h->ws_bytes, static_cast<cudaStream_t>(stream));
}

bsort_status bsort_keys_host(void *host_keys, size_t n, bsort_dtype dt, int descending, void *stream) {
    DtypeInfo di;
    const bsort_status st = check_args(host_keys, n, dt, &di);
    if (st != BSORT_OK) return st;
    if (n <= 1) return BSORT_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return BSORT_ERR_CUDA;
    bsort_handle *h = default_handle(dev);
    if (!h) return BSORT_ERR_NO_MEMORY;
    std::lock_guard<std::mutex> lk(h->mu);
    const size_t bytes = n * di.bytes;
    bsort_status gs = grow(&h->stage, &h->stage_bytes, bytes);
    if (gs != BSORT_OK) return gs;
    gs = grow(&h->ws, &h->ws_bytes, workspace_for(n, di));
    if (gs != BSORT_OK) return gs;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(h->stage, host_keys, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) return BSORT_ERR_CUDA;
    const bsort_status rs = run_sort(h, h->stage, n, di, descending, h->ws, h->ws_bytes, s);
    if (rs != BSORT_OK) return rs;
    if (cudaMemcpyAsync(host_keys, h->stage, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess) return BSORT_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return BSORT_ERR_CUDA;
    if (h->last_ctl) {
        uint32_t err = 0;
        if (cudaMemcpy(&err, &h->last_ctl->error, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return BSORT_ERR_CUDA;
        if (err & kErrCapacity) return BSORT_ERR_CAPACITY;
        if (err & kErrTimeout) return BSORT_ERR_TIMEOUT;
        if (err & kErrBounds) return BSORT_ERR_INTERNAL;
    }
    return BSORT_OK;
}

bsort_status bsort_segmented_workspace_bytes(size_t n, size_t num_segments, bsort_dtype dt, size_t *bytes) {
    DtypeInfo di;
    if (!bytes || !dtype_info(dt, &di)) return BSORT_ERR_INVALID_ARG;
    if (di.bytes < 4) return BSORT_ERR_UNSUPPORTED;
    *bytes = msd_layout(n, di.bytes, num_segments).total;
    return BSORT_OK;
}

bsort_status bsort_segmented_workspace_bytes_tuned(size_t n, size_t num_segments, bsort_dtype dt,
                                                   const bsort_tuning *tuning, size_t *bytes) {
    DtypeInfo di;
    if (!bytes || !dtype_info(dt, &di)) return BSORT_ERR_INVALID_ARG;
    if (di.bytes < 4) return BSORT_ERR_UNSUPPORTED;
    Tuning t;
    if (!to_tuning(tuning, di.bytes, &t)) return BSORT_ERR_INVALID_ARG;
    if (di.bytes == 16) t = Tuning();  // 16-byte keys run the defaults
    *bytes = msd_layout(n, di.bytes, num_segments, false, t).total;
    return BSORT_OK;
}

bsort_status bsort_keys_segmented_ws(bsort_handle *handle, void *keys, size_t n, const uint64_t *d_offsets,
                                     size_t num_segments, bsort_dtype dt, int descending, void *workspace,
                                     size_t ws_bytes, void *stream) {
    if (!handle) return BSORT_ERR_INVALID_ARG;
    DtypeInfo di;
    const bsort_status st = check_segmented(keys, n, d_offsets, num_segments, dt, &di);
    if (st != BSORT_OK || num_segments == 0 || n == 0) return st;
    if (!workspace) return BSORT_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(workspace) % kAlign) return BSORT_ERR_MISALIGNED;
    std::lock_guard<std::mutex> lk(handle->mu);
    return run_segmented(handle, keys, n, d_offsets, num_segments, di, descending, workspace, ws_bytes,
                         static_cast<cudaStream_t>(stream), true);
}

bsort_status bsort_keys_segmented(void *keys, size_t n, const uint64_t *d_offsets, size_t num_segments,
                                  bsort_dtype dt, int descending, void *stream) {
    DtypeInfo di;
    const bsort_status st = check_segmented(keys, n, d_offsets, num_segments, dt, &di);
    if (st != BSORT_OK || num_segments == 0 || n == 0) return st;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return BSORT_ERR_CUDA;
    bsort_handle *h = default_handle(dev);
    if (!h) return BSORT_ERR_NO_MEMORY;
    std::lock_guard<std::mutex> lk(h->mu);
    const bsort_status gs =
        grow(&h->ws, &h->ws_bytes, msd_layout(n, di.bytes, num_segments, false, tune_of(h, di.bytes)).total);
    if (gs != BSORT_OK) return gs;
    return run_segmented(h, keys, n, d_offsets, num_segments, di, descending, h->ws, h->ws_bytes,
                         static_cast<cudaStream_t>(stream), true);
}

struct bsort_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    Ctl *ctl = nullptr;
};

namespace {
// Captures one sort (plain: d_offsets == NULL) into an executable graph.
bsort_status capture(bsort_handle *h, void *keys, size_t n, const uint64_t *d_offsets, size_t nseg,
                     const DtypeInfo &di, int descending, void *ws, size_t ws_bytes, bsort_graph **out) {
    if (di.bytes == 4) msd_prepare<uint32_t>();
    else if (di.bytes == 8) msd_prepare<uint64_t>();
    else if (di.bytes == 16) msd_prepare<u128>();
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return BSORT_ERR_CUDA;
    bsort_graph *g = new (std::nothrow) bsort_graph();
    if (!g) {
        cudaStreamDestroy(cs);
        return BSORT_ERR_NO_MEMORY;
    }
    bsort_status st = BSORT_OK;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) st = BSORT_ERR_CUDA;
    if (st == BSORT_OK) {
        const bool prof = h->profiling;
        h->profiling = false;
        st = d_offsets ? run_segmented(h, keys, n, d_offsets, nseg, di, descending, ws, ws_bytes, cs, false)
                       : run_sort(h, keys, n, di, descending, ws, ws_bytes, cs);
        h->profiling = prof;
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(cs, &graph);
        if (st == BSORT_OK && e != cudaSuccess) st = BSORT_ERR_CUDA;
        g->graph = graph;
        if (st == BSORT_OK && cudaGraphInstantiate(&g->exec, graph, 0) != cudaSuccess) st = BSORT_ERR_CUDA;
    }
    g->ctl = h->last_ctl;
    cudaStreamDestroy(cs);
    if (st != BSORT_OK) {
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->graph) cudaGraphDestroy(g->graph);
        delete g;
        (void)cudaGetLastError();
        return st;
    }
    *out = g;
    return BSORT_OK;
}
}  // namespace

bsort_status bsort_graph_create(bsort_handle *handle, void *keys, size_t n, bsort_dtype dt, int descending,
                                void *workspace, size_t ws_bytes, bsort_graph **graph) {
    if (!handle || !graph) return BSORT_ERR_INVALID_ARG;
    DtypeInfo di;
    const bsort_status st = check_args(keys, n, dt, &di);
    if (st != BSORT_OK) return st;
    if (n <= 1 || !workspace) return BSORT_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(handle->mu);
    return capture(handle, keys, n, nullptr, 0, di, descending, workspace, ws_bytes, graph);
}

bsort_status bsort_graph_create_segmented(bsort_handle *handle, void *keys, size_t n, const uint64_t *d_offsets,
                                          size_t num_segments, bsort_dtype dt, int descending, void *workspace,
                                          size_t ws_bytes, bsort_graph **graph) {
    if (!handle || !graph) return BSORT_ERR_INVALID_ARG;
    DtypeInfo di;
    const bsort_status st = check_segmented(keys, n, d_offsets, num_segments, dt, &di);
    if (st != BSORT_OK) return st;
    if (num_segments == 0 || n == 0 || !workspace) return BSORT_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(handle->mu);
    return capture(handle, keys, n, d_offsets, num_segments, di, descending, workspace, ws_bytes, graph);
}

bsort_status bsort_graph_launch(bsort_graph *graph, void *stream) {
    if (!graph || !graph->exec) return BSORT_ERR_INVALID_ARG;
    return cudaGraphLaunch(graph->exec, static_cast<cudaStream_t>(stream)) == cudaSuccess ? BSORT_OK
                                                                                          : BSORT_ERR_CUDA;
}

bsort_status bsort_graph_error(bsort_graph *graph, void *stream) {
    if (!graph) return BSORT_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return BSORT_ERR_CUDA;
    if (!graph->ctl) return BSORT_OK;
    uint32_t err = 0;
    if (cudaMemcpy(&err, &graph->ctl->error, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return BSORT_ERR_CUDA;
    if (err & kErrCapacity) return BSORT_ERR_CAPACITY;
    if (err & kErrTimeout) return BSORT_ERR_TIMEOUT;
    if (err & kErrBounds) return BSORT_ERR_INTERNAL;
    return BSORT_OK;
}

bsort_status bsort_graph_destroy(bsort_graph *graph) {
    if (!graph) return BSORT_ERR_INVALID_ARG;
    if (graph->exec) cudaGraphExecDestroy(graph->exec);
    if (graph->graph) cudaGraphDestroy(graph->graph);
    delete graph;
    return BSORT_OK;
}

bsort_status bsort_handle_set_tuning(bsort_handle *handle, int key_bytes, const bsort_tuning *tuning) {
    if (!handle || (key_bytes != 4 && key_bytes != 8)) return BSORT_ERR_INVALID_ARG;
    Tuning t;
    if (!to_tuning(tuning, key_bytes, &t)) return BSORT_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(handle->mu);
    handle->tune[key_bytes == 8] = t;
    return BSORT_OK;
}

bsort_status bsort_workspace_bytes_tuned(size_t n, bsort_dtype dt, bsort_mode mode, const bsort_tuning *tuning,
                                         size_t *bytes) {
    DtypeInfo di;
    if (!bytes || !dtype_info(dt, &di)) return BSORT_ERR_INVALID_ARG;
    if (mode != BSORT_MODE_PINGPONG && mode != BSORT_MODE_INPLACE) return BSORT_ERR_INVALID_ARG;
    if (mode == BSORT_MODE_INPLACE && di.bytes > 8) return BSORT_ERR_UNSUPPORTED;
    Tuning t;
    if (di.bytes >= 4 && !to_tuning(tuning, di.bytes, &t)) return BSORT_ERR_INVALID_ARG;
    if (di.bytes == 16) t = Tuning();  // 16-byte keys run the defaults
    *bytes = workspace_for(n, di, mode == BSORT_MODE_INPLACE, t);
    return BSORT_OK;
}

bsort_status bsort_last_aux_bytes(bsort_handle *handle, size_t *bytes) {
    if (!handle || !bytes) return BSORT_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(handle->mu);
    *bytes = 0;
    if (handle->last_path == 0) return BSORT_OK;
    size_t used = handle->last_fixed_aux;
    if (handle->last_path == 2 && handle->last_inplace && handle->last_ctl) {
        if (cudaStreamSynchronize(handle->last_stream) != cudaSuccess) return BSORT_ERR_CUDA;
        unsigned long long aux = 0;
        if (cudaMemcpy(&aux, &handle->last_ctl->aux_used, sizeof(aux), cudaMemcpyDeviceToHost) != cudaSuccess)
            return BSORT_ERR_CUDA;
        used += static_cast<size_t>(aux);
    }
    *bytes = used;
    return BSORT_OK;
}

bsort_status bsort_keys_partial_ws(bsort_handle *handle, void *keys, size_t n, bsort_dtype dt, int descending,
                                   int levels, void *workspace, size_t ws_bytes, void *stream) {
    if (!handle || levels < 1) return BSORT_ERR_INVALID_ARG;
    DtypeInfo di;
    const bsort_status st = check_args(keys, n, dt, &di);
    if (st != BSORT_OK) return st;
    if (di.bytes <= 2) return BSORT_ERR_UNSUPPORTED;
    if (n <= 1) return BSORT_OK;
    if (!workspace) return BSORT_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(workspace) % kAlign) return BSORT_ERR_MISALIGNED;
    std::lock_guard<std::mutex> lk(handle->mu);
    handle->stop_levels = levels;
    const bsort_status rs = run_sort(handle, keys, n, di, descending, workspace, ws_bytes,
                                     static_cast<cudaStream_t>(stream));
    handle->stop_levels = 0;
    return rs;
}

bsort_status bsort_top_digit_counts(const void *keys, size_t n, bsort_dtype dt, int descending, int bits,
                                    uint64_t *d_counts, void *stream) {
    DtypeInfo di;
    if (!dtype_info(dt, &di)) return BSORT_ERR_INVALID_ARG;
    if (di.bytes > 8) return BSORT_ERR_UNSUPPORTED;
    if (bits < 1 || bits > kDigitCountsMaxBits || bits > di.bytes * 8 || !d_counts) return BSORT_ERR_INVALID_ARG;
    if (n > 0 && !keys) return BSORT_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(keys) % di.bytes || reinterpret_cast<uintptr_t>(d_counts) % 8)
        return BSORT_ERR_MISALIGNED;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(d_counts, 0, sizeof(uint64_t) << bits, st) != cudaSuccess) return BSORT_ERR_CUDA;
    if (n == 0) return BSORT_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return BSORT_ERR_CUDA;
    launch_digit_counts(keys, di.bytes, n, codec_for(di, descending), bits,
                        reinterpret_cast<unsigned long long *>(d_counts), st, num_sms_of(dev));
    return cudaGetLastError() == cudaSuccess ? BSORT_OK : BSORT_ERR_CUDA;
}

bsort_status bsort_selftest_bounded_wait(void *stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint32_t *d = nullptr;
    if (cudaMalloc(&d, 2 * sizeof(uint32_t)) != cudaSuccess) {
        (void)cudaGetLastError();
        return BSORT_ERR_NO_MEMORY;
    }
    uint32_t h[2] = {0, 0};
    bsort_status rs = BSORT_ERR_CUDA;
    if (cudaMemsetAsync(d, 0, 2 * sizeof(uint32_t), st) == cudaSuccess) {
        launch_wait_selftest(d, st);
        if (cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
            cudaStreamSynchronize(st) == cudaSuccess)
            rs = (h[1] & kErrTimeout) ? BSORT_ERR_TIMEOUT : BSORT_OK;
    }
    cudaFree(d);
    return rs;
}

bsort_status bsort_get_error(bsort_handle *handle, void *stream) {
    if (!handle) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return BSORT_ERR_CUDA;
        handle = default_handle(dev);
        if (!handle) return BSORT_ERR_NO_MEMORY;
    }
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return BSORT_ERR_CUDA;
    if (!handle->last_ctl) return BSORT_OK;
    uint32_t err = 0;
    if (cudaMemcpy(&err, &handle->last_ctl->error, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return BSORT_ERR_CUDA;
    if (err) {
        const uint32_t zero = 0;
        cudaMemcpy(&handle->last_ctl->error, &zero, 4, cudaMemcpyHostToDevice);
    }
    if (err & kErrCapacity) return BSORT_ERR_CAPACITY;
    if (err & kErrTimeout) return BSORT_ERR_TIMEOUT;
    if (err & kErrBounds) return BSORT_ERR_INTERNAL;
    return BSORT_OK;
}

bsort_status bsort_handle_set_profiling(bsort_handle *handle, int enable) {
    if (!handle) return BSORT_ERR_INVALID_ARG;
    handle->profiling = enable != 0;
    return BSORT_OK;
}

bsort_status bsort_last_launch_count(bsort_handle *handle, int *launches) {
    if (!handle || !launches) return BSORT_ERR_INVALID_ARG;
    *launches = handle->rec.launches;
    return BSORT_OK;
}

bsort_status bsort_handle_get_profile(bsort_handle *handle, bsort_profile *out) {
    if (!handle || !out) return BSORT_ERR_INVALID_ARG;
    std::memset(out, 0, sizeof(*out));
    if (cudaDeviceSynchronize() != cudaSuccess) return BSORT_ERR_CUDA;
    const int ncalls = handle->rec.calls;
    Ctl ctls[BSORT_PROFILE_MAX_CALLS];
    if (ncalls > 0 && handle->prof_ctl &&
        cudaMemcpy(ctls, handle->prof_ctl, sizeof(Ctl) * ncalls, cudaMemcpyDeviceToHost) != cudaSuccess)
        return BSORT_ERR_CUDA;
    out->num_calls = ncalls;
    out->num_launches = handle->rec.held_launches;
    for (int c = 0; c < ncalls; ++c) {
        out->finish_units_counting += ctls[c].fin_counting;
        out->finish_units_compare += ctls[c].fin_compare;
        out->finish_units_lsd += ctls[c].n_fb;
        out->finish_units_counting_fast += ctls[c].fin_fast;
    }
    const int nrec = handle->rec.count;
    for (int i = 0; i < nrec; ++i) {
        bsort_profile_record &r = out->rec[i];
        const Recorder::Rec &src = handle->rec.rec[i];
        r.kind = src.kind;
        r.level = src.level;
        r.call = src.call;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, src.a, src.b) != cudaSuccess) ms = -1.f;
        r.ms = ms;
        const Ctl &ctl = ctls[src.call];
        const uint64_t b = static_cast<uint64_t>(handle->prof_key_bytes[src.call]);
        const uint64_t n = handle->prof_n[src.call];
        // key-value calls: vb value bytes read with each key, ob written
        const uint64_t vb = static_cast<uint64_t>(handle->prof_val_bytes[src.call]);
        const uint64_t ob = static_cast<uint64_t>(handle->prof_out_bytes[src.call]);
        uint64_t keys = 0, bytes = 0;
        switch (r.kind) {
        case BSORT_K_HIST:
            keys = r.level >= 0 && r.level < kMaxLevels ? ctl.hist_keys[r.level] : 0;
            bytes = keys * b;
            break;
        case BSORT_K_SCATTER:
            keys = r.level >= 0 && r.level < kMaxLevels ? ctl.scatter_keys[r.level] : 0;
            bytes = 2 * keys * (b + vb);
            break;
        case BSORT_K_FINISH:
            keys = ctl.finish_keys;
            bytes = vb ? keys * (2 * b + vb + ob) : 2 * keys * b;
            break;
        case BSORT_K_FILL:
            keys = ctl.fill_keys;
            bytes = vb ? keys * (b + vb + ob) : keys * b;  // (an upper bound: runs in place move no values)
            break;
        case BSORT_K_COUNT_HIST:
        case BSORT_K_COUNT_FILL:
            keys = n;
            bytes = keys * b;
            break;
        default:
            break;
        }
        r.keys = keys;
        r.counted_bytes = bytes;
    }
    out->num_records = nrec;
    handle->rec.count = 0;
    handle->rec.calls = 0;
    handle->rec.held_launches = 0;
    (void)cudaGetLastError();
    return BSORT_OK;
}

}  // extern "C"
