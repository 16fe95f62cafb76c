// MSD digit-pass kernels of the bsort library (sm_103a), for 4- and 8-byte keys.
//
// One MSD level over every open bucket runs four launches:
//   k_hist      per chunk: key transform (first touch only) + digit histogram
//               + AND/OR of the keys (common-prefix detection)
//   k_colscan   per digit: exclusive prefix of the chunk counts inside each
//               bucket (segmented scan over the chunk list)
//   k_classify  per bucket: digit bases, then each child bucket becomes a
//               shared-memory finish unit, a bucket of the next level, or a
//               constant fill; buckets whose digit is constant skip ahead to
//               their highest varying bit without moving
//   k_scatter   per chunk: stable shared-memory digit ranking of each tile and
//               a scatter of the digit runs to their bucket offsets
// and after the last level k_finish sorts every unit in shared memory (LSD
// passes over its varying bits) and k_fill writes constant runs.
//
// The fixed launch sequence reads all work counts from device memory, so a
// call has no host synchronisation and no data-dependent host logic.
#include <cstdio>

#include "bsort_launch.h"

namespace bsort {

namespace {

constexpr unsigned kFull = 0xffffffffu;
// comparison finish: largest sub-bucket, and comparisons per key one LSD pass is worth
constexpr uint32_t kCmpMaxBucket = 64;
constexpr int kSplitBits = 12;  // finish split: up to 4096 sub-buckets per unit
constexpr int kSplitCap = 1 << kSplitBits;

// Programmatic dependent launch: every kernel of the sequence is launched
// with programmatic stream serialization, so it may be scheduled while its
// predecessor still runs; it first waits for the predecessor's completion
// (and memory) and then lets its own successor start launching.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <int THREADS>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *tmp, uint32_t &total) {
    constexpr int WARPS = THREADS / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) tmp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t s = lane < WARPS ? tmp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(kFull, s, o);
            if (lane >= o) s += y;
        }
        if (lane < WARPS) tmp[lane] = s;
    }
    __syncthreads();
    const uint32_t warp_excl = warp ? tmp[warp - 1] : 0;
    total = tmp[WARPS - 1];
    __syncthreads();
    return warp_excl + x - v;
}

template <int THREADS>
__device__ __forceinline__ unsigned long long block_exclusive_scan64(unsigned long long v, unsigned long long *tmp,
                                                                     unsigned long long &total) {
    constexpr int WARPS = THREADS / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) tmp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        unsigned long long s = lane < WARPS ? tmp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(kFull, s, o);
            if (lane >= o) s += y;
        }
        if (lane < WARPS) tmp[lane] = s;
    }
    __syncthreads();
    const unsigned long long warp_excl = warp ? tmp[warp - 1] : 0;
    total = tmp[WARPS - 1];
    __syncthreads();
    return warp_excl + x - v;
}

// Inclusive max-scan across the block (int values).
template <int THREADS>
__device__ __forceinline__ int block_inclusive_max(int v, int *tmp) {
    constexpr int WARPS = THREADS / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x = max(x, y);
    }
    if (lane == 31) tmp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int s = lane < WARPS ? tmp[lane] : -1;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(kFull, s, o);
            if (lane >= o) s = max(s, y);
        }
        if (lane < WARPS) tmp[lane] = s;
    }
    __syncthreads();
    const int r = warp ? max(x, tmp[warp - 1]) : x;
    __syncthreads();
    return r;
}

// AND / OR of one value per thread, result broadcast to every thread.
template <int THREADS>
__device__ __forceinline__ void block_and_or(unsigned long long &a, unsigned long long &o, unsigned long long *ta,
                                             unsigned long long *to) {
    constexpr int WARPS = THREADS / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        a &= __shfl_xor_sync(kFull, a, s);
        o |= __shfl_xor_sync(kFull, o, s);
    }
    if (lane == 0) {
        ta[warp] = a;
        to[warp] = o;
    }
    __syncthreads();
    a = ~0ull;
    o = 0;
#pragma unroll
    for (int w = 0; w < WARPS; ++w) {
        a &= ta[w];
        o |= to[w];
    }
    __syncthreads();
}

// Dynamic shared memory of every kernel below; each kernel lays its buffers
// out at compile-time offsets, so addresses are one base plus a constant.
extern __shared__ __align__(16) unsigned char g_dyn_smem[];

// 16-byte asynchronous copy global -> shared (no register, no stall until
// the wait), used to fetch the next work descriptor a unit ahead.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(smem))),
                 "l"(gmem)
                 : "memory");
    asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(smem))),
                 "l"(gmem)
                 : "memory");
}

// What the scatter needs of one chunk before it can stage keys: the chunk,
// the next chunk (same bucket or not), the bucket, and per digit the chunk's
// exclusive prefix, the next chunk's, and the bucket's digit base.
template <int NB>
struct ScatterPre {
    Chunk ch, chn;
    Bucket b;
    uint32_t hc[NB], hn[NB], bb[NB];
};

// Shared-memory buffers of one tile ranking, at byte offset BASE of dynamic
// shared memory.  Unstable ranking uses one CTA-wide counter row; stable
// ranking uses per-digit, per-warp counters laid out digit-major with one pad
// word per digit (stride WARPS + 1: the banks of a warp's counters spread,
// and the thread that scans digit d reads its WARPS counters at consecutive
// words) and two sets of per-warp peer masks.
template <int THREADS, size_t BASE, bool STABLE_BUFS>
struct RankSmem {
    static constexpr int WARPS = THREADS / 32;
    static constexpr int STRIDE = WARPS + 1;
    static constexpr size_t kCnt = BASE;
    static constexpr size_t kDstart = kCnt + 4 * kBins;
    static constexpr size_t kDcount = kDstart + 4 * kBins;
    static constexpr size_t kScan = kDcount + 4 * kBins;
    static constexpr size_t kWc = kScan + 16 * ((4 * (WARPS + 1) + 15) / 16);
    static constexpr size_t kWm = kWc + 16 * ((4 * kBins * STRIDE + 15) / 16);
    static constexpr size_t kEnd = STABLE_BUFS ? kWm + 8 * WARPS * kBins : kWc;
    __device__ static uint32_t *cnt() { return reinterpret_cast<uint32_t *>(g_dyn_smem + kCnt); }
    __device__ static uint32_t *dstart() { return reinterpret_cast<uint32_t *>(g_dyn_smem + kDstart); }
    __device__ static uint32_t *dcount() { return reinterpret_cast<uint32_t *>(g_dyn_smem + kDcount); }
    __device__ static uint32_t *scan() { return reinterpret_cast<uint32_t *>(g_dyn_smem + kScan); }
    __device__ static uint32_t *wc() { return reinterpret_cast<uint32_t *>(g_dyn_smem + kWc); }
    __device__ static uint32_t *wm() { return reinterpret_cast<uint32_t *>(g_dyn_smem + kWm); }
};

// Rank of a tile of keys held in registers (ITEMS per thread, bit j of
// `vmask` set for valid items) by digit (k >> shift) & mask, then placement
// of the valid keys in `out` in digit order; dstart / dcount describe the
// digit runs of the tile.
//
//  STABLE = false: one CTA-wide counter row; a key's rank among equal digits
//    is the value its shared-memory atomicAdd returns, so equal digits land in
//    arbitrary relative order.  That suffices wherever equal digits carry no
//    order to keep: every MSD digit pass, and the first LSD pass of a finish
//    (its input order is arbitrary).  A warp step whose 32 keys share one
//    digit (sorted or skewed data) takes one atomic for the whole warp.
//  STABLE = true: items are in warp-striped tile order (item j of lane l is
//    index warp*32*ITEMS + j*32 + l, valid items a prefix).  Lanes with equal
//    digits find each other through an atomicOr of their lane bit into the
//    warp's peer-mask word of that digit (two mask sets alternate by item, so
//    a set is cleared before its next use without a third barrier); the rank
//    is the number of lower lanes in the group plus the warp's count before
//    the step, so equal digits keep tile order.
template <typename K, int THREADS, int ITEMS, typename RS>
struct Ranker {
    static constexpr int WARPS = THREADS / 32;
    static constexpr int STRIDE = WARPS + 1;
    static_assert(THREADS >= kBins, "one thread per digit in the scans");

    template <bool STABLE>
    __device__ static void rank_and_place(const K (&keys)[ITEMS], uint32_t vmask, int shift, uint32_t mask, K *out) {
        struct {
            uint32_t *cnt = RS::cnt(), *dstart = RS::dstart(), *dcount = RS::dcount(), *scan = RS::scan(),
                     *wc = RS::wc(), *wm = RS::wm();
        } s;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const int t = threadIdx.x;
        // rank of each item among equal digits (< TILE), two per register
        uint32_t local[(ITEMS + 1) / 2];
#pragma unroll
        for (int j = 0; j < (ITEMS + 1) / 2; ++j) local[j] = 0;
        if (!STABLE) {
            if (t <= static_cast<int>(mask)) s.cnt[t] = 0;
            __syncthreads();
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) {
                const bool valid = (vmask >> j) & 1u;
                const uint32_t d = static_cast<uint32_t>(keys[j] >> shift) & mask;
                const uint32_t d0 = __shfl_sync(kFull, d, 0);
                uint32_t r;
                if (__all_sync(kFull, valid && d == d0)) {
                    uint32_t b = 0;
                    if (lane == 0) b = atomicAdd(&s.cnt[d0], 32u);
                    r = __shfl_sync(kFull, b, 0) + lane;
                } else {
                    r = valid ? atomicAdd(&s.cnt[d], 1u) : 0u;
                }
                local[j >> 1] |= r << ((j & 1) * 16);
            }
            __syncthreads();
            const uint32_t v = t <= static_cast<int>(mask) ? s.cnt[t] : 0u;
            uint32_t total;
            const uint32_t ex = block_exclusive_scan<THREADS>(v, s.scan, total);
            if (t <= static_cast<int>(mask)) {
                s.dstart[t] = ex;
                s.dcount[t] = v;
            }
            __syncthreads();
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) {
                if ((vmask >> j) & 1u) {
                    const uint32_t d = static_cast<uint32_t>(keys[j] >> shift) & mask;
                    out[s.dstart[d] + ((local[j >> 1] >> ((j & 1) * 16)) & 0xffffu)] = keys[j];
                }
            }
            __syncthreads();
        } else {
            for (int i = t; i < (static_cast<int>(mask) + 1) * STRIDE; i += THREADS) s.wc[i] = 0;
            __syncthreads();
            const unsigned lt = lanemask_lt();
            const unsigned bit = 1u << lane;
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) {
                const bool valid = (vmask >> j) & 1u;
                if (__any_sync(kFull, valid)) {  // warp-uniform
                    uint32_t *wm = s.wm + ((j & 1) * WARPS + warp) * kBins;
                    const uint32_t d = static_cast<uint32_t>(keys[j] >> shift) & mask;
                    uint32_t *wcd = s.wc + d * STRIDE + warp;
                    if (valid) atomicOr(&wm[d], bit);
                    __syncwarp();
                    const uint32_t peers = wm[d];
                    const uint32_t before = *wcd;
                    __syncwarp();
                    const uint32_t r = __popc(peers & lt);
                    if (valid && r == 0) {
                        *wcd = before + __popc(peers);
                        wm[d] = 0;
                    }
                    local[j >> 1] |= (before + r) << ((j & 1) * 16);
                }
            }
            __syncthreads();
            // thread d: total of digit d, prefix over digits, then the exclusive
            // prefix over warps written back as absolute tile offsets
            uint32_t run = 0;
            if (t <= static_cast<int>(mask)) {
#pragma unroll
                for (int w = 0; w < WARPS; ++w) run += s.wc[t * STRIDE + w];
            }
            uint32_t total;
            const uint32_t ex = block_exclusive_scan<THREADS>(run, s.scan, total);
            if (t <= static_cast<int>(mask)) {
                s.dstart[t] = ex;
                s.dcount[t] = run;
                uint32_t acc = ex;
#pragma unroll
                for (int w = 0; w < WARPS; ++w) {
                    const uint32_t x = s.wc[t * STRIDE + w];
                    s.wc[t * STRIDE + w] = acc;
                    acc += x;
                }
            }
            __syncthreads();
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) {
                if ((vmask >> j) & 1u) {
                    const uint32_t d = static_cast<uint32_t>(keys[j] >> shift) & mask;
                    out[s.wc[d * STRIDE + warp] + ((local[j >> 1] >> ((j & 1) * 16)) & 0xffffu)] = keys[j];
                }
            }
            __syncthreads();
        }
    }
};

// Loads the keys of the tile-relative range [lo_r, hi_r) of the 16-byte-
// aligned window starting at element `wstart` into registers.  Window index
// of item j of a thread: warp w owns [w*32*ITEMS, (w+1)*32*ITEMS); its group
// g = j / V (V keys per 16 bytes) of lane l covers ((w*G + g)*32 + l)*V +
// (j % V), so a warp reads 512 contiguous bytes per group.  Whole in-range
// vectors are one 16-byte load when `vec_ok` (buffer base 16-byte aligned);
// boundary vectors are scalar.  Returns the validity mask (bit j: item j
// holds a key).
template <typename K, int THREADS, int ITEMS>
struct TileLoad {
    static constexpr int V = 16 / static_cast<int>(sizeof(K));
    static constexpr int G = ITEMS / V;
    static_assert(ITEMS % V == 0, "items must be whole vectors");

    // Whole window in range and 16-byte aligned: plain vector loads.
    __device__ static void load_full(const K *__restrict__ w, K (&k)[ITEMS]) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const uint4 q = __ldcs(reinterpret_cast<const uint4 *>(w + ((warp * G + g) * 32 + lane) * V));
            memcpy(&k[g * V], &q, 16);
        }
    }

    __device__ static uint32_t load(const K *__restrict__ src, uint64_t wstart, uint32_t lo_r, uint32_t hi_r,
                                    bool vec_ok, K (&k)[ITEMS]) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const K *w = src + wstart;
        uint32_t vmask = 0;
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const uint32_t r0 = static_cast<uint32_t>(((warp * G + g) * 32 + lane) * V);
            if (vec_ok && r0 >= lo_r && r0 + V <= hi_r) {
                const uint4 q = __ldcs(reinterpret_cast<const uint4 *>(w + r0));
                memcpy(&k[g * V], &q, 16);
                vmask |= ((1u << V) - 1) << (g * V);
            } else {
#pragma unroll
                for (int e = 0; e < V; ++e) {
                    const uint32_t r = r0 + e;
                    const bool ok = r >= lo_r && r < hi_r;
                    k[g * V + e] = ok ? w[r] : K(0);
                    vmask |= static_cast<uint32_t>(ok) << (g * V + e);
                }
            }
        }
        return vmask;
    }
};

// Validity mask of warp-striped items whose tile index is below n_valid.
template <int ITEMS>
__device__ __forceinline__ uint32_t striped_mask(int n_valid) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int rem = n_valid - warp * 32 * ITEMS - lane;  // item j valid iff j*32 < rem
    uint32_t m = 0;
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) m |= static_cast<uint32_t>(j * 32 < rem) << j;
    return m;
}

// Maximum / sum of one value per thread, broadcast to every thread.
template <int THREADS>
__device__ __forceinline__ uint32_t block_reduce_max(uint32_t v, uint32_t *tmp) {
    constexpr int WARPS = THREADS / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = __reduce_max_sync(kFull, v);
    if (lane == 0) tmp[warp] = v;
    __syncthreads();
    uint32_t r = 0;
#pragma unroll
    for (int w = 0; w < WARPS; ++w) r = max(r, tmp[w]);
    __syncthreads();
    return r;
}

template <int THREADS>
__device__ __forceinline__ uint32_t block_reduce_sum(uint32_t v, uint32_t *tmp) {
    constexpr int WARPS = THREADS / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = __reduce_add_sync(kFull, v);
    if (lane == 0) tmp[warp] = v;
    __syncthreads();
    uint32_t r = 0;
#pragma unroll
    for (int w = 0; w < WARPS; ++w) r += tmp[w];
    __syncthreads();
    return r;
}

// AND / OR of one key per thread (key width), broadcast to every thread.
template <typename K, int THREADS>
__device__ __forceinline__ void block_and_or_k(K &a, K &o, K *ta, K *to) {
    constexpr int WARPS = THREADS / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        a &= shfl_xor_k(a, s);
        o |= shfl_xor_k(o, s);
    }
    if (lane == 0) {
        ta[warp] = a;
        to[warp] = o;
    }
    __syncthreads();
    a = static_cast<K>(~K(0));
    o = 0;
#pragma unroll
    for (int w = 0; w < WARPS; ++w) {
        a &= ta[w];
        o |= to[w];
    }
    __syncthreads();
}

template <typename K>
__device__ __forceinline__ const K *src_of(const Work &wk, int src) {
    return static_cast<const K *>(src ? wk.alt : wk.keys);
}

template <typename K>
__device__ __forceinline__ K *dst_of(const Work &wk, int src) {
    return static_cast<K *>(src ? wk.keys : wk.alt);
}

// ---------------------------------------------------------------------------

__global__ void k_init(Work wk, uint32_t n_chunks0, int direct_unit) {
    pdl_enter();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        Ctl *c = wk.ctl;
        uint32_t *words = reinterpret_cast<uint32_t *>(c);
        for (size_t i = 0; i < sizeof(Ctl) / 4; ++i) words[i] = 0;
        if (direct_unit) {
            Unit u;
            u.start = 0;
            u.len = static_cast<uint32_t>(wk.n);
            u.src = 0;
            u.raw = 1;
            u.vbits = 0;
            u.pad = 0;
            wk.units[0] = u;
            c->n_units = 1;
            c->finish_keys = wk.n;
        } else {
            Bucket b;
            b.start = 0;
            b.len = wk.n;
            b.first_chunk = 0;
            b.num_chunks = n_chunks0;
            b.h = wk.w;
            b.src = 0;
            b.raw = 1;
            b.scatter = 0;
            b.pad = 0;
            wk.buckets[0][0] = b;
            c->n_buckets[0] = 1;
            c->n_chunks[0] = n_chunks0;
        }
    }
    if (!direct_unit) {
        for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < n_chunks0; c += gridDim.x * blockDim.x) {
            Chunk ch;
            ch.start = static_cast<uint64_t>(c) * wk.chunk_keys;
            const uint64_t rem = wk.n - ch.start;
            ch.len = static_cast<uint32_t>(rem < wk.chunk_keys ? rem : wk.chunk_keys);
            ch.bucket = 0;
            wk.chunks[0][c] = ch;
        }
    }
}

// Clears the work lists and counters.
__global__ void k_zero_ctl(Work wk) {
    pdl_enter();
    uint32_t *words = reinterpret_cast<uint32_t *>(wk.ctl);
    for (size_t i = threadIdx.x; i < sizeof(Ctl) / 4; i += blockDim.x) words[i] = 0;
}

// Segmented sort: every segment [off[s], off[s+1]) of the keys buffer becomes
// an initial bucket (more than unit_cap keys) or finish unit (2..unit_cap
// keys); segments of 0 or 1 key are already sorted.  Offsets that decrease
// or pass n set the bounds error and the segment is skipped.
__global__ void k_seg_init(Work wk, const uint64_t *__restrict__ off, uint32_t nseg) {
    pdl_enter();
    const uint64_t vk = 128u / static_cast<uint32_t>(wk.w);
    for (uint32_t sg = blockIdx.x * blockDim.x + threadIdx.x; sg < nseg; sg += gridDim.x * blockDim.x) {
        const uint64_t a = off[sg], b = off[sg + 1];
        if (b < a || b > wk.n) {
            set_error(wk.ctl, kErrBounds);
            continue;
        }
        const uint64_t len = b - a;
        if (len <= 1) continue;
        if (len <= wk.unit_cap) {
            const uint32_t u = atomicAdd(&wk.ctl->n_units, 1u);
            if (u >= wk.max_units) {
                set_error(wk.ctl, kErrCapacity);
                continue;
            }
            atomicAdd(&wk.ctl->finish_keys, static_cast<unsigned long long>(len));
            Unit un;
            un.start = a;
            un.len = static_cast<uint32_t>(len);
            un.src = 0;
            un.raw = 1;
            un.vbits = 0;
            un.pad = 0;
            wk.units[u] = un;
            continue;
        }
        const uint64_t abase = a - a % vk;
        const uint32_t nch = static_cast<uint32_t>((b - abase + wk.chunk_keys - 1) / wk.chunk_keys);
        const uint32_t bi = atomicAdd(&wk.ctl->n_buckets[0], 1u);
        const uint32_t c0 = atomicAdd(&wk.ctl->n_chunks[0], nch);
        if (bi >= wk.max_buckets || c0 + nch > wk.max_chunks) {
            set_error(wk.ctl, kErrCapacity);
            continue;
        }
        Bucket bk;
        bk.start = a;
        bk.len = len;
        bk.first_chunk = c0;
        bk.num_chunks = nch;
        bk.h = wk.w;
        bk.src = 0;
        bk.raw = 1;
        bk.scatter = 0;
        bk.pad = 0;
        wk.buckets[0][bi] = bk;
        for (uint32_t i = 0; i < nch; ++i) {
            const uint64_t cs = i == 0 ? a : abase + static_cast<uint64_t>(i) * wk.chunk_keys;
            const uint64_t cl = abase + static_cast<uint64_t>(i + 1) * wk.chunk_keys;
            const uint64_t ce = cl < b ? cl : b;
            Chunk ch;
            ch.start = cs;
            ch.len = static_cast<uint32_t>(ce - cs);
            ch.bucket = bi;
            wk.chunks[0][c0 + i] = ch;
        }
    }
}

// Digit counts and AND/OR of the keys src[lo, hi) into the warp's
// shared-memory row `my`.  The 16-byte-aligned middle is read as vectors,
// U per thread in flight; a vector whose keys share one digit adds once.
template <typename K, int THREADS, bool RAW>
__device__ __forceinline__ void hist_range(const K *__restrict__ src, uint64_t lo, uint64_t hi, bool vec_ok,
                                           int shift, uint32_t mask, const Codec &codec, uint32_t *my, K &a, K &o) {
    constexpr int V = 16 / static_cast<int>(sizeof(K));
    constexpr int U = 4;
    auto one = [&](K key) {
        if (RAW) key = encode_key(key, codec);
        a &= key;
        o |= key;
        atomicAdd(&my[static_cast<uint32_t>(key >> shift) & mask], 1u);
    };
    if (!vec_ok) {  // buffer base not 16-byte aligned: scalar loads throughout
        for (uint64_t i = lo + threadIdx.x; i < hi; i += THREADS) one(src[i]);
        return;
    }
    uint64_t m0 = (lo + V - 1) / V * V;  // aligned middle [m0, m1)
    uint64_t m1 = hi / V * V;
    if (m0 > m1) m0 = m1 = hi;
    // head and tail, scalar
    for (uint64_t i = lo + threadIdx.x; i < m0; i += THREADS) one(src[i]);
    for (uint64_t i = m1 + threadIdx.x; i < hi; i += THREADS) one(src[i]);
    const uint4 *vec = reinterpret_cast<const uint4 *>(src + m0);
    const uint32_t nvec = static_cast<uint32_t>((m1 - m0) / V);
    uint32_t v = threadIdx.x;
    for (; v + (U - 1) * THREADS < nvec; v += U * THREADS) {
        uint4 q[U];
#pragma unroll
        for (int u = 0; u < U; ++u) q[u] = __ldcs(vec + v + u * THREADS);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            K kk[V];
            memcpy(kk, &q[u], 16);
            uint32_t d[V];
#pragma unroll
            for (int e = 0; e < V; ++e) {
                K key = kk[e];
                if (RAW) key = encode_key(key, codec);
                a &= key;
                o |= key;
                d[e] = static_cast<uint32_t>(key >> shift) & mask;
            }
            bool same = true;
#pragma unroll
            for (int e = 1; e < V; ++e) same &= d[e] == d[0];
            if (same) {
                atomicAdd(&my[d[0]], static_cast<uint32_t>(V));
            } else {
#pragma unroll
                for (int e = 0; e < V; ++e) atomicAdd(&my[d[e]], 1u);
            }
        }
    }
    for (; v < nvec; v += THREADS) {
        const uint4 q = __ldcs(vec + v);
        K kk[V];
        memcpy(kk, &q, 16);
#pragma unroll
        for (int e = 0; e < V; ++e) one(kk[e]);
    }
}

// Per-chunk digit histogram and AND/OR.  NB digit slots: with NB = kBins
// every warp counts into its own shared-memory row; with kWideBins (digits of
// 9..11 bits, where same-digit collisions inside a warp are rare) four rows
// are shared by the warps.  Rows 0 .. 2^radix_bits - 1 of the chunk's
// histogram column are written.
template <typename K, int THREADS, int NB>
__global__ void __launch_bounds__(THREADS) k_hist(Work wk, int level) {
    pdl_enter();
    constexpr int WARPS = THREADS / 32;
    constexpr int ROWS = NB <= kBins ? WARPS / 4 : 4;  // four warps per row
    __shared__ uint32_t sh[ROWS * NB];
    __shared__ K ta[WARPS], to[WARPS];
    const int p = level & 1;
    if (wk.ctl->error) return;  // an earlier launch found a problem: stop touching memory
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        wk.ctl->n_buckets[p ^ 1] = 0;
        wk.ctl->n_chunks[p ^ 1] = 0;
    }
    const int row = (threadIdx.x >> 5) % ROWS;
    const int nd = 1 << wk.radix_bits;  // <= NB
    const uint32_t nch = wk.ctl->n_chunks[p];
    for (uint32_t c = blockIdx.x; c < nch; c += gridDim.x) {
        const Chunk ch = wk.chunks[p][c];
        const Bucket b = wk.buckets[p][ch.bucket];
        const int r_eff = min(wk.radix_bits, b.h);
        const int shift = b.h - r_eff;
        const uint32_t mask = (1u << r_eff) - 1;
        for (int i = threadIdx.x; i < ROWS * NB; i += THREADS) sh[i] = 0;
        __syncthreads();
        K a = static_cast<K>(~K(0)), o = 0;
        const K *src = src_of<K>(wk, b.src);
        const bool vec_ok = b.src ? true : wk.keys_vec_ok;
        if (b.raw)
            hist_range<K, THREADS, true>(src, ch.start, ch.start + ch.len, vec_ok, shift, mask, wk.codec,
                                         sh + row * NB, a, o);
        else
            hist_range<K, THREADS, false>(src, ch.start, ch.start + ch.len, vec_ok, shift, mask, wk.codec,
                                          sh + row * NB, a, o);
        __syncthreads();
        for (int d = threadIdx.x; d < nd; d += THREADS) {
            uint32_t sum = 0;
#pragma unroll
            for (int w = 0; w < ROWS; ++w) sum += sh[w * NB + d];
            wk.hist[static_cast<size_t>(d) * wk.max_chunks + c] = sum;
        }
        block_and_or_k<K, THREADS>(a, o, ta, to);
        if (threadIdx.x == 0) store_and_or<K>(wk.chunk_and, wk.chunk_or, c, a, o);
        __syncthreads();
    }
}

// Per digit d: exclusive prefix of hist[d][c] over the chunks of each bucket
// (in place), and the bucket's digit total into bucket_base[bucket][d].
template <int THREADS>
__global__ void __launch_bounds__(THREADS) k_colscan(Work wk, int level) {
    pdl_enter();
    __shared__ uint32_t tmp[THREADS / 32 + 1];
    __shared__ int itmp[THREADS / 32 + 1];
    __shared__ unsigned long long sm_excl[THREADS];
    __shared__ unsigned long long sh_last;
    const int d = blockIdx.x;
    const int p = level & 1;
    if (wk.ctl->error) return;
    const uint32_t nch = wk.ctl->n_chunks[p];
    const Chunk *chunks = wk.chunks[p];
    uint32_t *col = wk.hist + static_cast<size_t>(d) * wk.max_chunks;
    unsigned long long carry_total = 0;  // unsegmented prefix before this block
    unsigned long long carry_seg = 0;    // unsegmented prefix at the latest segment head
    // this step's chunk data was loaded during the previous step's scans
    auto fetch = [&](uint32_t c, uint32_t &b, uint32_t &v, uint32_t &bp, uint32_t &bn) {
        const bool in = c < nch;
        b = in ? chunks[c].bucket : 0xffffffffu;
        v = in ? col[c] : 0;
        bp = in && c > 0 ? chunks[c - 1].bucket : 0xfffffffeu;
        bn = in && c + 1 < nch ? chunks[c + 1].bucket : 0xfffffffeu;
    };
    uint32_t nb_, nv_, nbp_, nbn_;
    fetch(threadIdx.x, nb_, nv_, nbp_, nbn_);
    for (uint32_t base = 0; base < nch; base += THREADS) {
        const uint32_t c = base + threadIdx.x;
        const bool in = c < nch;
        const uint32_t b = nb_, v = nv_, bprev = nbp_, bnext = nbn_;
        if (base + THREADS < nch) fetch(c + THREADS, nb_, nv_, nbp_, nbn_);
        const bool head = in && (c == 0 || bprev != b);
        const bool last = in && (c + 1 == nch || bnext != b);
        uint32_t block_total;
        const uint32_t ex = block_exclusive_scan<THREADS>(v, tmp, block_total);
        const unsigned long long ex_global = carry_total + ex;
        sm_excl[threadIdx.x] = ex_global;
        // latest segment head at or before this element inside the block
        // (the max-scan's barriers also publish sm_excl)
        const int hp = block_inclusive_max<THREADS>(head ? static_cast<int>(threadIdx.x) : -1, itmp);
        const unsigned long long seg0 = hp >= 0 ? sm_excl[hp] : carry_seg;
        if (in) {
            const uint32_t out = static_cast<uint32_t>(ex_global - seg0);
            col[c] = out;
            if (last) wk.bucket_base[static_cast<size_t>(b) * wk.bins + d] = out + v;
        }
        if (threadIdx.x == THREADS - 1) sh_last = seg0;
        __syncthreads();
        carry_seg = sh_last;
        carry_total += block_total;
        __syncthreads();
    }
}

// Block-cooperative emission of the next-level buckets of one parent.
// Each thread owns digit d = threadIdx.x (THREADS == kBins); `take` marks the
// children that become buckets, with their start/len/h/src in the arguments.
template <int THREADS>
__device__ void emit_buckets(const Work &wk, int q, bool take, uint64_t start, uint64_t len, int h, int src, int raw,
                             uint32_t *tmp, uint32_t *sh_bases) {
    // chunk boundaries sit on 16-byte boundaries of the buffer except the
    // bucket's own start, so every tile after the first is an aligned window
    const uint64_t vk = 128u / static_cast<uint32_t>(wk.w);
    const uint64_t abase = start - start % vk;
    const uint32_t nchunks =
        take ? static_cast<uint32_t>((start + len - abase + wk.chunk_keys - 1) / wk.chunk_keys) : 0;
    uint32_t nb_total, nc_total;
    const uint32_t slot_off = block_exclusive_scan<THREADS>(take ? 1u : 0u, tmp, nb_total);
    const uint32_t ch_off = block_exclusive_scan<THREADS>(nchunks, tmp, nc_total);
    if (nb_total == 0) return;  // block-uniform
    if (threadIdx.x == 0) {
        const uint32_t b0 = atomicAdd(&wk.ctl->n_buckets[q], nb_total);
        const uint32_t c0 = atomicAdd(&wk.ctl->n_chunks[q], nc_total);
        const bool ok = b0 + nb_total <= wk.max_buckets && c0 + nc_total <= wk.max_chunks;
        if (!ok) set_error(wk.ctl, kErrCapacity);
        sh_bases[0] = ok ? b0 : 0xffffffffu;
        sh_bases[1] = c0;
    }
    __syncthreads();
    const uint32_t b0 = sh_bases[0], c0 = sh_bases[1];
    if (b0 != 0xffffffffu) {
        if (take) {
            Bucket nb;
            nb.start = start;
            nb.len = len;
            nb.first_chunk = c0 + ch_off;
            nb.num_chunks = nchunks;
            nb.h = h;
            nb.src = static_cast<uint8_t>(src);
            nb.raw = static_cast<uint8_t>(raw);
            nb.scatter = 0;
            nb.pad = 0;
            wk.buckets[q][b0 + slot_off] = nb;
        }
        __syncthreads();
        // the children's chunk records are written by the next kernel's grid
        // (write_child_chunks), not by this one CTA
    }
    __syncthreads();
}

// Fill pieces for every thread whose `take` is set (thread-private loop).
template <typename K>
__device__ void emit_fill(const Work &wk, uint64_t start, uint64_t len, K value, int src) {
    const uint32_t pieces = static_cast<uint32_t>((len + kFillPiece - 1) / kFillPiece);
    const uint32_t f0 = atomicAdd(&wk.ctl->n_fills, pieces);
    if (f0 + pieces > wk.max_fills) {
        set_error(wk.ctl, kErrCapacity);
        return;
    }
    atomicAdd(&wk.ctl->fill_keys, static_cast<unsigned long long>(len));
    for (uint32_t i = 0; i < pieces; ++i) {
        Fill f;
        f.start = start + static_cast<uint64_t>(i) * kFillPiece;
        const uint64_t rem = len - static_cast<uint64_t>(i) * kFillPiece;
        f.len = static_cast<uint32_t>(rem < kFillPiece ? rem : kFillPiece);
        f.value = static_cast<uint64_t>(value);
        if constexpr (sizeof(K) > 8) f.value_hi = static_cast<uint64_t>(value >> 64);
        else f.value_hi = 0;
        f.src = static_cast<uint32_t>(src);
        wk.fills[f0 + i] = f;
    }
}

// Per bucket of this level: common-prefix test, digit bases, child classes.
// Thread t takes digit page * THREADS + t; digits wider than 8 bits take
// several pages, with the running digit base carried between them (a run of
// merged small children ends at a page boundary).
template <int THREADS, typename K>
__global__ void __launch_bounds__(THREADS) k_classify(Work wk, int level) {
    pdl_enter();
    static_assert(THREADS == kBins, "one thread per digit of a page");
    __shared__ K ta[THREADS / 32], to[THREADS / 32];
    __shared__ unsigned long long tmp64[THREADS / 32 + 1];
    __shared__ uint32_t tmp[THREADS / 32 + 1];
    __shared__ uint32_t sh_bases[2];
    __shared__ int itmp[THREADS / 32 + 1], sh_i2[THREADS];
    __shared__ uint32_t sh_u[THREADS], sh_u2[THREADS];
    const int p = level & 1, q = p ^ 1;
    if (wk.ctl->error) return;
    const uint32_t nb = wk.ctl->n_buckets[p];
    const int t = threadIdx.x;
    for (uint32_t i = blockIdx.x; i < nb; i += gridDim.x) {
        const Bucket b = wk.buckets[p][i];
        K a = static_cast<K>(~K(0)), o = 0;
        {
            // eight chunks per thread in flight at once (a big bucket has thousands)
            const uint32_t c_end = b.first_chunk + b.num_chunks;
            uint32_t c = b.first_chunk + threadIdx.x;
            for (; c + 7 * THREADS < c_end; c += 8 * THREADS) {
                K ra[8], ro[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    ra[u] = load_word_k<K>(wk.chunk_and, c + u * THREADS);
                    ro[u] = load_word_k<K>(wk.chunk_or, c + u * THREADS);
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    a &= ra[u];
                    o |= ro[u];
                }
            }
            for (; c < c_end; c += THREADS) {
                a &= load_word_k<K>(wk.chunk_and, c);
                o |= load_word_k<K>(wk.chunk_or, c);
            }
        }
        block_and_or_k<K, THREADS>(a, o, ta, to);
        if (threadIdx.x == 0) atomicAdd(&wk.ctl->hist_keys[level], static_cast<unsigned long long>(b.len));
        if (a == o) {  // every key identical: write the value, no sort needed
            if (threadIdx.x == 0) {
                wk.buckets[p][i].scatter = 0;
                emit_fill<K>(wk, b.start, b.len, a, b.raw ? 2 : b.src);
            }
            continue;
        }
        const int r_eff = min(wk.radix_bits, b.h);
        const int shift = b.h - r_eff;
        const uint32_t mask = (1u << r_eff) - 1;
        const int hb = msb_pos<K>(a ^ o);
        if (hb < shift) {
            // the digit is constant: re-open the bucket at its highest varying bit
            if (threadIdx.x == 0) wk.buckets[p][i].scatter = 0;
            emit_buckets<THREADS>(wk, q, threadIdx.x == 0, b.start, b.len, hb + 1, b.src, b.raw, tmp, sh_bases);
            continue;
        }
        if (threadIdx.x == 0) {
            wk.buckets[p][i].scatter = 1;
            atomicAdd(&wk.ctl->scatter_keys[level], static_cast<unsigned long long>(b.len));
        }
        const int hc = shift;  // bits left in the children
        const int dst = wk.inplace ? 0 : b.src ^ 1;
        const int pages = static_cast<int>((mask + THREADS) / THREADS);
        unsigned long long carry = 0;  // keys of the digits of earlier pages
        for (int pg = 0; pg < pages; ++pg) {
            const uint32_t d = static_cast<uint32_t>(pg * THREADS + t);
            const bool in = d <= mask;
            uint32_t *bbase = wk.bucket_base + static_cast<size_t>(i) * wk.bins + d;
            const unsigned long long tot = in ? *bbase : 0ull;
            unsigned long long total;
            const unsigned long long ex = carry + block_exclusive_scan64<THREADS>(tot, tmp64, total);
            const unsigned long long base = b.start + ex;
            if (in) *bbase = static_cast<uint32_t>(ex);
            carry += total;
            const bool big = tot > wk.unit_cap;
            // children with no bits left are constant: value = common prefix | digit
            if (big && hc == 0) {
                emit_fill<K>(wk, base, tot, static_cast<K>(high_bits<K>(a, b.h) | static_cast<K>(d)), dst);
            }
            emit_buckets<THREADS>(wk, q, big && hc > 0, base, tot, hc, dst, 0, tmp, sh_bases);
            // Small children become finish units.  Children of at most
            // merge_cap / 4 keys ("tiny") merge with their tiny neighbours:
            // inside a run of adjacent tiny children (empty children do not
            // break a run), child e joins group floor(P_e / merge_cap) of the
            // run, P_e being the keys of the run before it, so a group holds
            // < 1.25 * merge_cap keys.
            const uint32_t len = static_cast<uint32_t>(tot);
            const bool small = tot > 0 && tot <= wk.unit_cap;
            const bool tiny = small && len <= wk.merge_cap / 4;
            const bool solid = tot > 0 && !tiny;  // breaks runs
            // latest solid child before e, latest tiny child before e
            const int last_solid = block_inclusive_max<THREADS>(solid ? t : -1, itmp);
            const int last_tiny_incl = block_inclusive_max<THREADS>(tiny ? t : -1, itmp);
            sh_i2[t] = last_tiny_incl;
            __syncthreads();
            const int prev_tiny = t > 0 ? sh_i2[t - 1] : -1;
            const bool run_start = tiny && (prev_tiny < 0 || prev_tiny < last_solid);
            uint32_t dummy;
            const uint32_t g_ex = block_exclusive_scan<THREADS>(tiny ? len : 0u, tmp, dummy);
            sh_u[t] = g_ex;
            const int rs_idx = block_inclusive_max<THREADS>(run_start ? t : -1, itmp);
            // (barriers inside the scans publish sh_u)
            const uint32_t pre = tiny ? g_ex - sh_u[rs_idx] : 0u;
            const uint32_t gid = pre / wk.merge_cap;
            sh_u2[t] = gid;
            __syncthreads();
            const bool head = tiny && (run_start || sh_u2[prev_tiny] != gid);
            const int head_idx = block_inclusive_max<THREADS>(head ? t : -1, itmp);
            sh_u[t] = 0;
            __syncthreads();
            if (tiny) atomicAdd(&sh_u[head_idx], len);
            __syncthreads();
            const bool emit = (small && !tiny) || head;
            const uint32_t ulen = head ? sh_u[t] : len;
            uint32_t n_emit;
            const uint32_t slot = block_exclusive_scan<THREADS>(emit ? 1u : 0u, tmp, n_emit);
            uint32_t keys_total;
            (void)block_exclusive_scan<THREADS>(emit ? ulen : 0u, tmp, keys_total);
            if (threadIdx.x == 0 && n_emit) {
                const uint32_t u0 = atomicAdd(&wk.ctl->n_units, n_emit);
                sh_bases[0] = u0;
                if (u0 + n_emit > wk.max_units) set_error(wk.ctl, kErrCapacity);
                atomicAdd(&wk.ctl->finish_keys, static_cast<unsigned long long>(keys_total));
            }
            __syncthreads();
            if (emit && n_emit && sh_bases[0] + n_emit <= wk.max_units) {
                Unit un;
                un.start = base;
                un.len = ulen;
                un.src = static_cast<uint8_t>(dst);
                un.raw = 0;
                // one child agrees above the digit; a merged group above the parent's bits.
                // The fast counting finish that this enables needs sparse
                // sub-buckets (under 16 keys per 16 values): a child averaging
                // more than one key per 4 values, or a merged group whose
                // children may (up to merge_cap / 4 keys each), goes to the
                // general path without trying it
                const uint32_t most = head ? wk.merge_cap / 4 : ulen;
                const bool dense = hc < 18 && most > (1u << (hc >= 2 ? hc - 2 : 0));
                un.vbits = dense ? 0 : static_cast<uint8_t>(head ? b.h : hc);
                un.pad = 0;
                wk.units[sh_bases[0] + slot] = un;
            }
            __syncthreads();
        }
    }
}

// Unstable rank of a tile by a digit of up to SPLIT_BITS bits (one CTA-wide
// counter row of 2^SPLIT_BITS words, padded by one word per 16 so that the
// thread scanning 16 consecutive counters hits 16 different banks), then
// placement in digit order.  Afterwards cnt[pad(d)] is the start of digit d
// in `out` and cnt[pad(2^bits)] the number of keys.
__device__ __forceinline__ int split_pad(int d) { return d + (d >> 4); }

template <typename K, int THREADS, int ITEMS>
__device__ void split_rank(const K (&keys)[ITEMS], uint32_t vmask, int shift, int bits, uint32_t *cnt,
                           uint32_t *scan_tmp, K *out) {
    const int lane = threadIdx.x & 31;
    const int nb = 1 << bits;                       // <= kSplitCap
    const int e_per = nb > THREADS ? nb / THREADS : 1;  // counters per scanning thread (1..16)
    const int owners = nb / e_per;
    const uint32_t mask = static_cast<uint32_t>(nb - 1);
    for (int i = threadIdx.x; i <= split_pad(nb); i += THREADS) cnt[i] = 0;
    __syncthreads();
    uint32_t local[(ITEMS + 1) / 2];
#pragma unroll
    for (int j = 0; j < (ITEMS + 1) / 2; ++j) local[j] = 0;
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const bool valid = (vmask >> j) & 1u;
        const int d = static_cast<int>(static_cast<uint32_t>(keys[j] >> shift) & mask);
        const uint32_t r = valid ? atomicAdd(&cnt[split_pad(d)], 1u) : 0u;
        local[j >> 1] |= r << ((j & 1) * 16);
    }
    __syncthreads();
    const int g0 = split_pad(threadIdx.x * e_per);  // this thread's counters are contiguous after padding
    uint32_t sum = 0;
    if (threadIdx.x < owners)
        for (int e = 0; e < e_per; ++e) sum += cnt[g0 + e];
    uint32_t total;
    uint32_t run = block_exclusive_scan<THREADS>(sum, scan_tmp, total);
    if (threadIdx.x < owners) {
        for (int e = 0; e < e_per; ++e) {
            const uint32_t c = cnt[g0 + e];
            cnt[g0 + e] = run;
            run += c;
        }
    }
    if (threadIdx.x == 0) cnt[split_pad(nb)] = total;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        if ((vmask >> j) & 1u) {
            const int d = static_cast<int>(static_cast<uint32_t>(keys[j] >> shift) & mask);
            out[cnt[split_pad(d)] + ((local[j >> 1] >> ((j & 1) * 16)) & 0xffffu)] = keys[j];
        }
    }
    __syncthreads();
    (void)lane;
}

// Staging of one tile's keys: each key takes the next slot of its digit from
// the cursor row (shared-memory atomicAdd).  FULL: every item is valid.
// SKEW: a warp whose 32 keys share one digit takes its 32 slots with one
// atomic (sorted and skewed inputs, where same-address atomics serialise).
template <typename K, int ITEMS, bool FULL, bool SKEW>
__device__ __forceinline__ void stage_keys(const K (&k)[ITEMS], uint32_t vmask, int shift, uint32_t mask,
                                           uint32_t *cur, K *sm_keys, int cap, bool &overflow) {
    const int lane = threadIdx.x & 31;
    if (SKEW && FULL) {
        // the warp's whole tile in one digit (presorted or heavily skewed
        // input): one atomic for its 32 * ITEMS keys -- same-address atomics
        // of every warp and item would serialise
        const uint32_t d0 = __shfl_sync(kFull, static_cast<uint32_t>(k[0] >> shift) & mask, 0);
        bool same = true;
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) same &= (static_cast<uint32_t>(k[j] >> shift) & mask) == d0;
        if (__all_sync(kFull, same)) {
            uint32_t base = 0;
            if (lane == 0) base = atomicAdd(&cur[d0], 32u * ITEMS);
            base = __shfl_sync(kFull, base, 0);
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) {
                const uint32_t slot = base + static_cast<uint32_t>(j * 32 + lane);
                overflow |= slot >= static_cast<uint32_t>(cap);
                sm_keys[min(slot, static_cast<uint32_t>(cap - 1))] = k[j];
            }
            return;
        }
    }
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const bool valid = FULL || ((vmask >> j) & 1u);
        const uint32_t dg = static_cast<uint32_t>(k[j] >> shift) & mask;
        uint32_t slot = 0;
        if (SKEW) {
            const uint32_t d0 = __shfl_sync(kFull, dg, 0);
            if (__all_sync(kFull, valid && dg == d0)) {
                uint32_t base = 0;
                if (lane == 0) base = atomicAdd(&cur[d0], 32u);
                slot = __shfl_sync(kFull, base, 0) + lane;
            } else if (valid) {
                slot = atomicAdd(&cur[dg], 1u);
            }
        } else if (valid) {
            slot = atomicAdd(&cur[dg], 1u);
        }
        if (valid) {
            overflow |= slot >= static_cast<uint32_t>(cap);
            sm_keys[min(slot, static_cast<uint32_t>(cap - 1))] = k[j];
        }
    }
}

// Per chunk: the chunk's digit counts are known from the histogram pass
// (difference of consecutive per-chunk exclusive offsets), so each key takes
// its slot in the chunk's shared-memory staging area with one atomicAdd on
// its digit's cursor (unstable: equal digits need no order in an MSD pass),
// and the staged digit runs are then written to their bucket offsets, one
// warp per run.  The whole chunk (CHUNK_TILES tiles) is staged before the
// write-out, so runs are long and coalesced.  Every run's destination is
// checked against the bucket before anything is written.
//
// NB digit slots (kBins, or kWideBins for digits of 9..11 bits): with NB >
// THREADS each thread owns NB / THREADS consecutive digits in the per-chunk
// bookkeeping.
template <typename K, int THREADS, int ITEMS, int CHUNK_TILES, int NB>
__host__ __device__ constexpr size_t scatter_pre_offset() {
    return (sizeof(K) * THREADS * ITEMS * CHUNK_TILES + sizeof(unsigned long long) * NB +
            sizeof(uint32_t) * (NB + THREADS / 32 + 1) + 16 + 15) &
           ~size_t(15);
}

template <typename K, int THREADS, int ITEMS, int CHUNK_TILES, int NB>
__global__ void __launch_bounds__(THREADS, 2) k_scatter(Work wk, int level) {
    pdl_enter();
    using L = TileLoad<K, THREADS, ITEMS>;
    using Pre = ScatterPre<NB>;
    constexpr int TILE = THREADS * ITEMS;
    constexpr int CAP = TILE * CHUNK_TILES;
    constexpr int V = L::V;
    constexpr int WARPS = THREADS / 32;
    constexpr int DPT = NB > THREADS ? NB / THREADS : 1;  // digits per thread
    static_assert(NB <= THREADS || NB % THREADS == 0, "whole digits per thread");
    K *sm_keys = reinterpret_cast<K *>(g_dyn_smem);
    unsigned long long *off = reinterpret_cast<unsigned long long *>(g_dyn_smem + sizeof(K) * CAP);
    uint32_t *cur = reinterpret_cast<uint32_t *>(off + NB);  // [NB] staging cursors
    uint32_t *tmp = cur + NB;                                // [WARPS + 1]
    int *bad = reinterpret_cast<int *>(tmp + WARPS + 1);
    constexpr size_t kPreOff = scatter_pre_offset<K, THREADS, ITEMS, CHUNK_TILES, NB>();
    Pre *pre = reinterpret_cast<Pre *>(g_dyn_smem + kPreOff);
    const int p = level & 1;
    const int t = threadIdx.x;
    if (wk.ctl->error) return;
    write_child_chunks(wk, p ^ 1);  // records of the buckets this level's classify opened
    if (t == 0) *bad = 0;  // stays 0 unless a check fails (then the CTA stops)
    const uint32_t nch = wk.ctl->n_chunks[p];
    // Chunk metadata arrives by cp.async two chunks ahead in a ring of three
    // slots: stage 1 (needs only the chunk index) fetches the chunk records
    // and the chunk's prefix counts; stage 2 (needs the chunk's bucket) the
    // bucket and its digit bases.
    // (digits >= 2^radix_bits are never read: their rows are not fetched)
    const int nd = 1 << wk.radix_bits;
    auto stage1 = [&](uint32_t c, int slot) {
        Pre &P = pre[slot];
        if (t == 0) {
            cp_async16(&P.ch, &wk.chunks[p][c]);
            if (c + 1 < nch) cp_async16(&P.chn, &wk.chunks[p][c + 1]);
            else P.chn.bucket = 0xffffffffu;
        }
        for (int d = t; d < nd; d += THREADS) {
            cp_async4(&P.hc[d], &wk.hist[static_cast<size_t>(d) * wk.max_chunks + c]);
            if (c + 1 < nch) cp_async4(&P.hn[d], &wk.hist[static_cast<size_t>(d) * wk.max_chunks + c + 1]);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    auto stage2 = [&](int slot) {
        Pre &P = pre[slot];
        const uint32_t bk = P.ch.bucket;
        if (t == 0) {
            cp_async16(&P.b, &wk.buckets[p][bk]);
            cp_async16(reinterpret_cast<char *>(&P.b) + 16, reinterpret_cast<const char *>(&wk.buckets[p][bk]) + 16);
        }
        for (int d = t; d < nd; d += THREADS)
            cp_async4(&P.bb[d], &wk.bucket_base[static_cast<size_t>(bk) * wk.bins + d]);
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    if (blockIdx.x < nch) {
        stage1(blockIdx.x, 0);
        cp_async_wait_all();
        __syncthreads();
        stage2(0);
        if (blockIdx.x + gridDim.x < nch) stage1(blockIdx.x + gridDim.x, 1);
    }
    int it = 0;
    for (uint32_t c = blockIdx.x; c < nch; c += gridDim.x, ++it) {
        cp_async_wait_all();
        __syncthreads();
        {
            const uint32_t c1 = c + gridDim.x, c2 = c1 + gridDim.x;
            if (c1 < nch) stage2((it + 1) % 3);
            if (c2 < nch) stage1(c2, (it + 2) % 3);
        }
        const Pre &P = pre[it % 3];
        const Chunk ch = P.ch;
        const Bucket b = P.b;
        if (!b.scatter) continue;  // block-uniform
        const K *__restrict__ src = src_of<K>(wk, b.src);
        K *__restrict__ dst = dst_of<K>(wk, b.src);
        const bool vec_ok = b.src ? true : wk.keys_vec_ok;
        const int r_eff = min(wk.radix_bits, b.h);
        const int shift = b.h - r_eff;
        const uint32_t mask = (1u << r_eff) - 1;
        const bool next_same = P.chn.bucket == ch.bucket;
        // chunk digit counts and destinations (thread t: digits t * DPT ..)
        uint32_t n_d[DPT];
        uint32_t n_sum = 0, n_max = 0;
#pragma unroll
        for (int e = 0; e < DPT; ++e) {
            const int d = threadIdx.x * DPT + e;
            n_d[e] = 0;
            if (d < NB && static_cast<uint32_t>(d) <= mask) {
                const uint32_t ex = P.hc[d];
                uint32_t ex_next;
                if (next_same) {
                    ex_next = P.hn[d];
                } else {  // last chunk of the bucket: the digit's bucket total
                    const uint32_t base_n =
                        static_cast<uint32_t>(d) < mask ? P.bb[d + 1] : static_cast<uint32_t>(b.len);
                    ex_next = base_n - P.bb[d];
                }
                n_d[e] = ex_next - ex;
                const unsigned long long o = b.start + P.bb[d] + ex;
                off[d] = o;
                if (n_d[e] && o + n_d[e] > b.start + b.len) *bad = 1;  // never write outside the bucket
            }
            n_sum += n_d[e];
            n_max = max(n_max, n_d[e]);
        }
        __syncthreads();
        uint32_t total;
        uint32_t st = block_exclusive_scan<THREADS>(n_sum, tmp, total);
#pragma unroll
        for (int e = 0; e < DPT; ++e) {
            const int d = threadIdx.x * DPT + e;
            if (d < NB) {
                cur[d] = st;
                off[d] -= st;  // the key at staging slot q of digit d goes to off[d] + q (mod 2^64)
                st += n_d[e];
            }
        }
        if (total != ch.len && threadIdx.x == 0) *bad = 1;
        __syncthreads();
        if (*bad) {
            if (threadIdx.x == 0) set_error(wk.ctl, kErrBounds);
            cp_async_wait_all();  // no copy may land after the CTA is gone
            return;               // block-uniform
        }
        // stage: every key takes the next slot of its digit.  The loop body
        // is specialised per tile (block-uniform): keys still raw or already
        // encoded, a whole aligned tile or a partial one, and -- from the
        // chunk's known counts -- whether warps often share one digit.
        const uint64_t cend = ch.start + ch.len;
        const bool skew = block_reduce_max<THREADS>(n_max, tmp) * 8u > ch.len;
        bool overflow = false;
        for (uint64_t pos = ch.start; pos < cend;) {
            const uint64_t wstart = pos - pos % V;
            const uint64_t thi = min(cend, wstart + TILE);
            K k[ITEMS];
            const bool full = vec_ok && wstart == pos && thi - pos == static_cast<uint64_t>(TILE);
            uint32_t vmask;
            if (full) {
                L::load_full(src + wstart, k);
                vmask = (ITEMS == 32) ? 0xffffffffu : ((1u << ITEMS) - 1);
            } else {
                vmask = L::load(src, wstart, static_cast<uint32_t>(pos - wstart), static_cast<uint32_t>(thi - wstart),
                                vec_ok, k);
            }
            if (b.raw) {
#pragma unroll
                for (int j = 0; j < ITEMS; ++j) k[j] = encode_key(k[j], wk.codec);
            }
            if (full && !skew)
                stage_keys<K, ITEMS, true, false>(k, vmask, shift, mask, cur, sm_keys, CAP, overflow);
            else if (full)
                stage_keys<K, ITEMS, true, true>(k, vmask, shift, mask, cur, sm_keys, CAP, overflow);
            else
                stage_keys<K, ITEMS, false, true>(k, vmask, shift, mask, cur, sm_keys, CAP, overflow);
            pos = thi;
        }
        if (__syncthreads_or(overflow)) {
            if (threadIdx.x == 0) set_error(wk.ctl, kErrBounds);
            cp_async_wait_all();
            return;
        }
        // write-out in staging order: the key at staging slot q belongs to
        // digit d's run, so it goes to off[d] + q (off[d] holds the run's
        // destination minus its staging start); consecutive slots are
        // consecutive addresses inside a run
        for (uint32_t q = threadIdx.x; q < ch.len; q += THREADS) {
            const K key = sm_keys[q];
            const uint32_t dg = static_cast<uint32_t>(key >> shift) & mask;
            dst[off[dg] + q] = key;
        }
        __syncthreads();
    }
}

template <typename K, int THREADS, int ITEMS, int CHUNK_TILES, int NB>
constexpr size_t scatter_smem() {
    return scatter_pre_offset<K, THREADS, ITEMS, CHUNK_TILES, NB>() + 3 * sizeof(ScatterPre<NB>);
}

// Shared-memory layout of k_finish.  Three alternatives share the first region:
//   counting path: words[sb] (u64: sixteen 4-bit counters, one per value of
//                  the unit's low 4 varying bits, in sub-bucket sb of the bits
//                  above), totals[sb] and starts[sb] (u16), and the output
//                  staging buffer over the words once positions are known;
//   fast counting path (keys known to agree above bit 16): the same words,
//                  then fstarts[sb] (u16) over the totals and the output
//                  staging of the keys' low 16 bits, stage16[TILE + V], from
//                  the starts on;
//   compare path:  keys[TILE] then the split counters cnt[split_pad(d)].
// The per-warp AND/OR slots and the scan scratch follow the shared region.
template <typename K, int THREADS, int ITEMS>
struct FinLayout {
    static constexpr int WARPS = THREADS / 32;
    static constexpr int V = 16 / static_cast<int>(sizeof(K));
    static constexpr size_t kTile = static_cast<size_t>(THREADS) * ITEMS;
    static constexpr size_t kPadded = kSplitCap + kSplitCap / 16 + 4;
    static constexpr size_t kWords = 0;                           // u64[kSplitCap]
    static constexpr size_t kTotals = kWords + 8 * kSplitCap;     // u16[kSplitCap]
    static constexpr size_t kStarts = kTotals + 2 * kSplitCap;    // u16[kSplitCap]
    static constexpr size_t kNibEnd = kStarts + 2 * kSplitCap;
    static constexpr size_t kFStarts = kTotals;                   // u16[kSplitCap]
    static constexpr size_t kStage16 = kStarts;                   // u16[kTile + V]
    static constexpr size_t kFastEnd = kStage16 + 2 * (kTile + V);
    static constexpr size_t kStage = kWords;                      // K[kTile + V]
    static constexpr size_t kCnt = sizeof(K) * kTile;
    static constexpr size_t kCmpEnd = kCnt + 4 * kPadded;
    static constexpr size_t kShared0 = kNibEnd > kCmpEnd ? kNibEnd : kCmpEnd;
    static constexpr size_t kShared = ((kShared0 > kFastEnd ? kShared0 : kFastEnd) + 15) & ~size_t(15);
    static constexpr size_t kTa = kShared;
    static constexpr size_t kTo = kTa + sizeof(K) * WARPS;
    static constexpr size_t kScan = kTo + sizeof(K) * WARPS;
    static constexpr size_t kNext = (kScan + 4 * (WARPS + 1) + 15) & ~size_t(15);  // Unit[2]
    static constexpr size_t kEnd = kNext + 2 * sizeof(Unit);
    static_assert(sizeof(K) * (kTile + V) <= kTotals, "staging overlaps only the counter words");
    static_assert(kSplitCap == 16 * THREADS, "the scan gives each thread 16 sub-buckets");
};

// Counting finish of a unit whose keys agree on every bit at or above vb
// (8 <= vb <= 16, 16-byte aligned buffers): the keys' low vb bits f are the
// whole sort key.  Keys arrive as 16-byte vectors; one shared atomic per key
// on a 4-bit counter of (sub-bucket f >> 4, low value f & 15) gives its
// arrival rank; multiplying a sub-bucket's counter word by 0x1111... leaves
// in nibble i the count of the values below i and in the top nibble the
// sub-bucket's total (exact while the total is under 16, which the sum of the
// totals confirms: a larger total always reads smaller); the totals' scan and
// those nibbles place every key.  The low bits are staged as u16 and the
// output rebuilt from the unit's common upper bits, decoded by one xor (the
// key's top bit lies in the common part).  Expects the counter words zero and
// leaves them zero.  Returns false with nothing written when a counter would
// overflow or a sub-bucket holds 16 keys or more (counter words then dirty).
template <typename K, int THREADS, int ITEMS>
__device__ __forceinline__ bool finish_count_fast(const Work &wk, const Unit &un, int vb) {
    using FL = FinLayout<K, THREADS, ITEMS>;
    constexpr int V = FL::V;
    constexpr int NV = ITEMS / V;  // 16-byte vectors per thread
    static_assert(ITEMS % V == 0, "whole vectors per thread");
    static_assert(kSplitCap == 16 * THREADS, "one thread scans 16 sub-buckets");
    uint32_t *w32 = reinterpret_cast<uint32_t *>(g_dyn_smem + FL::kWords);
    uint16_t *fst = reinterpret_cast<uint16_t *>(g_dyn_smem + FL::kFStarts);
    uint16_t *stage = reinterpret_cast<uint16_t *>(g_dyn_smem + FL::kStage16);
    uint32_t *scan_tmp = reinterpret_cast<uint32_t *>(g_dyn_smem + FL::kScan);
    const int t = threadIdx.x;
    const K *__restrict__ src = src_of<K>(wk, un.src);
    const int len = static_cast<int>(un.len);
    const uint64_t wstart = un.start - un.start % V;
    const int lo_r = static_cast<int>(un.start - wstart);
    const int hi_r = lo_r + len;
    const int nvec = (hi_r + V - 1) / V;
    const int rows = (nvec + THREADS - 1) / THREADS;  // vector rows in use (block-uniform, <= NV)
    const uint32_t fmask = (1u << vb) - 1u;
    const K common = src[un.start] & ~static_cast<K>(fmask);  // encoded bits shared by the unit
    // every load first (nothing between them, so all are in flight at once),
    // then the counting atomics; fr[i] = f | rank << 16 | valid << 20.  Rows
    // past the unit's last vector are skipped by block-uniform branches.
    uint32_t fr[ITEMS];
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) fr[i] = 0;
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        if (j < rows) {
            const int q = j * THREADS + t;
            K kk[V];
            uint32_t ok = 0;
#pragma unroll
            for (int e = 0; e < V; ++e) kk[e] = 0;
            if (q < nvec) {
                const int r0 = q * V;
                if (r0 >= lo_r && r0 + V <= hi_r) {
                    const uint4 v = *reinterpret_cast<const uint4 *>(src + wstart + r0);
                    memcpy(kk, &v, 16);
                    ok = (1u << V) - 1u;
                } else {
#pragma unroll
                    for (int e = 0; e < V; ++e) {
                        const bool in = r0 + e >= lo_r && r0 + e < hi_r;
                        if (in) kk[e] = src[wstart + r0 + e];
                        ok |= static_cast<uint32_t>(in) << e;
                    }
                }
            }
#pragma unroll
            for (int e = 0; e < V; ++e)
                fr[j * V + e] = (static_cast<uint32_t>(kk[e]) & fmask) | (((ok >> e) & 1u) << 20);
        }
    }
    uint32_t ovf = 0;
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        if (j < rows) {
#pragma unroll
            for (int e = 0; e < V; ++e) {
                const uint32_t v = fr[j * V + e];
                if (v >> 20) {
                    const uint32_t f = v & 0xffffu;
                    const int sh = static_cast<int>(f & 7u) << 2;
                    const uint32_t old = atomicAdd(&w32[f >> 3], 1u << sh);
                    const uint32_t r = (old >> sh) & 15u;
                    ovf |= r + 1u;  // bit 4 set iff r == 15
                    fr[j * V + e] = v | (r << 16);
                }
            }
        }
    }
    if (__syncthreads_or(ovf & 16u)) return false;
    // counter words to exclusive prefix nibbles in place, 32-bit halves: the
    // low half (values 0-7) times 0x11111111 holds in nibble i the keys of
    // values <= i and in its top nibble the half's total s; the high half
    // times 0x11111111 plus s times 0x11111111 continues the count, its top
    // nibble the sub-bucket's total (exact while under 16; a larger total
    // always reads smaller, so the sum over the unit exposes it).  Thread t
    // owns sub-buckets [16t, 16t + 16), visited from pair (e + t) % 8 on so
    // that the eight threads of one shared-memory phase touch eight
    // different 16-byte bank groups.
    constexpr uint32_t kOnes = 0x11111111u;
    const int nsb = 1 << (vb - 4);
    const bool owner = 16 * t < nsb;
    uint64_t tops = 0;
    uint32_t sum = 0;
    if (owner) {
        uint4 *wv = reinterpret_cast<uint4 *>(w32) + 8 * t;
#pragma unroll
        for (int ee = 0; ee < 8; ++ee) {
            const int e = (ee + t) & 7;
            const uint4 q = wv[e];
            const uint32_t l0 = q.x * kOnes, s0 = l0 >> 28, h0 = q.y * kOnes + s0 * kOnes, t0 = h0 >> 28;
            const uint32_t l1 = q.z * kOnes, s1 = l1 >> 28, h1 = q.w * kOnes + s1 * kOnes, t1 = h1 >> 28;
            tops |= static_cast<uint64_t>(t0 | (t1 << 4)) << (8 * e);
            sum += t0 + t1;
            wv[e] = make_uint4(l0 << 4, (h0 << 4) | s0, l1 << 4, (h1 << 4) | s1);
        }
    }
    uint32_t total;
    uint32_t run = block_exclusive_scan<THREADS>(sum, scan_tmp, total);
    if (total != static_cast<uint32_t>(len)) return false;  // a sub-bucket of 16 or more keys
    if (owner) {
        uint32_t st[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const uint32_t a = run;
            run += static_cast<uint32_t>(tops >> (8 * e)) & 15u;
            st[e] = a | (run << 16);
            run += static_cast<uint32_t>(tops >> (8 * e + 4)) & 15u;
        }
        uint4 *sv = reinterpret_cast<uint4 *>(fst) + 2 * t;
        sv[0] = make_uint4(st[0], st[1], st[2], st[3]);
        sv[1] = make_uint4(st[4], st[5], st[6], st[7]);
    }
    __syncthreads();
    // positions: sub-bucket start + keys of lower low values + arrival rank
    bool bad = false;
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        if (j < rows) {
#pragma unroll
            for (int e = 0; e < V; ++e) {
                const uint32_t v = fr[j * V + e];
                if (v >> 20) {
                    const uint32_t f = v & 0xffffu;
                    const int sh = static_cast<int>(f & 7u) << 2;
                    const uint32_t pos = fst[f >> 4] + ((w32[f >> 3] >> sh) & 15u) + ((v >> 16) & 15u);
                    if (pos < static_cast<uint32_t>(len)) stage[lo_r + pos] = static_cast<uint16_t>(f);
                    else bad = true;
                }
            }
        }
    }
    if (bad) set_error(wk.ctl, kErrBounds);
    __syncthreads();
    // counters back to zero for the next unit, then the keys out
    for (int i = t; i < nsb / 2; i += THREADS) reinterpret_cast<uint4 *>(w32)[i] = make_uint4(0, 0, 0, 0);
    const K base = decode_key(common, wk.codec);  // decode flips by the top bit, which f never holds
    K *__restrict__ dstp = static_cast<K *>(wk.keys) + un.start;
    if (wk.keys_vec_ok) {
        const int a_i = (V - lo_r) % V;  // first key of a whole 16-byte group of the output
        const int nout = (len - a_i) > 0 ? (len - a_i) / V : 0;
        const int b_i = a_i + nout * V;
        for (int q = t; q < nout; q += THREADS) {
            const uint16_t *sp = stage + lo_r + a_i + q * V;
            K kv[V];
            if constexpr (V == 4) {
                const uint2 h = *reinterpret_cast<const uint2 *>(sp);
                kv[0] = base ^ static_cast<K>(h.x & 0xffffu);
                kv[1 % V] = base ^ static_cast<K>(h.x >> 16);
                kv[2 % V] = base ^ static_cast<K>(h.y & 0xffffu);
                kv[3 % V] = base ^ static_cast<K>(h.y >> 16);
            } else if constexpr (V == 2) {
                const uint32_t h = *reinterpret_cast<const uint32_t *>(sp);
                kv[0] = base ^ static_cast<K>(h & 0xffffu);
                kv[1 % V] = base ^ static_cast<K>(h >> 16);
            } else {
                kv[0] = base ^ static_cast<K>(sp[0]);
            }
            reinterpret_cast<uint4 *>(dstp + a_i)[q] = *reinterpret_cast<const uint4 *>(kv);
        }
        if (t < 2 * V) {
            const int i = t < V ? t : b_i + (t - V);
            if ((t < V && i < a_i && i < len) || (t >= V && i < len)) dstp[i] = base ^ static_cast<K>(stage[lo_r + i]);
        }
    } else {
        for (int i = t; i < len; i += THREADS) dstp[i] = base ^ static_cast<K>(stage[lo_r + i]);
    }
    if (t == 0) {
        atomicAdd(&wk.ctl->fin_counting, 1ull);
        atomicAdd(&wk.ctl->fin_fast, 1ull);
    }
    return true;
}

// Direct counting finish of a unit whose keys vary in at most 12 bits
// [lo, lo + span) with at least half a key per value: one counter per value,
// a scan, and every value's run written from its count into u16 staging
// (equal keys are bit-identical), then the keys rebuilt from the bits they
// all share (`a`) and written, decoded.  The keys are read again here (from
// L2: the caller has just read them) so that this path keeps its registers
// out of the caller's; thread t owns the values [t * per, (t + 1) * per).
// cnt: 2^span words, staged: len halfwords, both shared memory.
template <typename K, int THREADS>
__device__ __noinline__ void finish_direct(const K *__restrict__ src, K *__restrict__ dstp, int len, bool raw,
                                           Codec codec, K a, int lo, int span, uint32_t *cnt, uint16_t *staged,
                                           uint32_t *scan_tmp, Ctl *ctl) {
    const int t = threadIdx.x;
    const int nv = 1 << span;
    const uint32_t fmask = static_cast<uint32_t>(nv - 1);
    for (int i = t; i < nv; i += THREADS) cnt[i] = 0;
    __syncthreads();
    for (int i = t; i < len; i += THREADS) {
        K key = src[i];
        if (raw) key = encode_key(key, codec);
        atomicAdd(&cnt[static_cast<uint32_t>(key >> lo) & fmask], 1u);
    }
    __syncthreads();
    const int per = nv > THREADS ? nv / THREADS : 1;
    const int v0 = t * per;
    uint32_t sum = 0;
    if (v0 < nv)
        for (int e = 0; e < per; ++e) sum += cnt[v0 + e];
    uint32_t total;
    uint32_t at = block_exclusive_scan<THREADS>(sum, scan_tmp, total);
    const bool ok = total == static_cast<uint32_t>(len);
    if (ok && v0 < nv) {
        for (int e = 0; e < per; ++e) {
            const uint32_t c = cnt[v0 + e];
            for (uint32_t q = 0; q < c; ++q) staged[at + q] = static_cast<uint16_t>(v0 + e);
            at += c;
        }
    }
    __syncthreads();
    if (!ok) {
        if (t == 0) set_error(ctl, kErrBounds);
        return;
    }
    const K common = a & ~(static_cast<K>(fmask) << lo);  // the bits every key shares
    for (int i = t; i < len; i += THREADS)
        dstp[i] = decode_key(static_cast<K>(common | (static_cast<K>(staged[i]) << lo)), codec);
    if (t == 0) atomicAdd(&ctl->fin_counting, 1ull);
}

// Sorts every unit in shared memory and writes it, decoded, to its final
// place.  With at most 16 varying bits (and enough keys to fill the
// sub-buckets) one counting pass finishes the unit: the bits above the low 4
// select a sub-bucket, a 4-bit counter per (sub-bucket, low value) gives each
// key its arrival rank, and a scan over the sub-bucket totals plus the
// counters below the key's low value give its position -- the full
// remaining-bit counting sort, which is exact because keys with equal bits are
// identical.  Otherwise (more varying bits, or 16 equal keys overflowing a
// counter) the unit is split on its top log2(len)-ish varying bits in one
// unstable pass, and each key is ranked inside its sub-bucket -- a few keys --
// by comparison: strict order by (key, position), so a sub-bucket's ranks are
// a permutation of it.  A unit whose sub-buckets are too large for that goes
// to k_finish_lsd before anything is written.  Keys are loaded warp-striped
// (item j of thread t is key j*THREADS + t); a unit marked raw still holds the
// caller's encoding (an array or segment that fits one tile).
template <typename K, int THREADS, int ITEMS>
__global__ void __launch_bounds__(THREADS, 4) k_finish(Work wk) {
    pdl_enter();
    using FL = FinLayout<K, THREADS, ITEMS>;
    K *sm_keys = reinterpret_cast<K *>(g_dyn_smem);
    K *ta = reinterpret_cast<K *>(g_dyn_smem + FL::kTa);
    K *to = reinterpret_cast<K *>(g_dyn_smem + FL::kTo);
    uint32_t *cnt = reinterpret_cast<uint32_t *>(g_dyn_smem + FL::kCnt);
    uint32_t *scan_tmp = reinterpret_cast<uint32_t *>(g_dyn_smem + FL::kScan);
    uint64_t *words = reinterpret_cast<uint64_t *>(g_dyn_smem + FL::kWords);
    uint32_t *w32 = reinterpret_cast<uint32_t *>(g_dyn_smem + FL::kWords);
    uint32_t *tot32 = reinterpret_cast<uint32_t *>(g_dyn_smem + FL::kTotals);
    uint32_t *st32 = reinterpret_cast<uint32_t *>(g_dyn_smem + FL::kStarts);
    const uint16_t *st16 = reinterpret_cast<const uint16_t *>(g_dyn_smem + FL::kStarts);
    K *stage = reinterpret_cast<K *>(g_dyn_smem + FL::kStage);
    const int t = threadIdx.x;
    if (wk.ctl->error) return;
    const uint32_t nu = min(wk.ctl->n_units, wk.max_units);
    K *__restrict__ out = static_cast<K *>(wk.keys);
    Unit *next = reinterpret_cast<Unit *>(g_dyn_smem + FL::kNext);  // descriptors, double-buffered
    if (t == 0 && blockIdx.x < nu) cp_async16(&next[0], &wk.units[blockIdx.x]);
    int it = 0;
    bool clean = false;  // every counter word of the fast counting path is zero
    for (uint32_t u = blockIdx.x; u < nu; u += gridDim.x, ++it) {
        if (t == 0) cp_async_wait_all();
        __syncthreads();
        const Unit un = next[it & 1];
        if (t == 0 && u + gridDim.x < nu) cp_async16(&next[(it + 1) & 1], &wk.units[u + gridDim.x]);
        const bool raw = un.raw;
        {
            const int vb = un.vbits;
            const bool vec = un.src ? true : wk.keys_vec_ok;
            if (!raw && vec && vb >= 8 && vb <= 16 && (1 << (vb - 4)) <= 4 * static_cast<int>(un.len)) {
                if (!clean) {
                    uint4 *z = reinterpret_cast<uint4 *>(g_dyn_smem + FL::kWords);
                    for (int i = t; i < kSplitCap / 2; i += THREADS) z[i] = make_uint4(0, 0, 0, 0);
                    __syncthreads();
                }
                clean = finish_count_fast<K, THREADS, ITEMS>(wk, un, vb);
                if (clean) continue;
                __syncthreads();  // the general path below reuses the counter words
            }
        }
        clean = false;
        const K *__restrict__ src = src_of<K>(wk, un.src) + un.start;
        K *__restrict__ dstp = out + un.start;
        const int len = static_cast<int>(un.len);
        const int jmax = (len + THREADS - 1) / THREADS;
        // bit j: item j (key j*THREADS + t) exists
        const int rem = len - t;
        uint32_t vm = 0;
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) vm |= static_cast<uint32_t>(j * THREADS < rem) << j;
        K k[ITEMS];
        K a = static_cast<K>(~K(0)), o = 0;
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            k[j] = 0;
            if ((vm >> j) & 1u) {
                K key = src[j * THREADS + t];
                if (raw) key = encode_key(key, wk.codec);
                k[j] = key;
                a &= key;
                o |= key;
            }
        }
        block_and_or_k<K, THREADS>(a, o, ta, to);
        const K v = a ^ o;
        if (v == 0) {  // one repeated key: write it len times
            const K val = decode_key(a, wk.codec);
            for (int i = t; i < len; i += THREADS) dstp[i] = val;
            continue;
        }
        const int lo = lsb_pos<K>(v);
        const int hi = msb_pos<K>(v) + 1;
        const int span = hi - lo;
        const int lbits = span < 4 ? span : 4;
        const int sbits = span - lbits;
        if constexpr (sizeof(K) == 4) {  // (wider keys rarely leave so few varying bits with so many keys)
            if (__builtin_expect(span <= kSplitBits && (1 << span) <= 2 * len, 0)) {
                finish_direct<K, THREADS>(src, dstp, len, raw, wk.codec, a, lo, span, w32,
                                          reinterpret_cast<uint16_t *>(g_dyn_smem + FL::kStage16), scan_tmp, wk.ctl);
                continue;
            }
        }
        if (span <= kSplitBits + 4 && (1 << sbits) <= 4 * len) {
            // counting path: count (every table entry is cleared and scanned:
            // 16 sub-buckets per thread, unused ones stay zero)
            {
                uint4 *z = reinterpret_cast<uint4 *>(g_dyn_smem + FL::kWords);
                for (int i = t; i < (10 * kSplitCap) / 16; i += THREADS) z[i] = make_uint4(0, 0, 0, 0);
            }
            __syncthreads();
            const uint32_t fmask = (1u << span) - 1u, lmask = (1u << lbits) - 1u;
            uint32_t arr[(ITEMS + 7) / 8];
#pragma unroll
            for (int j = 0; j < (ITEMS + 7) / 8; ++j) arr[j] = 0;
            bool ovf = false;
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) {
                if ((vm >> j) & 1u) {
                    const uint32_t f = static_cast<uint32_t>(k[j] >> lo) & fmask;
                    const uint32_t low = f & lmask, sb = f >> lbits;
                    const int sh = 4 * static_cast<int>(low & 7u);
                    const uint32_t old = atomicAdd(&w32[2 * sb + (low >> 3)], 1u << sh);
                    atomicAdd(&tot32[sb >> 1], 1u << (16 * (sb & 1u)));
                    const uint32_t r = (old >> sh) & 15u;
                    ovf |= r == 15u;  // the 16th equal key: its counter wraps
                    arr[j >> 3] |= r << (4 * (j & 7));
                }
            }
            if (!__syncthreads_or(ovf)) {
                // sub-bucket starts: thread t owns sub-buckets [16t, 16t + 16)
                bool small;
                {
                    const uint4 *tv = reinterpret_cast<const uint4 *>(tot32) + 2 * t;
                    const uint4 q0 = tv[0], q1 = tv[1];
                    const uint32_t c[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
                    uint32_t sum = 0;
#pragma unroll
                    for (int e = 0; e < 8; ++e) sum += (c[e] & 0xffffu) + (c[e] >> 16);
                    uint32_t total;
                    uint32_t run = block_exclusive_scan<THREADS>(sum, scan_tmp, total);
                    uint32_t o[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const uint32_t s0 = run;
                        run += c[e] & 0xffffu;
                        o[e] = s0 | (run << 16);
                        run += c[e] >> 16;
                    }
                    uint4 *sv = reinterpret_cast<uint4 *>(st32) + 2 * t;
                    sv[0] = make_uint4(o[0], o[1], o[2], o[3]);
                    sv[1] = make_uint4(o[4], o[5], o[6], o[7]);
                    small = true;
#pragma unroll
                    for (int e = 0; e < 8; ++e) small &= (c[e] & 0xffffu) < 16u && (c[e] >> 16) < 16u;
                }
                // every sub-bucket under 16 keys: turn its counters into exclusive
                // prefix counters in place (multiplying by 0x1111... sums the
                // nibbles below each nibble without carries), so a key's
                // offset inside its sub-bucket is one nibble
                const bool prefix = __syncthreads_and(small);
                if (prefix) {
#pragma unroll
                    for (int e = 0; e < kSplitCap / THREADS; ++e) {
                        const int sb = e * THREADS + t;
                        words[sb] = (words[sb] * 0x1111111111111111ull) << 4;
                    }
                    __syncthreads();
                }
                // positions: sub-bucket start + keys of lower low values + arrival rank
                uint32_t posr[(ITEMS + 1) / 2];
#pragma unroll
                for (int j = 0; j < (ITEMS + 1) / 2; ++j) posr[j] = 0;
                if (prefix) {
#pragma unroll
                    for (int j = 0; j < ITEMS; ++j) {
                        if ((vm >> j) & 1u) {
                            const uint32_t f = static_cast<uint32_t>(k[j] >> lo) & fmask;
                            const uint32_t low = f & lmask, sb = f >> lbits;
                            const uint32_t below = (w32[2 * sb + (low >> 3)] >> (4 * (low & 7u))) & 15u;
                            const uint32_t pos = st16[sb] + below + ((arr[j >> 3] >> (4 * (j & 7))) & 15u);
                            posr[j >> 1] |= pos << ((j & 1) * 16);
                        }
                    }
                } else {
#pragma unroll
                for (int j = 0; j < ITEMS; ++j) {
                    if ((vm >> j) & 1u) {
                        const uint32_t f = static_cast<uint32_t>(k[j] >> lo) & fmask;
                        const uint32_t low = f & lmask, sb = f >> lbits;
                        const uint64_t wd = words[sb];
                        const uint32_t x = static_cast<uint32_t>(wd), y = static_cast<uint32_t>(wd >> 32);
                        const uint32_t mk = (1u << (4 * (low & 7u))) - 1u;
                        const bool upper = low >= 8u;
                        const uint32_t xm = x & (upper ? ~0u : mk), ym = y & (upper ? mk : 0u);
                        constexpr uint32_t m4 = 0x0F0F0F0Fu;
                        const uint32_t below =
                            __dp4a((xm & m4) + ((xm >> 4) & m4) + (ym & m4) + ((ym >> 4) & m4), 0x01010101u, 0u);
                        const uint32_t pos = st16[sb] + below + ((arr[j >> 3] >> (4 * (j & 7))) & 15u);
                        posr[j >> 1] |= pos << ((j & 1) * 16);
                    }
                }
                }
                __syncthreads();
                // keys to the staging buffer (slot lo_r + position), then out
                const int lo_r = static_cast<int>(un.start % FL::V);
                bool bad = false;
#pragma unroll
                for (int j = 0; j < ITEMS; ++j) {
                    if ((vm >> j) & 1u) {
                        const uint32_t pos = (posr[j >> 1] >> ((j & 1) * 16)) & 0xffffu;
                        if (pos < static_cast<uint32_t>(len)) stage[lo_r + pos] = k[j];
                        else bad = true;
                    }
                }
                if (bad) set_error(wk.ctl, kErrBounds);
                if (t == 0) atomicAdd(&wk.ctl->fin_counting, 1ull);
                __syncthreads();
                if (wk.keys_vec_ok) {
                    constexpr int V = FL::V;
                    const int a_i = (V - lo_r) % V;                        // first key of a whole 16-byte group
                    const int nvec = (len - a_i) > 0 ? (len - a_i) / V : 0;
                    const int b_i = a_i + nvec * V;
                    const uint4 *sv = reinterpret_cast<const uint4 *>(stage + lo_r + a_i);
                    uint4 *dv = reinterpret_cast<uint4 *>(dstp + a_i);
                    for (int q = t; q < nvec; q += THREADS) {
                        K kv[V];
                        *reinterpret_cast<uint4 *>(kv) = sv[q];
#pragma unroll
                        for (int e = 0; e < V; ++e) kv[e] = decode_key(kv[e], wk.codec);
                        dv[q] = *reinterpret_cast<uint4 *>(kv);
                    }
                    if (t < 2 * V) {
                        const int i = t < V ? t : b_i + (t - V);
                        if ((t < V && i < a_i && i < len) || (t >= V && i < len))
                            dstp[i] = decode_key(stage[lo_r + i], wk.codec);
                    }
                } else {
                    for (int i = t; i < len; i += THREADS) dstp[i] = decode_key(stage[lo_r + i], wk.codec);
                }
                __syncthreads();
                continue;
            }
        }
        const int want = max(8, 32 - __clz(len - 1));
        const int bits = min(span, min(want, kSplitBits));
        const int top = hi - bits;
        const int nb = 1 << bits;
        const uint32_t dmask = static_cast<uint32_t>(nb - 1);
        // split: count
        for (int i = t; i <= split_pad(nb); i += THREADS) cnt[i] = 0;
        __syncthreads();
        uint32_t local[(ITEMS + 1) / 2];
#pragma unroll
        for (int j = 0; j < (ITEMS + 1) / 2; ++j) local[j] = 0;
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            if (j < jmax && j * THREADS + t < len) {
                const int d = static_cast<int>(static_cast<uint32_t>(k[j] >> top) & dmask);
                local[j >> 1] |= atomicAdd(&cnt[split_pad(d)], 1u) << ((j & 1) * 16);
            }
        }
        __syncthreads();
        // split: exclusive starts (thread t scans e_per consecutive counters);
        // a sub-bucket too large for comparison ranking sends the unit to the
        // LSD finish before anything is written
        bool too_big = false;
        {
            const int e_per = nb > THREADS ? nb / THREADS : 1;
            const int g0 = split_pad(t * e_per);
            const bool owner = t * e_per < nb;
            uint32_t sum = 0;
            if (owner)
                for (int e = 0; e < e_per; ++e) {
                    const uint32_t c = cnt[g0 + e];
                    sum += c;
                    too_big |= c > kCmpMaxBucket;
                }
            uint32_t total;
            uint32_t run = block_exclusive_scan<THREADS>(sum, scan_tmp, total);
            if (owner)
                for (int e = 0; e < e_per; ++e) {
                    const uint32_t c = cnt[g0 + e];
                    cnt[g0 + e] = run;
                    run += c;
                }
            if (t == 0) cnt[split_pad(nb)] = total;
        }
        too_big = __syncthreads_or(too_big) && bits < span;
        if (too_big) {
            if (t == 0) {
                const uint32_t f = atomicAdd(&wk.ctl->n_fb, 1u);
                if (f < wk.max_units) wk.fb_units[f] = un;
                else set_error(wk.ctl, kErrCapacity);
            }
            continue;
        }
        if (t == 0) atomicAdd(&wk.ctl->fin_compare, 1ull);
        // split: place
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            if (j < jmax && j * THREADS + t < len) {
                const int d = static_cast<int>(static_cast<uint32_t>(k[j] >> top) & dmask);
                sm_keys[cnt[split_pad(d)] + ((local[j >> 1] >> ((j & 1) * 16)) & 0xffffu)] = k[j];
            }
        }
        __syncthreads();
        if (bits == span) {
            for (int i = t; i < len; i += THREADS) dstp[i] = decode_key(sm_keys[i], wk.codec);
            __syncthreads();
            continue;
        }
        // rank inside sub-buckets by comparison, write to the final place
        for (int p2 = t; p2 < len; p2 += THREADS) {
            const K kp = sm_keys[p2];
            const int d = static_cast<int>(static_cast<uint32_t>(kp >> top) & dmask);
            const int s0 = static_cast<int>(cnt[split_pad(d)]);
            const int s1 = static_cast<int>(cnt[split_pad(d + 1)]);
            int r = 0;
            for (int q = s0; q < s1; ++q) {
                const K kq = sm_keys[q];
                r += (kq < kp) | ((kq == kp) & (q < p2));
            }
            dstp[s0 + r] = decode_key(kp, wk.codec);
        }
        __syncthreads();
    }
}

template <typename K, int THREADS, int ITEMS>
constexpr size_t finish_smem() {
    return FinLayout<K, THREADS, ITEMS>::kEnd;
}

// Finish of the units k_finish handed over (skewed: a sub-bucket too large
// for comparison ranking): LSD passes over the unit's varying bits, the
// first unstable (its input order is arbitrary), the later ones stable,
// then the decoded keys go to their final place.
template <typename K, int THREADS, int ITEMS>
__global__ void __launch_bounds__(THREADS, 4) k_finish_lsd(Work wk) {
    pdl_enter();
    using L = TileLoad<K, THREADS, ITEMS>;
    constexpr int TILE = THREADS * ITEMS;
    constexpr int V = L::V;
    constexpr int WARPS = THREADS / 32;
    using RS = RankSmem<THREADS, sizeof(K) * (TILE + 2 * WARPS), true>;
    using R = Ranker<K, THREADS, ITEMS, RS>;
    K *sm_keys = reinterpret_cast<K *>(g_dyn_smem);
    K *ta = reinterpret_cast<K *>(g_dyn_smem + sizeof(K) * TILE);
    K *to = ta + WARPS;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (wk.ctl->error) return;
    for (int i = threadIdx.x; i < 2 * WARPS * kBins; i += THREADS) RS::wm()[i] = 0;  // peer masks start clear
    const uint32_t nu = min(wk.ctl->n_fb, wk.max_units);
    K *__restrict__ out = static_cast<K *>(wk.keys);
    for (uint32_t u = blockIdx.x; u < nu; u += gridDim.x) {
        const Unit un = wk.fb_units[u];
        const K *__restrict__ src = src_of<K>(wk, un.src);
        const bool vec_ok = un.src ? true : wk.keys_vec_ok;
        const int len = static_cast<int>(un.len);
        const uint64_t wstart = un.start - un.start % V;
        const uint32_t lo_r = static_cast<uint32_t>(un.start - wstart);
        K k[ITEMS];
        uint32_t vmask = L::load(src, wstart, lo_r, lo_r + un.len, vec_ok, k);
        K a = static_cast<K>(~K(0)), o = 0;
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            if (un.raw) k[j] = encode_key(k[j], wk.codec);
            if ((vmask >> j) & 1u) {
                a &= k[j];
                o |= k[j];
            }
        }
        block_and_or_k<K, THREADS>(a, o, ta, to);
        K *__restrict__ dstp = out + un.start;
        const K v = a ^ o;
        const int lo = v ? lsb_pos<K>(v) : 0;
        const int hi = v ? msb_pos<K>(v) + 1 : 1;
        const int passes = (hi - lo + kRadixBits - 1) / kRadixBits;
        const int width = (hi - lo + passes - 1) / passes;
        R::template rank_and_place<false>(k, vmask, lo, (1u << width) - 1, sm_keys);
        vmask = striped_mask<ITEMS>(len);
        for (int ps = 1, sh = lo + width; ps < passes; ++ps, sh += width) {
            const K *row = sm_keys + warp * 32 * ITEMS + lane;
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) k[j] = (vmask >> j) & 1u ? row[j * 32] : K(0);
            __syncthreads();
            R::template rank_and_place<true>(k, vmask, sh, (1u << min(width, hi - sh)) - 1, sm_keys);
        }
        for (int i = threadIdx.x; i < len; i += THREADS) dstp[i] = decode_key(sm_keys[i], wk.codec);
        __syncthreads();
    }
}

template <typename K, int THREADS, int ITEMS>
constexpr size_t finish_lsd_smem() {
    return RankSmem<THREADS, sizeof(K) * (THREADS * ITEMS + 2 * (THREADS / 32)), true>::kEnd;
}

template <typename K>
__global__ void k_fill(Work wk) {
    pdl_enter();
    if (wk.ctl->error) return;
    const uint32_t nf = wk.ctl->n_fills;
    K *out = static_cast<K *>(wk.keys);
    for (uint32_t f = blockIdx.x; f < nf; f += gridDim.x) {
        const Fill fl = wk.fills[f];
        if (fl.start + fl.len > wk.n) {
            set_error(wk.ctl, kErrBounds);
            continue;
        }
        K val = static_cast<K>(fl.value);
        if constexpr (sizeof(K) > 8) val |= static_cast<K>(fl.value_hi) << 64;
        const K v = decode_key(val, wk.codec);
        for (uint32_t i = threadIdx.x; i < fl.len; i += blockDim.x) out[fl.start + i] = v;
    }
}

// Intermediate state only: the buckets still open before `level` (partitioned
// by the bits above their h, unsorted below) are written, decoded, to their
// place in the caller's buffer as they are.
template <typename K>
__global__ void k_drain(Work wk, int level) {
    pdl_enter();
    if (wk.ctl->error) return;
    const int p = level & 1;
    const uint32_t nb = wk.ctl->n_buckets[p];
    K *out = static_cast<K *>(wk.keys);
    for (uint32_t i = blockIdx.x; i < nb; i += gridDim.x) {
        const Bucket b = wk.buckets[p][i];
        if (b.src == 0 && b.raw) continue;  // never moved, never encoded
        const K *src = src_of<K>(wk, b.src);
        for (uint64_t j = threadIdx.x; j < b.len; j += blockDim.x)
            out[b.start + j] = decode_key(src[b.start + j], wk.codec);
    }
}

// ---- key-value sorting (stable): values travel with their keys -------------
//
// The keys-only levels partition freely inside a digit (equal keys are
// bit-identical).  With values riding along, equal keys must keep their input
// order, so the scatter and the finish below rank stably: a tile's keys sit
// warp-striped (item j of lane l of warp w is tile index (w * ITEMS + j) * 32
// + l) and each key's place is its digit's start in the tile plus the keys of
// that digit before it in tile order -- per-(digit, warp) counters and
// per-warp peer masks.  The histogram, column scan and classify steps only
// look at keys and are shared with keys-only sorting; a chunk's tiles are
// ranked in order, each digit's destination moving on by the tile's count.

// Scatter tiles per chunk of the key-value sort.
constexpr uint32_t kKvChunkTiles = 4;

// Key-value finish of 8-byte keys: units with more varying bits than
// kKvWideBits are sorted by their top 16 bits, then runs of ties up to
// kKvTieRun keys by comparison.
constexpr int kKvWideBits = 24;
constexpr int kKvTieRun = 16;

// Shared memory of the stable ranking at byte offset BASE: two sets of
// per-(digit, warp) counters, digit-major with one pad word per digit
// (successive rankings alternate between the sets, so that one is cleared
// while the other is in use), the per-warp peer masks (two sets, alternating
// by item), and the scan scratch.
template <int THREADS, size_t BASE>
struct StableSmem {
    static constexpr int WARPS = THREADS / 32;
    static constexpr int STRIDE = WARPS + 1;
    static constexpr int kWcWords = kBins * STRIDE;
    static constexpr size_t kWc = BASE;
    static constexpr size_t kWm = kWc + 16 * ((8 * kWcWords + 15) / 16);
    static constexpr size_t kScan = kWm + 8 * WARPS * kBins;
    static constexpr size_t kEnd = kScan + 16 * ((4 * (WARPS + 1) + 15) / 16);
    __device__ static uint32_t *wc(int set) {
        return reinterpret_cast<uint32_t *>(g_dyn_smem + kWc) + set * kWcWords;
    }
    __device__ static uint32_t *wm() { return reinterpret_cast<uint32_t *>(g_dyn_smem + kWm); }
    __device__ static uint32_t *scan() { return reinterpret_cast<uint32_t *>(g_dyn_smem + kScan); }
    // Both counter sets (and the peer masks) zeroed; the caller syncs before the first ranking.
    __device__ static void clear() {
        for (int i = threadIdx.x; i < 2 * kWcWords; i += blockDim.x) wc(0)[i] = 0;
        for (int i = threadIdx.x; i < 2 * WARPS * kBins; i += blockDim.x) wm()[i] = 0;
    }
};

// Places every valid item of the tile -- key and value -- in out_k / out_v
// ordered by digit, ties in tile order; thread d <= mask also gets the
// tile's count of digit d.  Counter set `set` must be zero on entry; the
// other set is zeroed here for the next ranking (the caller passes the sets
// alternately and has a barrier between this call's last read of the
// counters -- the lookups at the end -- and the next call; the placed items
// are visible after the caller's next barrier).  A rank inside a warp's
// digit is below 2^16 (the tile is smaller), so two share a register.
// Three barriers.
template <typename K, typename V, int THREADS, int ITEMS, typename SS>
__device__ __forceinline__ void stable_rank_place(const K (&keys)[ITEMS], const V (&vals)[ITEMS], uint32_t vmask,
                                                  int shift, uint32_t mask, int set, uint32_t &count, K *out_k,
                                                  V *out_v) {
    constexpr int WARPS = THREADS / 32;
    constexpr int STRIDE = WARPS + 1;
    static_assert(THREADS >= kBins, "one thread per digit in the scans");
    static_assert(THREADS * ITEMS < 65536, "ranks fit 16 bits");
    uint32_t *wc = SS::wc(set);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int t = threadIdx.x;
    {
        uint32_t *wc_next = SS::wc(set ^ 1);
        for (int i = t; i < SS::kWcWords; i += THREADS) wc_next[i] = 0;
    }
    const unsigned lt = lanemask_lt();
    uint32_t rank[(ITEMS + 1) / 2];  // item j's rank in its warp's digit at bit 16 (j & 1)
#pragma unroll
    for (int j = 0; j < (ITEMS + 1) / 2; ++j) rank[j] = 0;
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const bool valid = (vmask >> j) & 1u;
        if (__any_sync(kFull, valid)) {  // warp-uniform
            const uint32_t d = static_cast<uint32_t>(keys[j] >> shift) & mask;
            uint32_t *wcd = wc + d * STRIDE + warp;
            // lanes of one digit find each other through the warp's mask word
            // of the digit (two mask sets alternate by item, so a set is
            // cleared before its next use without another barrier); the
            // lowest lane of the group advances the warp's counter
            uint32_t *wm = SS::wm() + ((j & 1) * WARPS + warp) * kBins;
            if (valid) atomicOr(&wm[d], 1u << lane);
            __syncwarp();
            const uint32_t peers = wm[d];
            const uint32_t before = *wcd;
            __syncwarp();
            const uint32_t r = __popc(peers & lt);
            if (valid && r == 0) {
                *wcd = before + __popc(peers);
                wm[d] = 0;
            }
            rank[j >> 1] |= (before + r) << ((j & 1) * 16);
        }
    }
    __syncthreads();
    // thread d: total of digit d; exclusive prefix over digits (warp scan,
    // then the totals of the warps before); the warps' starts written back
    uint32_t run = 0;
    if (t <= static_cast<int>(mask)) {
#pragma unroll
        for (int w = 0; w < WARPS; ++w) run += wc[t * STRIDE + w];
    }
    count = run;
    uint32_t x = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    uint32_t *tmp = SS::scan();
    if (lane == 31) tmp[warp] = x;
    __syncthreads();
    uint32_t acc = x - run;
#pragma unroll
    for (int w = 0; w < WARPS; ++w)
        if (w < warp) acc += tmp[w];
    if (t <= static_cast<int>(mask)) {
#pragma unroll
        for (int w = 0; w < WARPS; ++w) {
            const uint32_t c = wc[t * STRIDE + w];
            wc[t * STRIDE + w] = acc;
            acc += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        if ((vmask >> j) & 1u) {
            const uint32_t p = wc[(static_cast<uint32_t>(keys[j] >> shift) & mask) * STRIDE + warp] +
                               ((rank[j >> 1] >> ((j & 1) * 16)) & 0xffffu);
            out_k[p] = keys[j];
            out_v[p] = vals[j];
        }
    }
}

template <typename V>
__device__ __forceinline__ const V *vals_of(const Work &wk, int src) {
    return static_cast<const V *>(src ? wk.vals_alt : wk.vals);
}

template <typename V>
__device__ __forceinline__ V *vals_dst_of(const Work &wk, int src) {
    return static_cast<V *>(src ? wk.vals : wk.vals_alt);
}


// Stable scatter of one level, keys and values: each tile of a chunk is
// loaded warp-striped, ranked stably by digit, staged (keys and values) in
// digit order, and written out in staging order to its digit runs.  The
// chunk's destinations come from the histogram pass exactly as in k_scatter
// and move on by each tile's digit counts; every one is checked against the
// bucket before it is written.  The loop is software-pipelined: the next
// tile's keys and values are loaded into the (then free) registers while the
// staged tile is written out, and the next chunk's record while this tile is
// ranked.
template <typename K, typename V, int THREADS, int ITEMS>
struct ScatterKvSmem {
    static constexpr int TILE = THREADS * ITEMS;
    static constexpr size_t kVals = sizeof(K) * TILE;
    static constexpr size_t kRank = ((kVals + sizeof(V) * TILE) + 15) & ~size_t(15);
    using RS = StableSmem<THREADS, kRank>;
    static constexpr size_t kOff = (RS::kEnd + 15) & ~size_t(15);  // u64[kBins]
    static constexpr size_t kEnd = kOff + 8 * kBins;
};

// Keys and values of tile positions [0, len) of a buffer range into
// registers, warp-striped with IT items per thread (item j of lane l of warp
// w is position (w * IT + j) * 32 + l); raw argsort ranges make their
// positions.  Returns the validity mask.
template <typename K, typename V, int ITEMS>
__device__ __forceinline__ uint32_t kv_load(const Work &wk, int src, bool raw, uint64_t start, uint32_t len, int it,
                                            K (&k)[ITEMS], V (&v)[ITEMS]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const K *__restrict__ ks = src_of<K>(wk, src);
    const V *__restrict__ vs = vals_of<V>(wk, src);
    const bool make_pos = wk.kv_positions && raw;
    uint32_t vmask = 0;
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const uint32_t idx = static_cast<uint32_t>((warp * it + j) * 32 + lane);
        k[j] = 0;
        v[j] = 0;
        if (j < it && idx < len) {
            k[j] = ks[start + idx];
            v[j] = make_pos ? static_cast<V>(start + idx) : vs[start + idx];
            vmask |= 1u << j;
        }
    }
    return vmask;
}

template <typename K, typename V, int THREADS, int ITEMS, int MINB>
__global__ void __launch_bounds__(THREADS, MINB) k_scatter_kv(Work wk, int level) {
    pdl_enter();
    using SM = ScatterKvSmem<K, V, THREADS, ITEMS>;
    using RS = typename SM::RS;
    constexpr uint32_t TILE = THREADS * ITEMS;
    constexpr int WARPS = THREADS / 32;
    constexpr int STRIDE = WARPS + 1;
    K *sm_keys = reinterpret_cast<K *>(g_dyn_smem);
    V *sm_vals = reinterpret_cast<V *>(g_dyn_smem + SM::kVals);
    unsigned long long *off = reinterpret_cast<unsigned long long *>(g_dyn_smem + SM::kOff);
    const int p = level & 1;
    const int t = threadIdx.x;
    if (wk.ctl->error) return;
    write_child_chunks(wk, p ^ 1);  // records of the buckets this level's classify opened
    RS::clear();
    __syncthreads();
    int set = 0;  // counter set of the next ranking
    const uint32_t nch = wk.ctl->n_chunks[p];
    // pipeline position: tile ti of chunk c (record ch, its bucket b), whose
    // keys and values are in k / v
    K k[ITEMS];
    V v[ITEMS];
    uint32_t vmask = 0;
    uint32_t c = blockIdx.x, ti = 0;
    Chunk ch = {};
    Bucket b = {};
    auto tile_len = [&](const Chunk &x, uint32_t i) -> uint32_t {
        const uint32_t s0 = i * TILE;
        return s0 < x.len ? min(x.len - s0, TILE) : 0u;
    };
    auto load_tile = [&]() {
        vmask = b.scatter ? kv_load<K, V, ITEMS>(wk, b.src, b.raw, ch.start + static_cast<uint64_t>(ti) * TILE,
                                                 tile_len(ch, ti), ITEMS, k, v)
                          : 0u;
    };
    if (c < nch) {
        ch = wk.chunks[p][c];
        b = wk.buckets[p][ch.bucket];
        load_tile();
    }
    uint64_t dest = 0;  // thread d <= mask: where digit d's next key of this chunk goes
    while (c < nch) {
        const uint32_t ntiles = b.scatter ? max(1u, (ch.len + TILE - 1) / TILE) : 1u;
        const bool last_tile = ti + 1 >= ntiles;
        const uint32_t cn = c + gridDim.x;
        Chunk chn = {};
        if (last_tile && cn < nch) chn = wk.chunks[p][cn];  // arrives while this tile is ranked
        const int r_eff = min(wk.radix_bits, b.h);
        const int shift = b.h - r_eff;
        const uint32_t mask = (1u << r_eff) - 1;
        const uint32_t tl = tile_len(ch, ti);
        if (b.scatter) {  // block-uniform
            // a chunk's digit d starts at bucket start + digit base + keys of
            // digit d in the bucket's earlier chunks; each tile moves it on
            if (ti == 0 && t <= static_cast<int>(mask))
                dest = b.start + wk.bucket_base[static_cast<size_t>(ch.bucket) * wk.bins + t] +
                       wk.hist[static_cast<size_t>(t) * wk.max_chunks + c];
            if (b.raw) {
#pragma unroll
                for (int j = 0; j < ITEMS; ++j) k[j] = encode_key(k[j], wk.codec);
            }
            uint32_t cnt;
            stable_rank_place<K, V, THREADS, ITEMS, RS>(k, v, vmask, shift, mask, set, cnt, sm_keys,
                                                          sm_vals);
            // digit d's run: staging slots from its tile start, so the key at
            // staging slot q goes to off[d] + q
            if (t <= static_cast<int>(mask)) {
                off[t] = dest - RS::wc(set)[t * STRIDE];
                dest += cnt;
            }
            set ^= 1;
            __syncthreads();
        }
        const Bucket cb = b;
        // the next tile into the registers; its loads overlap the write-out below
        if (!last_tile) {
            ++ti;
            load_tile();
        } else {
            c = cn;
            ti = 0;
            if (c < nch) {
                ch = chn;
                b = wk.buckets[p][ch.bucket];
                load_tile();
            }
        }
        if (cb.scatter) {
            K *__restrict__ dst = dst_of<K>(wk, cb.src);
            V *__restrict__ vdst = vals_dst_of<V>(wk, cb.src);
            bool oob = false;
            for (uint32_t q = t; q < tl; q += THREADS) {
                const K key = sm_keys[q];
                const uint64_t pos = off[static_cast<uint32_t>(key >> shift) & mask] + q;
                if (pos - cb.start < cb.len) {
                    dst[pos] = key;
                    vdst[pos] = sm_vals[q];
                } else {
                    oob = true;
                }
            }
            if (oob) set_error(wk.ctl, kErrBounds);
        }
        // (the next tile stages only after the barriers inside its ranking)
    }
}

// Stable finish of a unit, keys and values: loaded warp-striped (input
// order, IT = ceil(len / THREADS) items per thread so that every warp has
// work), then one stable pass per digit of at most 8 bits over the unit's
// varying bits, least significant first, each staging keys and values in
// shared memory; the last pass's staging is the sorted unit, written decoded
// to its final place (values beside, or int64 positions for an argsort).
// The next unit is loaded into the registers while the staged one is written.
template <typename K, typename V, int THREADS, int ITEMS>
struct FinishKvSmem {
    static constexpr int TILE = THREADS * ITEMS;
    static constexpr int WARPS = THREADS / 32;
    static constexpr size_t kVals = sizeof(K) * TILE;
    static constexpr size_t kTa = (kVals + sizeof(V) * TILE + 15) & ~size_t(15);
    static constexpr size_t kTo = kTa + sizeof(K) * WARPS;
    static constexpr size_t kRank = (kTo + sizeof(K) * WARPS + 15) & ~size_t(15);
    using RS = StableSmem<THREADS, kRank>;
    static constexpr size_t kEnd = RS::kEnd;
};

template <typename V>
__device__ __forceinline__ void kv_out(const Work &wk, uint64_t i, V v) {
    if (wk.kv_positions) {
        if (wk.out_idx) wk.out_idx[i] = static_cast<int64_t>(v);
        if (wk.out_vals) static_cast<V *>(wk.out_vals)[i] = v;  // 32-bit positions for a gather of the values
    } else {
        static_cast<V *>(wk.out_vals)[i] = v;
    }
}

template <typename K, typename V, int THREADS, int ITEMS, int MINB>
__global__ void __launch_bounds__(THREADS, MINB) k_finish_kv(Work wk) {
    pdl_enter();
    using SM = FinishKvSmem<K, V, THREADS, ITEMS>;
    using RS = typename SM::RS;
    K *sm_keys = reinterpret_cast<K *>(g_dyn_smem);
    V *sm_vals = reinterpret_cast<V *>(g_dyn_smem + SM::kVals);
    K *ta = reinterpret_cast<K *>(g_dyn_smem + SM::kTa);
    K *to = reinterpret_cast<K *>(g_dyn_smem + SM::kTo);
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (wk.ctl->error) return;
    RS::clear();  // (the AND/OR reduction's barriers come before the first ranking)
    int set = 0;  // counter set of the next ranking
    const uint32_t nu = min(wk.ctl->n_units, wk.max_units);
    K *__restrict__ out = static_cast<K *>(wk.keys);
    // a unit that fits the tile and the buffer, else an empty one (and the bounds error)
    auto fetch = [&](uint32_t u) {
        Unit un = wk.units[u];
        if (un.len > static_cast<uint32_t>(SM::TILE) || un.start + un.len > wk.n) {
            if (t == 0) set_error(wk.ctl, kErrBounds);
            un.len = 0;
        }
        return un;
    };
    K k[ITEMS];
    V v[ITEMS];
    uint32_t vmask = 0;
    int it = 0;
    uint32_t u = blockIdx.x;
    Unit un = {};
    if (u < nu) {
        un = fetch(u);
        it = static_cast<int>((un.len + THREADS - 1) / THREADS);
        vmask = kv_load<K, V, ITEMS>(wk, un.src, un.raw, un.start, un.len, it, k, v);
    }
    for (; u < nu; u += gridDim.x) {
        const uint32_t un_next = u + gridDim.x;
        const Unit cur = un;
        const int cit = it;
        const int len = static_cast<int>(cur.len);
        K a = static_cast<K>(~K(0)), o = 0;
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            if ((vmask >> j) & 1u) {
                if (cur.raw) k[j] = encode_key(k[j], wk.codec);
                a &= k[j];
                o |= k[j];
            }
        }
        block_and_or_k<K, THREADS>(a, o, ta, to);
        const K diff = a ^ o;
        if (diff == 0) {  // one repeated key (or an empty unit): the values stay in input order
            const K val = decode_key(a, wk.codec);
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) {
                if ((vmask >> j) & 1u) {
                    const uint64_t i = cur.start + static_cast<uint64_t>((warp * cit + j) * 32 + lane);
                    out[i] = val;
                    kv_out<V>(wk, i, v[j]);
                }
            }
            if (un_next < nu) {
                un = fetch(un_next);
                it = static_cast<int>((un.len + THREADS - 1) / THREADS);
                vmask = kv_load<K, V, ITEMS>(wk, un.src, un.raw, un.start, un.len, it, k, v);
            }
            continue;
        }
        const int lo = lsb_pos<K>(diff);
        const int hi = msb_pos<K>(diff) + 1;
        if constexpr (sizeof(K) == 8) {
            // Stable passes of at most 8 bits over the bits [from, to), least
            // significant first; the unit ends staged in shared memory in that
            // order.  Many varying bits (8-byte keys): the passes cover the top
            // 16 only; the keys that still tie there form short runs in input
            // order, each sorted in place by the whole key (insertion sort:
            // stable) by the thread that finds its start.  A run longer than
            // kKvTieRun sends the unit through the passes of the low bits and
            // then the top bits again, from this order (still stable: equal keys
            // keep their order).
            const bool wide = hi - lo > kKvWideBits;
            const int top = wide ? hi - 16 : lo;
            int from = top, to = hi;
            bool reload = false;  // the registers are stale: the unit is staged
            for (int step = 0;; ++step) {
                const int passes = (to - from + kRadixBits - 1) / kRadixBits;
                const int width = (to - from + passes - 1) / passes;
                for (int ps = 0; ps < passes; ++ps) {
                    if (ps > 0 || reload) {  // back to registers in tile order
#pragma unroll
                        for (int j = 0; j < ITEMS; ++j) {
                            const int idx = (warp * cit + j) * 32 + lane;
                            if ((vmask >> j) & 1u) {
                                k[j] = sm_keys[idx];
                                v[j] = sm_vals[idx];
                            }
                        }
                    }
                    const int sh = from + ps * width;
                    const uint32_t m = (1u << min(width, to - sh)) - 1u;
                    uint32_t cnt;
                    stable_rank_place<K, V, THREADS, ITEMS, RS>(k, v, vmask, sh, m, set, cnt, sm_keys,
                                                                  sm_vals);
                    set ^= 1;
                    __syncthreads();
                }
                if (!wide || step == 2) break;
                reload = true;
                if (step == 1) {  // the low bits are done: the top bits again
                    from = top;
                    to = hi;
                    continue;
                }
                uint32_t longest = 0;
                for (int i = t; i < len; i += THREADS) {
                    const K ki = sm_keys[i];
                    if (i > 0 && ((sm_keys[i - 1] ^ ki) >> top) == 0) continue;  // inside a run
                    int e = i + 1;
                    while (e < len && e - i <= kKvTieRun && ((sm_keys[e] ^ ki) >> top) == 0) ++e;
                    const uint32_t run = static_cast<uint32_t>(e - i);
                    longest = max(longest, run);
                    if (run >= 2 && run <= static_cast<uint32_t>(kKvTieRun)) {
                        for (int x = i + 1; x < e; ++x) {
                            const K kx = sm_keys[x];
                            const V vx = sm_vals[x];
                            int y = x - 1;
                            while (y >= i && sm_keys[y] > kx) {
                                sm_keys[y + 1] = sm_keys[y];
                                sm_vals[y + 1] = sm_vals[y];
                                --y;
                            }
                            sm_keys[y + 1] = kx;
                            sm_vals[y + 1] = vx;
                        }
                    }
                }
                if (block_reduce_max<THREADS>(longest, RS::scan()) <= static_cast<uint32_t>(kKvTieRun)) break;
                from = lo;  // a long run: every pass, the low bits first
                to = top;
            }
        } else {
            // 4-byte keys: stable passes of at most 8 bits over the varying bits,
            // least significant first; the unit ends staged in shared memory.
            const int passes = (hi - lo + kRadixBits - 1) / kRadixBits;
            const int width = (hi - lo + passes - 1) / passes;
            for (int ps = 0; ps < passes; ++ps) {
                const int sh = lo + ps * width;
                const uint32_t m = (1u << min(width, hi - sh)) - 1u;
                uint32_t cnt;
                stable_rank_place<K, V, THREADS, ITEMS, RS>(k, v, vmask, sh, m, set, cnt, sm_keys,
                                                              sm_vals);
                set ^= 1;
                __syncthreads();
                if (ps + 1 < passes) {  // back to registers in tile order for the next pass
#pragma unroll
                    for (int j = 0; j < ITEMS; ++j) {
                        const int idx = (warp * cit + j) * 32 + lane;
                        if ((vmask >> j) & 1u) {
                            k[j] = sm_keys[idx];
                            v[j] = sm_vals[idx];
                        }
                    }
                }
            }
        }
        if (un_next < nu) {  // next unit into the registers; its loads overlap the write-out
            un = fetch(un_next);
            it = static_cast<int>((un.len + THREADS - 1) / THREADS);
            vmask = kv_load<K, V, ITEMS>(wk, un.src, un.raw, un.start, un.len, it, k, v);
        }
        for (int i = t; i < len; i += THREADS) {
            out[cur.start + i] = decode_key(sm_keys[i], wk.codec);
            kv_out<V>(wk, cur.start + i, sm_vals[i]);
        }
        // (the next unit stages only after the barriers of its AND/OR and ranking)
    }
}

// Constant runs of the key-value sort: the key written len times, the run's
// values moved, in their order, to the output (src 1: from the alternate
// values; 0: already in place unless they are argsort positions; 2: a run
// never moved, its values the input's).  Four elements per thread in flight.
template <typename K, typename V>
__global__ void __launch_bounds__(256) k_fill_kv(Work wk) {
    pdl_enter();
    constexpr int U = 4;
    if (wk.ctl->error) return;
    const uint32_t nf = wk.ctl->n_fills;
    K *out = static_cast<K *>(wk.keys);
    for (uint32_t f = blockIdx.x; f < nf; f += gridDim.x) {
        const Fill fl = wk.fills[f];
        if (fl.start + fl.len > wk.n) {
            if (threadIdx.x == 0) set_error(wk.ctl, kErrBounds);
            continue;
        }
        K val = static_cast<K>(fl.value);
        if constexpr (sizeof(K) > 8) val |= static_cast<K>(fl.value_hi) << 64;
        const K key = decode_key(val, wk.codec);
        const bool move = fl.src == 1 || (fl.src == 0 && wk.kv_positions);
        const bool make = fl.src == 2 && wk.kv_positions;
        const V *__restrict__ vsrc = vals_of<V>(wk, fl.src == 1 ? 1 : 0);
        for (uint32_t i0 = threadIdx.x; i0 < fl.len; i0 += U * blockDim.x) {
            V x[U];
#pragma unroll
            for (int e = 0; e < U; ++e) {
                const uint32_t i = i0 + e * blockDim.x;
                x[e] = (move && i < fl.len) ? vsrc[fl.start + i] : static_cast<V>(fl.start + i);
            }
#pragma unroll
            for (int e = 0; e < U; ++e) {
                const uint32_t i = i0 + e * blockDim.x;
                if (i < fl.len) {
                    out[fl.start + i] = key;
                    if (move || make) kv_out<V>(wk, fl.start + i, x[e]);
                }
            }
        }
    }
}

template <typename K>
struct Cfg;
template <>
struct Cfg<uint32_t> {
    static constexpr int kThreads = 512;  // scatter tile: 512 x 16 = 8192 keys
    static constexpr int kItems = 16;
    static constexpr int kFinThreads = 256;  // finish tile: 256 x 20 = 5120 keys, 4 CTAs per SM
    static constexpr int kFinItems = 20;
};
template <>
struct Cfg<uint64_t> {
    static constexpr int kThreads = 512;  // 512 x 8 = 4096 keys
    static constexpr int kItems = 8;
    static constexpr int kFinThreads = 256;  // 256 x 10 = 2560 keys
    static constexpr int kFinItems = 10;
};
template <>
struct Cfg<u128> {
    static constexpr int kThreads = 512;  // 512 x 4 = 2048 keys
    static constexpr int kItems = 4;
    static constexpr int kFinThreads = 256;  // 256 x 5 = 1280 keys
    static constexpr int kFinItems = 5;
};

constexpr uint64_t kKvBigChild = 2600;

// Key-value sorting: 256-thread CTAs; the scatter tile is 4096 pairs (a
// chunk is kKvChunkTiles of them), the finish tile holds the largest unit.
template <typename K, typename V>
struct KvCfg {
    static constexpr int kPairBytes = static_cast<int>(sizeof(K) + sizeof(V));
    static constexpr int kThreads = 256;
    static constexpr int kItems = 16;
    static constexpr int kScatterCtas = 2;
    static constexpr int kFinThreads = 256;
    static constexpr int kFinItems = kPairBytes <= 8 ? 20 : (kPairBytes <= 12 ? 12 : 10);
    static constexpr int kFinCtas = 3;
    // 4-byte keys with 8-byte values, large arrays: a 5120-pair finish (96 KB
    // of shared memory, two CTAs per SM), so that level-1 children of ~4096
    // pairs finish without a third scatter level; chosen when the average
    // level-1 child passes kKvBigChild pairs (smaller arrays keep the
    // 3072-pair finish at three CTAs per SM)
    static constexpr bool kHasBig = sizeof(K) == 4 && sizeof(V) == 8;
    static constexpr int kFinItemsBig = 20;
    static constexpr int kFinCtasBig = 2;
};

}  // namespace

MsdShape msd_shape(int key_bytes, const Tuning &t, bool inplace, int kv_bytes, uint64_t n) {
    MsdShape s;
    uint32_t fin;
    if (kv_bytes) {  // key-value sorting: fixed shape, 8-bit digits, one scatter tile per chunk
        const bool k4 = key_bytes == 4, v4 = kv_bytes == 4;
        s.tile = k4 ? (v4 ? KvCfg<uint32_t, uint32_t>::kThreads * KvCfg<uint32_t, uint32_t>::kItems
                          : KvCfg<uint32_t, uint64_t>::kThreads * KvCfg<uint32_t, uint64_t>::kItems)
                    : (v4 ? KvCfg<uint64_t, uint32_t>::kThreads * KvCfg<uint64_t, uint32_t>::kItems
                          : KvCfg<uint64_t, uint64_t>::kThreads * KvCfg<uint64_t, uint64_t>::kItems);
        fin = k4 ? (v4 ? KvCfg<uint32_t, uint32_t>::kFinThreads * KvCfg<uint32_t, uint32_t>::kFinItems
                       : KvCfg<uint32_t, uint64_t>::kFinThreads * KvCfg<uint32_t, uint64_t>::kFinItems)
                 : (v4 ? KvCfg<uint64_t, uint32_t>::kFinThreads * KvCfg<uint64_t, uint32_t>::kFinItems
                       : KvCfg<uint64_t, uint64_t>::kFinThreads * KvCfg<uint64_t, uint64_t>::kFinItems);
        if (k4 && !v4 && n / (1u << (2 * kRadixBits)) > kKvBigChild)
            fin = KvCfg<uint32_t, uint64_t>::kFinThreads * KvCfg<uint32_t, uint64_t>::kFinItemsBig;
        s.radix_bits = kRadixBits;
        s.bins = kBins;
        s.levels = (key_bytes * 8 + kRadixBits - 1) / kRadixBits;
        s.chunk = s.tile * kKvChunkTiles;
        s.unit_cap = fin;  // the finish loads a unit with scalar loads: no alignment slack
        s.merge_cap = (s.unit_cap * 4 / 5) & ~63u;
        return s;
    }
    if (key_bytes == 4) {
        s.tile = Cfg<uint32_t>::kThreads * Cfg<uint32_t>::kItems;
        fin = Cfg<uint32_t>::kFinThreads * Cfg<uint32_t>::kFinItems;
    } else if (key_bytes == 16) {
        s.tile = Cfg<u128>::kThreads * Cfg<u128>::kItems;
        fin = Cfg<u128>::kFinThreads * Cfg<u128>::kFinItems;
    } else {
        s.tile = Cfg<uint64_t>::kThreads * Cfg<uint64_t>::kItems;
        fin = Cfg<uint64_t>::kFinThreads * Cfg<uint64_t>::kFinItems;
    }
    s.radix_bits = t.radix_bits ? t.radix_bits : kRadixBits;
    if (inplace && s.radix_bits > kRadixBits) s.radix_bits = kRadixBits;  // the permutation's tables are 8-bit
    s.bins = s.radix_bits > kRadixBits ? kWideBins : kBins;
    s.levels = (key_bytes * 8 + s.radix_bits - 1) / s.radix_bits;
    s.chunk = (t.chunk_tiles ? t.chunk_tiles : kMaxChunkTiles) * s.tile;
    // a unit plus its misalignment fits one aligned finish window
    s.unit_cap = t.unit_keys ? static_cast<uint32_t>(t.unit_keys) : fin - 16;
    // tiny buckets (<= merge_cap / 4) group below 1.25 * merge_cap <= unit_cap
    s.merge_cap = t.merge_keys ? static_cast<uint32_t>(t.merge_keys) : (s.unit_cap * 4 / 5) & ~63u;
    return s;
}

bool tuning_valid(int key_bytes, const Tuning &t) {
    const MsdShape d = msd_shape(key_bytes);
    if (t.radix_bits && (t.radix_bits < kMinRadixBits || t.radix_bits > kMaxRadixBits)) return false;
    if (t.chunk_tiles < 0 || t.chunk_tiles > kMaxChunkTiles) return false;
    if (t.unit_keys && (t.unit_keys < 256 || static_cast<uint32_t>(t.unit_keys) > d.unit_cap)) return false;
    const uint32_t unit = t.unit_keys ? static_cast<uint32_t>(t.unit_keys) : d.unit_cap;
    if (t.merge_keys && (t.merge_keys < 64 || 5ull * static_cast<uint32_t>(t.merge_keys) > 4ull * unit)) return false;
    return true;
}

// Launches `kern` on `st` with programmatic stream serialization (the
// kernel calls pdl_enter() before touching memory).
template <typename... P, typename... A>
void launch_pdl(void (*kern)(P...), unsigned grid, unsigned block, size_t smem, cudaStream_t st, A... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kern, static_cast<P>(args)...);
}

template <typename K>
void msd_prepare() {
    constexpr int T = Cfg<K>::kThreads, I = Cfg<K>::kItems, CT = kMaxChunkTiles;
    constexpr int FT = Cfg<K>::kFinThreads, FI = Cfg<K>::kFinItems;
    if constexpr (sizeof(K) <= 8) ip_prepare<K>();  // the in-place mode takes keys of up to 8 bytes
    static const bool attrs = [] {  // once per process; thread-safe static initialisation
        cudaFuncSetAttribute(k_scatter<K, T, I, CT, kBins>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(scatter_smem<K, T, I, CT, kBins>()));
        cudaFuncSetAttribute(k_scatter<K, T, I, CT, kWideBins>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(scatter_smem<K, T, I, CT, kWideBins>()));
        cudaFuncSetAttribute(k_finish<K, FT, FI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(finish_smem<K, FT, FI>()));
        cudaFuncSetAttribute(k_finish_lsd<K, FT, FI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(finish_lsd_smem<K, FT, FI>()));
        return true;
    }();
    (void)attrs;
}

// The MSD levels, the finish and the fills, after the level-0 lists exist.
template <typename K>
void msd_levels_and_finish(const Work &wk, cudaStream_t st, Recorder &rec, int num_sms, bool levels) {
    constexpr int T = Cfg<K>::kThreads, I = Cfg<K>::kItems;
    constexpr int FT = Cfg<K>::kFinThreads, FI = Cfg<K>::kFinItems;
    constexpr int CT = kMaxChunkTiles;  // staging capacity in tiles (a chunk holds 1 or 2)
    const bool wide = wk.bins > static_cast<uint32_t>(kBins);
    if (levels) {
        for (int level = 0; level < wk.stop_level; ++level) {
            rec.begin(BSORT_K_HIST, level);
            if (wide) launch_pdl(k_hist<K, 512, kWideBins>, num_sms * 4, 512, 0, st, wk, level);
            else launch_pdl(k_hist<K, 512, kBins>, num_sms * 4, 512, 0, st, wk, level);
            rec.end();
            rec.begin(BSORT_K_SCAN, level);
            launch_pdl(k_colscan<1024>, 1u << wk.radix_bits, 1024, 0, st, wk, level);
            rec.end();
            rec.begin(BSORT_K_CLASSIFY, level);
            launch_pdl(k_classify<kBins, K>, num_sms * 4, kBins, 0, st, wk, level);
            rec.end();
            if (wk.inplace) {
                if constexpr (sizeof(K) <= 8) launch_ip_level<K>(wk, st, rec, num_sms, level);
            } else {
                rec.begin(BSORT_K_SCATTER, level);
                if (wide)
                    launch_pdl(k_scatter<K, T, I, CT, kWideBins>, num_sms * 2, T, scatter_smem<K, T, I, CT, kWideBins>(),
                               st, wk, level);
                else
                    launch_pdl(k_scatter<K, T, I, CT, kBins>, num_sms * 2, T, scatter_smem<K, T, I, CT, kBins>(), st, wk, level);
                rec.end();
            }
        }
    }
    if (levels && wk.stop_level < wk.levels) {
        rec.begin(BSORT_K_FILL, wk.stop_level);
        launch_pdl(k_drain<K>, num_sms * 2, 256, 0, st, wk, wk.stop_level);
        rec.end();
    }
    rec.begin(BSORT_K_FINISH, -1);
    launch_pdl(k_finish<K, FT, FI>, num_sms * 8, FT, finish_smem<K, FT, FI>(), st, wk);
    launch_pdl(k_finish_lsd<K, FT, FI>, num_sms * 4, FT, finish_lsd_smem<K, FT, FI>(), st, wk);
    rec.more(1);
    rec.end();
    if (levels) {
        rec.begin(BSORT_K_FILL, -1);
        launch_pdl(k_fill<K>, num_sms * 2, 256, 0, st, wk);
        rec.end();
    }
}

template <typename K>
void launch_msd(const Work &wk, cudaStream_t st, Recorder &rec, int num_sms) {
    msd_prepare<K>();
    const bool direct = wk.n <= wk.unit_cap;
    const uint32_t nc0 = direct ? 0u : static_cast<uint32_t>((wk.n + wk.chunk_keys - 1) / wk.chunk_keys);
    rec.begin(BSORT_K_INIT, -1);
    k_init<<<direct ? 1 : max(1u, min(1024u, (nc0 + 255) / 256)), 256, 0, st>>>(wk, nc0, direct ? 1 : 0);
    rec.end();
    msd_levels_and_finish<K>(wk, st, rec, num_sms, !direct);
}

template <typename K>
void launch_msd_segmented(const Work &wk, const uint64_t *d_offsets, uint32_t nseg, cudaStream_t st, Recorder &rec,
                          int num_sms) {
    msd_prepare<K>();
    rec.begin(BSORT_K_INIT, -1);
    k_zero_ctl<<<1, 256, 0, st>>>(wk);
    k_seg_init<<<max(1u, min(static_cast<uint32_t>(num_sms) * 4, (nseg + 255) / 256)), 256, 0, st>>>(wk, d_offsets,
                                                                                                      nseg);
    rec.more(1);
    rec.end();
    msd_levels_and_finish<K>(wk, st, rec, num_sms, true);
}

// Stable key-value sort: the keys-only histogram, column scan and classify
// steps, the value-carrying scatter per level, then the stable finish and the
// fills.
template <typename K, typename V>
void launch_msd_kv(const Work &wk, cudaStream_t st, Recorder &rec, int num_sms) {
    using C = KvCfg<K, V>;
    constexpr int T = C::kThreads, I = C::kItems, SB = C::kScatterCtas;
    constexpr int FT = C::kFinThreads, FI = C::kFinItems, FB = C::kFinCtas;
    constexpr int FIB = C::kFinItemsBig, FBB = C::kFinCtasBig;
    constexpr size_t kScatterSmem = ScatterKvSmem<K, V, T, I>::kEnd;
    constexpr size_t kFinishSmem = FinishKvSmem<K, V, FT, FI>::kEnd;
    constexpr size_t kFinishSmemBig = FinishKvSmem<K, V, FT, FIB>::kEnd;
    static const bool attrs = [] {  // once per process
        cudaFuncSetAttribute(k_scatter_kv<K, V, T, I, SB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(kScatterSmem));
        cudaFuncSetAttribute(k_finish_kv<K, V, FT, FI, FB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(kFinishSmem));
        if constexpr (C::kHasBig)
            cudaFuncSetAttribute(k_finish_kv<K, V, FT, FIB, FBB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(kFinishSmemBig));
        return true;
    }();
    (void)attrs;
    // the finish whose tile the shape's unit capacity was sized for
    const bool big = C::kHasBig && wk.unit_cap > static_cast<uint32_t>(FT * FI);
    const bool direct = wk.n <= wk.unit_cap;
    const uint32_t nc0 = direct ? 0u : static_cast<uint32_t>((wk.n + wk.chunk_keys - 1) / wk.chunk_keys);
    rec.begin(BSORT_K_INIT, -1);
    k_init<<<direct ? 1 : max(1u, min(1024u, (nc0 + 255) / 256)), 256, 0, st>>>(wk, nc0, direct ? 1 : 0);
    rec.end();
    if (!direct) {
        for (int level = 0; level < wk.levels; ++level) {
            rec.begin(BSORT_K_HIST, level);
            launch_pdl(k_hist<K, 512, kBins>, num_sms * 4, 512, 0, st, wk, level);
            rec.end();
            rec.begin(BSORT_K_SCAN, level);
            launch_pdl(k_colscan<1024>, kBins, 1024, 0, st, wk, level);
            rec.end();
            rec.begin(BSORT_K_CLASSIFY, level);
            launch_pdl(k_classify<kBins, K>, num_sms * 4, kBins, 0, st, wk, level);
            rec.end();
            rec.begin(BSORT_K_SCATTER, level);
            launch_pdl(k_scatter_kv<K, V, T, I, SB>, num_sms * SB, T, kScatterSmem, st, wk, level);
            rec.end();
        }
    }
    rec.begin(BSORT_K_FINISH, -1);
    if (big) {
        if constexpr (C::kHasBig)
            launch_pdl(k_finish_kv<K, V, FT, FIB, FBB>, num_sms * FBB, FT, kFinishSmemBig, st, wk);
    } else {
        launch_pdl(k_finish_kv<K, V, FT, FI, FB>, num_sms * FB, FT, kFinishSmem, st, wk);
    }
    rec.end();
    if (!direct) {
        rec.begin(BSORT_K_FILL, -1);
        launch_pdl(k_fill_kv<K, V>, num_sms * 4, 256, 0, st, wk);
        rec.end();
    }
}

template void launch_msd_kv<uint32_t, uint32_t>(const Work &, cudaStream_t, Recorder &, int);
template void launch_msd_kv<uint32_t, uint64_t>(const Work &, cudaStream_t, Recorder &, int);
template void launch_msd_kv<uint64_t, uint32_t>(const Work &, cudaStream_t, Recorder &, int);
template void launch_msd_kv<uint64_t, uint64_t>(const Work &, cudaStream_t, Recorder &, int);
template void msd_prepare<uint32_t>();
template void msd_prepare<uint64_t>();
template void msd_prepare<u128>();
template void launch_msd_segmented<u128>(const Work &, const uint64_t *, uint32_t, cudaStream_t, Recorder &, int);
template void launch_msd<u128>(const Work &, cudaStream_t, Recorder &, int);
template void launch_msd_segmented<uint32_t>(const Work &, const uint64_t *, uint32_t, cudaStream_t, Recorder &, int);
template void launch_msd_segmented<uint64_t>(const Work &, const uint64_t *, uint32_t, cudaStream_t, Recorder &, int);
template void launch_msd<uint32_t>(const Work &, cudaStream_t, Recorder &, int);
template void launch_msd<uint64_t>(const Work &, cudaStream_t, Recorder &, int);

}  // namespace bsort
