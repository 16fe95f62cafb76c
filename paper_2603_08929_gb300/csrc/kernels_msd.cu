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

// Stable rank of a tile held in registers, warp-striped: item j of lane l in
// warp w has tile index w*32*ITEMS + j*32 + l, and items with index >= n_valid
// take no part.  Each warp counts its digits in its own shared-memory row
// (match-any groups equal digits inside a warp step, so skewed tiles cost no
// more than uniform ones); the rows are then scanned per digit across warps
// and across digits.  The valid keys land in `out` in digit order, equal
// digits in tile order; dstart/dcount describe the digit runs.
template <typename K, int THREADS, int ITEMS>
struct Ranker {
    static constexpr int WARPS = THREADS / 32;
    static constexpr int TILE = THREADS * ITEMS;
    struct Smem {
        uint16_t warp_cnt[WARPS * kBins];  // per-warp digit counts (<= 32 * ITEMS), then prefixes (< TILE)
        uint32_t dstart[kBins];
        uint32_t dcount[kBins];
        uint32_t scan_tmp[WARPS + 1];
    };

    __device__ static void rank_and_place(const K (&keys)[ITEMS], int n_valid, int shift, uint32_t mask, Smem &s,
                                          K *out) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        uint16_t *wc = s.warp_cnt + warp * kBins;
        for (int i = lane; i <= static_cast<int>(mask); i += 32) wc[i] = 0;
        __syncwarp();
        const unsigned lt = lanemask_lt();
        const int wbase = warp * 32 * ITEMS;
        uint32_t local[ITEMS];
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            const int base = wbase + j * 32;
            local[j] = 0;
            if (base < n_valid) {  // warp-uniform
                const bool valid = base + lane < n_valid;
                const unsigned act = __ballot_sync(kFull, valid);
                if (valid) {
                    const uint32_t d = static_cast<uint32_t>(keys[j] >> shift) & mask;
                    const unsigned peers = __match_any_sync(act, d);
                    const uint32_t before = wc[d];
                    const uint32_t r = __popc(peers & lt);
                    local[j] = before + r;
                    __syncwarp(act);
                    if (r == 0) wc[d] = static_cast<uint16_t>(before + __popc(peers));
                }
                __syncwarp();
            }
        }
        __syncthreads();
        // per digit: exclusive prefix over warps, digit totals
        for (int d = threadIdx.x; d <= static_cast<int>(mask); d += THREADS) {
            uint32_t run = 0;
#pragma unroll 4
            for (int w = 0; w < WARPS; ++w) {
                const uint32_t c = s.warp_cnt[w * kBins + d];
                s.warp_cnt[w * kBins + d] = static_cast<uint16_t>(run);
                run += c;
            }
            s.dcount[d] = run;
        }
        __syncthreads();
        uint32_t total;
        const uint32_t v = threadIdx.x <= mask ? s.dcount[threadIdx.x] : 0;
        const uint32_t ex = block_exclusive_scan<THREADS>(v, s.scan_tmp, total);
        if (threadIdx.x <= mask) s.dstart[threadIdx.x] = ex;
        __syncthreads();
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            if (wbase + j * 32 + lane < n_valid) {
                const uint32_t d = static_cast<uint32_t>(keys[j] >> shift) & mask;
                out[s.dstart[d] + s.warp_cnt[warp * kBins + d] + local[j]] = keys[j];
            }
        }
        __syncthreads();
    }
};

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
            u.pad[0] = u.pad[1] = 0;
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

// Per-chunk digit histogram (one shared-memory row per warp) and AND/OR.
template <typename K, int THREADS>
__global__ void __launch_bounds__(THREADS) k_hist(Work wk, int level) {
    constexpr int WARPS = THREADS / 32;
    constexpr int U = 8;
    __shared__ uint32_t sh[WARPS * kBins];
    __shared__ unsigned long long ta[WARPS], to[WARPS];
    const int p = level & 1;
    if (wk.ctl->error) return;  // an earlier launch found a problem: stop touching memory
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        wk.ctl->n_buckets[p ^ 1] = 0;
        wk.ctl->n_chunks[p ^ 1] = 0;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t nch = wk.ctl->n_chunks[p];
    for (uint32_t c = blockIdx.x; c < nch; c += gridDim.x) {
        const Chunk ch = wk.chunks[p][c];
        const Bucket b = wk.buckets[p][ch.bucket];
        const int r_eff = min(kRadixBits, b.h);
        const int shift = b.h - r_eff;
        const uint32_t mask = (1u << r_eff) - 1;
        for (int i = threadIdx.x; i < WARPS * kBins; i += THREADS) sh[i] = 0;
        __syncthreads();
        uint32_t *my = sh + warp * kBins;
        K a = static_cast<K>(~K(0)), o = 0;
        const K *s = src_of<K>(wk, b.src) + ch.start;
        const uint32_t len = ch.len;
        const bool raw = b.raw;
        for (uint32_t base = 0; base < len; base += THREADS * U) {
            K kk[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint32_t i = base + u * THREADS + threadIdx.x;
                kk[u] = i < len ? s[i] : K(0);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint32_t i = base + u * THREADS + threadIdx.x;
                const bool valid = i < len;
                K key = kk[u];
                if (raw) key = encode_key(key, wk.codec);
                const uint32_t d = valid ? (static_cast<uint32_t>(key >> shift) & mask) : 0xffffffffu;
                if (valid) {
                    a &= key;
                    o |= key;
                }
                const uint32_t d0 = __shfl_sync(kFull, d, 0);
                if (__all_sync(kFull, d == d0)) {
                    if (lane == 0 && d0 != 0xffffffffu) atomicAdd(&my[d0], 32u);
                } else if (valid) {
                    atomicAdd(&my[d], 1u);
                }
            }
        }
        __syncthreads();
        for (int d = threadIdx.x; d < kBins; d += THREADS) {
            uint32_t sum = 0;
#pragma unroll
            for (int w = 0; w < WARPS; ++w) sum += sh[w * kBins + d];
            wk.hist[static_cast<size_t>(d) * wk.max_chunks + c] = sum;
        }
        unsigned long long aa = a, oo = o;
        block_and_or<THREADS>(aa, oo, ta, to);
        if (threadIdx.x == 0) {
            wk.chunk_and[c] = aa;
            wk.chunk_or[c] = oo;
        }
        __syncthreads();
    }
}

// Per digit d: exclusive prefix of hist[d][c] over the chunks of each bucket
// (in place), and the bucket's digit total into bucket_base[bucket][d].
template <int THREADS>
__global__ void __launch_bounds__(THREADS) k_colscan(Work wk, int level) {
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
    for (uint32_t base = 0; base < nch; base += THREADS) {
        const uint32_t c = base + threadIdx.x;
        const bool in = c < nch;
        const uint32_t b = in ? chunks[c].bucket : 0xffffffffu;
        const uint32_t v = in ? col[c] : 0;
        const bool head = in && (c == 0 || chunks[c - 1].bucket != b);
        const bool last = in && (c + 1 == nch || chunks[c + 1].bucket != b);
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
            if (last) wk.bucket_base[static_cast<size_t>(b) * kBins + d] = static_cast<unsigned long long>(out) + v;
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
                             uint32_t *tmp, uint32_t *sh_choff, uint32_t *sh_slot, uint32_t *sh_bases) {
    const uint32_t nchunks = take ? static_cast<uint32_t>((len + wk.chunk_keys - 1) / wk.chunk_keys) : 0;
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
    sh_choff[threadIdx.x] = ch_off;
    sh_slot[threadIdx.x] = take ? slot_off : 0xffffffffu;
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
        // chunk records: k-th chunk of this parent belongs to the child whose
        // [choff, choff + nchunks) contains k
        for (uint32_t k = threadIdx.x; k < nc_total; k += THREADS) {
            int lo = 0, hi = THREADS - 1;  // largest d with choff[d] <= k and a bucket
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (sh_choff[mid] <= k) lo = mid;
                else hi = mid - 1;
            }
            // children without chunks never satisfy choff <= k past the owner
            const int d = lo;
            const Bucket &nbk = wk.buckets[q][b0 + sh_slot[d]];
            const uint32_t i = k - sh_choff[d];
            Chunk ch;
            ch.start = nbk.start + static_cast<uint64_t>(i) * wk.chunk_keys;
            const uint64_t rem = nbk.len - static_cast<uint64_t>(i) * wk.chunk_keys;
            ch.len = static_cast<uint32_t>(rem < wk.chunk_keys ? rem : wk.chunk_keys);
            ch.bucket = b0 + sh_slot[d];
            wk.chunks[q][c0 + k] = ch;
        }
    }
    __syncthreads();
}

// Fill pieces for every thread whose `take` is set (thread-private loop).
__device__ void emit_fill(const Work &wk, uint64_t start, uint64_t len, uint64_t value) {
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
        f.value = value;
        f.pad = 0;
        wk.fills[f0 + i] = f;
    }
}

__device__ void emit_unit(const Work &wk, uint64_t start, uint32_t len, int src) {
    const uint32_t u = atomicAdd(&wk.ctl->n_units, 1u);
    if (u >= wk.max_units) {
        set_error(wk.ctl, kErrCapacity);
        return;
    }
    atomicAdd(&wk.ctl->finish_keys, static_cast<unsigned long long>(len));
    Unit un;
    un.start = start;
    un.len = len;
    un.src = static_cast<uint8_t>(src);
    un.raw = 0;
    un.pad[0] = un.pad[1] = 0;
    wk.units[u] = un;
}

// Per bucket of this level: common-prefix test, digit bases, child classes.
template <int THREADS>
__global__ void __launch_bounds__(THREADS) k_classify(Work wk, int level) {
    static_assert(THREADS == kBins, "one thread per digit");
    __shared__ unsigned long long ta[THREADS / 32], to[THREADS / 32];
    __shared__ unsigned long long tmp64[THREADS / 32 + 1];
    __shared__ uint32_t tmp[THREADS / 32 + 1];
    __shared__ uint32_t sh_choff[THREADS], sh_slot[THREADS], sh_bases[2];
    __shared__ unsigned long long sh_len[THREADS], sh_base[THREADS];
    const int p = level & 1, q = p ^ 1;
    if (wk.ctl->error) return;
    const uint32_t nb = wk.ctl->n_buckets[p];
    const int d = threadIdx.x;
    for (uint32_t i = blockIdx.x; i < nb; i += gridDim.x) {
        const Bucket b = wk.buckets[p][i];
        unsigned long long a = ~0ull, o = 0;
        for (uint32_t c = b.first_chunk + threadIdx.x; c < b.first_chunk + b.num_chunks; c += THREADS) {
            a &= wk.chunk_and[c];
            o |= wk.chunk_or[c];
        }
        block_and_or<THREADS>(a, o, ta, to);
        if (threadIdx.x == 0) atomicAdd(&wk.ctl->hist_keys[level], static_cast<unsigned long long>(b.len));
        if (a == o) {  // every key identical: write the value, no sort needed
            if (threadIdx.x == 0) {
                wk.buckets[p][i].scatter = 0;
                emit_fill(wk, b.start, b.len, a);
            }
            continue;
        }
        const int r_eff = min(kRadixBits, b.h);
        const int shift = b.h - r_eff;
        const uint32_t mask = (1u << r_eff) - 1;
        const int hb = 63 - __clzll(a ^ o);
        if (hb < shift) {
            // the digit is constant: re-open the bucket at its highest varying bit
            if (threadIdx.x == 0) wk.buckets[p][i].scatter = 0;
            emit_buckets<THREADS>(wk, q, threadIdx.x == 0, b.start, b.len, hb + 1, b.src, b.raw, tmp, sh_choff,
                                  sh_slot, sh_bases);
            continue;
        }
        const unsigned long long tot =
            static_cast<uint32_t>(d) <= mask ? wk.bucket_base[static_cast<size_t>(i) * kBins + d] : 0ull;
        unsigned long long total;
        const unsigned long long ex = block_exclusive_scan64<THREADS>(tot, tmp64, total);
        const unsigned long long base = b.start + ex;
        if (static_cast<uint32_t>(d) <= mask) wk.bucket_base[static_cast<size_t>(i) * kBins + d] = base;
        if (threadIdx.x == 0) {
            wk.buckets[p][i].scatter = 1;
            atomicAdd(&wk.ctl->scatter_keys[level], static_cast<unsigned long long>(b.len));
        }
        sh_len[d] = tot;
        sh_base[d] = base;
        const int hc = shift;  // bits left in the children
        const int dst = b.src ^ 1;
        const bool big = tot > wk.unit_cap;
        // children with no bits left are constant: value = common prefix | digit
        if (big && hc == 0) {
            const unsigned long long hi_mask = b.h >= 64 ? 0ull : (~0ull << b.h);
            emit_fill(wk, base, tot, (a & hi_mask) | static_cast<unsigned long long>(d));
        }
        emit_buckets<THREADS>(wk, q, big && hc > 0, base, tot, hc, dst, 0, tmp, sh_choff, sh_slot, sh_bases);
        // small children: adjacent ones merge into units up to merge_cap keys
        if (threadIdx.x == 0) {
            unsigned long long run_start = 0;
            uint32_t run_len = 0;
            for (uint32_t e = 0; e <= mask; ++e) {
                const unsigned long long len = sh_len[e];
                if (len == 0) continue;
                if (len > wk.unit_cap) {
                    if (run_len) emit_unit(wk, run_start, run_len, dst);
                    run_len = 0;
                    continue;
                }
                if (run_len && run_len + len <= wk.merge_cap) {
                    run_len += static_cast<uint32_t>(len);
                } else {
                    if (run_len) emit_unit(wk, run_start, run_len, dst);
                    run_start = sh_base[e];
                    run_len = static_cast<uint32_t>(len);
                }
            }
            if (run_len) emit_unit(wk, run_start, run_len, dst);
        }
        __syncthreads();
    }
}

// Stable shared-memory digit ranking of each tile, then coalesced runs to
// the digit offsets of the chunk.
template <typename K, int THREADS, int ITEMS>
__global__ void __launch_bounds__(THREADS, 2) k_scatter(Work wk, int level) {
    using R = Ranker<K, THREADS, ITEMS>;
    constexpr int TILE = R::TILE;
    __shared__ typename R::Smem rs;
    __shared__ K sm_keys[TILE];
    __shared__ unsigned long long off[kBins];
    const int p = level & 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (wk.ctl->error) return;
    const uint32_t nch = wk.ctl->n_chunks[p];
    for (uint32_t c = blockIdx.x; c < nch; c += gridDim.x) {
        const Chunk ch = wk.chunks[p][c];
        const Bucket b = wk.buckets[p][ch.bucket];
        if (!b.scatter) continue;  // block-uniform
        const uint64_t lo_pos = b.start, hi_pos = b.start + b.len;
        const K *src = src_of<K>(wk, b.src);
        K *dst = dst_of<K>(wk, b.src);
        const int r_eff = min(kRadixBits, b.h);
        const int shift = b.h - r_eff;
        const uint32_t mask = (1u << r_eff) - 1;
        for (int d = threadIdx.x; d <= static_cast<int>(mask); d += THREADS)
            off[d] = wk.bucket_base[static_cast<size_t>(ch.bucket) * kBins + d] +
                     wk.hist[static_cast<size_t>(d) * wk.max_chunks + c];
        __syncthreads();
        for (uint32_t t0 = 0; t0 < ch.len; t0 += TILE) {
            const int nv = static_cast<int>(min(static_cast<uint32_t>(TILE), ch.len - t0));
            const K *s = src + ch.start + t0;
            K k[ITEMS];
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) {
                const int idx = warp * 32 * ITEMS + j * 32 + lane;
                k[j] = idx < nv ? s[idx] : K(0);
            }
            if (b.raw) {
#pragma unroll
                for (int j = 0; j < ITEMS; ++j) k[j] = encode_key(k[j], wk.codec);
            }
            R::rank_and_place(k, nv, shift, mask, rs, sm_keys);
            bool oob = false;
            for (int i = threadIdx.x; i < nv; i += THREADS) {
                const K key = sm_keys[i];
                const uint32_t d = static_cast<uint32_t>(key >> shift) & mask;
                const uint64_t pos = off[d] + (i - rs.dstart[d]);
                if (pos >= lo_pos && pos < hi_pos) dst[pos] = key;  // bounds check: never write outside the bucket
                else oob = true;
            }
            if (oob) set_error(wk.ctl, kErrBounds);
            __syncthreads();
            for (int d = threadIdx.x; d <= static_cast<int>(mask); d += THREADS) off[d] += rs.dcount[d];
            __syncthreads();
        }
    }
}

// Shared-memory finish of every unit: LSD passes over the unit's varying
// bits (bits above its highest varying bit are common to the whole run),
// then the decoded keys go to their final place in the caller's buffer.
template <typename K, int THREADS, int ITEMS>
__global__ void __launch_bounds__(THREADS, 2) k_finish(Work wk) {
    using R = Ranker<K, THREADS, ITEMS>;
    __shared__ typename R::Smem rs;
    __shared__ K sm_keys[R::TILE];
    __shared__ unsigned long long ta[THREADS / 32], to[THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (wk.ctl->error) return;
    const uint32_t nu = wk.ctl->n_units;
    K *out = static_cast<K *>(wk.keys);
    for (uint32_t u = blockIdx.x; u < nu; u += gridDim.x) {
        const Unit un = wk.units[u];
        const K *s = src_of<K>(wk, un.src) + un.start;
        const int len = static_cast<int>(un.len);
        K k[ITEMS];
        unsigned long long a = ~0ull, o = 0;
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            const int idx = warp * 32 * ITEMS + j * 32 + lane;
            K key = idx < len ? s[idx] : K(0);
            if (un.raw) key = encode_key(key, wk.codec);
            k[j] = key;
            if (idx < len) {
                a &= key;
                o |= key;
            }
        }
        block_and_or<THREADS>(a, o, ta, to);
        const unsigned long long v = a ^ o;
        if (v == 0) {
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) {
                const int idx = warp * 32 * ITEMS + j * 32 + lane;
                if (idx < len) out[un.start + idx] = decode_key(k[j], wk.codec);
            }
            continue;
        }
        const int lo = __ffsll(static_cast<long long>(v)) - 1;
        const int hi = 64 - __clzll(v);
        const int passes = (hi - lo + kRadixBits - 1) / kRadixBits;
        const int width = (hi - lo + passes - 1) / passes;
        for (int ps = 0, sh = lo; ps < passes; ++ps, sh += width) {
            const int bits = min(width, hi - sh);
            R::rank_and_place(k, len, sh, (1u << bits) - 1, rs, sm_keys);
            if (ps + 1 < passes) {
#pragma unroll
                for (int j = 0; j < ITEMS; ++j) {
                    const int idx = warp * 32 * ITEMS + j * 32 + lane;
                    if (idx < len) k[j] = sm_keys[idx];
                }
                __syncthreads();
            }
        }
        for (int i = threadIdx.x; i < len; i += THREADS) out[un.start + i] = decode_key(sm_keys[i], wk.codec);
        __syncthreads();
    }
}

template <typename K>
__global__ void k_fill(Work wk) {
    if (wk.ctl->error) return;
    const uint32_t nf = wk.ctl->n_fills;
    K *out = static_cast<K *>(wk.keys);
    for (uint32_t f = blockIdx.x; f < nf; f += gridDim.x) {
        const Fill fl = wk.fills[f];
        if (fl.start + fl.len > wk.n) {
            set_error(wk.ctl, kErrBounds);
            continue;
        }
        const K v = decode_key(static_cast<K>(fl.value), wk.codec);
        for (uint32_t i = threadIdx.x; i < fl.len; i += blockDim.x) out[fl.start + i] = v;
    }
}

template <typename K>
struct Cfg;
template <>
struct Cfg<uint32_t> {
    static constexpr int kThreads = 512;
    static constexpr int kItems = 16;
};
template <>
struct Cfg<uint64_t> {
    static constexpr int kThreads = 512;
    static constexpr int kItems = 8;
};

}  // namespace

MsdShape msd_shape(int key_bytes) {
    MsdShape s;
    if (key_bytes == 4) {
        s.tile = Cfg<uint32_t>::kThreads * Cfg<uint32_t>::kItems;
        s.levels = 4;
    } else {
        s.tile = Cfg<uint64_t>::kThreads * Cfg<uint64_t>::kItems;
        s.levels = 8;
    }
    s.chunk = 2 * s.tile;
    s.unit_cap = s.tile;
    s.merge_cap = s.tile / 2;
    return s;
}

template <typename K>
void launch_msd(const Work &wk, cudaStream_t st, Recorder &rec, int num_sms) {
    constexpr int T = Cfg<K>::kThreads, I = Cfg<K>::kItems;
    const MsdShape shape = msd_shape(sizeof(K));
    const bool direct = wk.n <= shape.unit_cap;
    const uint32_t nc0 = direct ? 0u : static_cast<uint32_t>((wk.n + wk.chunk_keys - 1) / wk.chunk_keys);
    rec.begin(BSORT_K_INIT, -1);
    k_init<<<direct ? 1 : max(1u, min(1024u, (nc0 + 255) / 256)), 256, 0, st>>>(wk, nc0, direct ? 1 : 0);
    rec.end();
    if (!direct) {
        for (int level = 0; level < shape.levels; ++level) {
            rec.begin(BSORT_K_HIST, level);
            k_hist<K, 512><<<num_sms * 4, 512, 0, st>>>(wk, level);
            rec.end();
            rec.begin(BSORT_K_SCAN, level);
            k_colscan<1024><<<kBins, 1024, 0, st>>>(wk, level);
            rec.end();
            rec.begin(BSORT_K_CLASSIFY, level);
            k_classify<kBins><<<num_sms * 4, kBins, 0, st>>>(wk, level);
            rec.end();
            rec.begin(BSORT_K_SCATTER, level);
            k_scatter<K, T, I><<<num_sms * 2, T, 0, st>>>(wk, level);
            rec.end();
        }
    }
    rec.begin(BSORT_K_FINISH, -1);
    k_finish<K, T, I><<<num_sms * 2, T, 0, st>>>(wk);
    rec.end();
    if (!direct) {
        rec.begin(BSORT_K_FILL, -1);
        k_fill<K><<<num_sms * 2, 256, 0, st>>>(wk);
        rec.end();
    }
}

template void launch_msd<uint32_t>(const Work &, cudaStream_t, Recorder &, int);
template void launch_msd<uint64_t>(const Work &, cudaStream_t, Recorder &, int);

}  // namespace bsort
