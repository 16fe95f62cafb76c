// In-place digit pass of the bsort library (sm_103a), for 4- and 8-byte keys.
//
// The paper's partition (Alg. 1) swaps keys inside the array and needs only
// O(w) extra memory.  The ping-pong pipeline moves each digit pass to a second
// buffer; this file replaces that scatter with a permutation inside the
// caller's buffer, at the granularity of 128-byte blocks:
//
//   small buckets (at most kSmemCap keys): one CTA holds the whole bucket in
//     shared memory and writes it back in digit order (k_ip_smem);
//   larger buckets, in three launches:
//     k_ip_stripe   each CTA streams one stripe (a block-aligned piece of the
//                   bucket) and collects keys per digit in shared memory; every
//                   full block of B keys of one digit is written back to the
//                   front of the stripe (never past what has been read), the
//                   under-full rest of each digit goes to a per-stripe buffer;
//     k_ip_permute  digit d owns the block slots [A_d, A_d + N_d) of the bucket,
//                   A_d = ceil(D_d / B) (D_d: digit base, N_d: its full blocks).
//                   Each block's slot is fixed by the classification (its
//                   stripe's share of digit d, claimed per stripe, plus its
//                   rank there) and written into the state word of the slot
//                   it sits in.  Groups of lanes carry blocks: the block at
//                   the destination, if not yet moved, is taken along (an
//                   atomic OR on the slot's state word decides who takes it
//                   and returns where it goes) while its read is in flight,
//                   so every block moves exactly once in one round trip per
//                   hop and nothing ever waits for anything but a read in
//                   progress;
//     k_ip_cleanup  per digit, the partial blocks of all stripes and the part of
//                   the digit's last block that crossed D_{d+1} (kept aside by
//                   the carrier) fill the rest of the digit's range.
// Auxiliary memory: counters, one partial-block buffer per stripe, one
// overflow block per (bucket, digit) and one state word per block slot.
#include "bsort_launch.h"

namespace bsort {

namespace {

constexpr unsigned kFullMask = 0xffffffffu;

// Slot state word: bits 31-30 the state, bits 29-0 the destination slot of
// the block the slot held after classification (while the stripe is being
// classified: bits 29-22 its digit, bits 21-0 its rank among the stripe's
// blocks of that digit).  OR-ing kSlotTaken takes a full slot and leaves the
// other states as they are; the old word says where the taken block goes.
constexpr uint32_t kSlotFull = 0u << 30;   // holds a block that has not moved yet
constexpr uint32_t kSlotTaken = 1u << 30;  // a group is reading the block out
constexpr uint32_t kSlotHole = 3u << 30;   // nothing left to read
constexpr uint32_t kSlotStateMask = 3u << 30;

constexpr int kIpStripeThreads = 512;
constexpr int kIpPermuteThreads = 256;
constexpr int kIpCleanupThreads = 256;
constexpr int kIpSmemThreads = 1024;
constexpr int kSpinLimit = 1 << 20;  // polls of about a microsecond each: about a second

template <typename K>
struct IpCfg {
    static constexpr int B = kIpBlockBytes / static_cast<int>(sizeof(K));  // keys per block
    static constexpr int kTile = 32768 / static_cast<int>(sizeof(K));       // stripe pass tile (32 KB)
    static constexpr int kSmemCap = kIpSmemCapBytes / static_cast<int>(sizeof(K));
};

extern __shared__ __align__(16) unsigned char g_ip_smem[];

// Waits, at most kSpinLimit polls (a fraction of a second), until
// (*word & mask) == want; returns whether it did.  The one kind of wait in
// the library: a caller that gives up sets an error bit and returns.
__device__ __forceinline__ uint32_t bounded_wait(uint32_t *word, uint32_t mask, uint32_t want) {
    for (int i = 0; i < kSpinLimit; ++i) {
        if ((atomicAdd(word, 0u) & mask) == want) {
            __threadfence();
            return 1;
        }
        __nanosleep(32);
    }
    return 0;
}

// Self-test of the bounded wait: waits on a flag nothing sets and records
// the timeout in err (kErrTimeout), then returns.
__global__ void k_wait_selftest(uint32_t *flag, uint32_t *err) {
    if (threadIdx.x == 0 && !bounded_wait(flag, 0xffffffffu, 1u)) atomicOr(err, kErrTimeout);
}

__device__ __forceinline__ void ip_error(const Work &wk, uint32_t bits) { atomicOr(&wk.ctl->error, bits); }

// Digit geometry of bucket i of this level (same rule as the ping-pong pass).
struct DigitGeo {
    int shift;
    uint32_t mask;
};

__device__ __forceinline__ DigitGeo digit_geo(const Bucket &b, int radix_bits) {
    const int r_eff = b.h < radix_bits ? b.h : radix_bits;
    DigitGeo g;
    g.shift = b.h - r_eff;
    g.mask = (1u << r_eff) - 1u;
    return g;
}

template <typename K>
__device__ __forceinline__ uint32_t digit_of(K key, const DigitGeo &g) {
    return static_cast<uint32_t>(key >> g.shift) & g.mask;
}

// D_d relative to the bucket start: the digit base, len past the last digit.
__device__ __forceinline__ uint64_t dbase(const Work &wk, uint32_t bucket, const DigitGeo &g, uint32_t d,
                                          uint64_t len) {
    return d <= g.mask ? wk.bucket_base[static_cast<size_t>(bucket) * wk.bins + d] : len;
}

// ---------------------------------------------------------------------------
// Lists of this level: big buckets, their stripes and slot states.
template <typename K>
__global__ void k_ip_plan(Work wk, int level) {
    constexpr int B = IpCfg<K>::B;
    const int p = level & 1;
    if (wk.ctl->error) return;
    write_child_chunks(wk, p ^ 1);  // records of the buckets this level's classify opened
    const uint32_t nb = wk.ctl->n_buckets[p];
    __shared__ uint32_t sh[3];
    for (uint32_t i = blockIdx.x; i < nb; i += gridDim.x) {
        const Bucket b = wk.buckets[p][i];
        if (!b.scatter || b.len <= static_cast<uint64_t>(IpCfg<K>::kSmemCap)) continue;  // block-uniform
        const uint64_t stripe_keys = kIpStripeBytes / sizeof(K);
        const uint32_t ns = static_cast<uint32_t>((b.len + stripe_keys - 1) / stripe_keys);
        const uint32_t nslots = static_cast<uint32_t>((b.len + B - 1) / B);
        if (threadIdx.x == 0) {
            const uint32_t bb = atomicAdd(&wk.ctl->n_big, 1u);
            const uint32_t s0 = atomicAdd(&wk.ctl->n_stripes, ns);
            const uint32_t st0 = atomicAdd(&wk.ctl->n_slots, nslots);
            const bool ok = bb < wk.max_big && s0 + ns <= wk.max_stripes && st0 + nslots <= wk.max_slots;
            if (!ok) ip_error(wk, kErrCapacity);
            sh[0] = ok ? bb : 0xffffffffu;
            sh[1] = s0;
            sh[2] = st0;
            if (ok) {
                IpBig g;
                g.start = b.start;
                g.len = b.len;
                g.bucket = i;
                g.first_stripe = s0;
                g.num_stripes = ns;
                g.state0 = st0;
                wk.ip_big[bb] = g;
            }
        }
        __syncthreads();
        const uint32_t bb = sh[0], s0 = sh[1];
        if (bb != 0xffffffffu) {
            for (uint32_t j = threadIdx.x; j < ns; j += blockDim.x) {
                IpStripe s;
                const uint64_t off = static_cast<uint64_t>(j) * stripe_keys;
                s.start = b.start + off;
                const uint64_t rest = b.len - off;
                s.len = static_cast<uint32_t>(rest < stripe_keys ? rest : stripe_keys);
                s.big = bb;
                s.slot0 = static_cast<uint32_t>(off / B);
                s.nfull = 0;
                wk.ip_stripes[s0 + j] = s;
            }
            for (uint32_t d = threadIdx.x; d < kBins; d += blockDim.x) {
                wk.ip_ncnt[static_cast<size_t>(bb) * kBins + d] = 0;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Whole-bucket pass: the bucket's keys in shared memory, written back at
// bucket start + digit base + (unstable) rank.
template <typename K>
__global__ void __launch_bounds__(kIpSmemThreads) k_ip_smem(Work wk, int level) {
    constexpr int T = kIpSmemThreads;
    K *keys_s = reinterpret_cast<K *>(g_ip_smem);
    uint32_t *cur = reinterpret_cast<uint32_t *>(g_ip_smem + sizeof(K) * IpCfg<K>::kSmemCap);
    const int p = level & 1;
    if (wk.ctl->error) return;
    const uint32_t nb = wk.ctl->n_buckets[p];
    K *keys = static_cast<K *>(wk.keys);
    for (uint32_t i = blockIdx.x; i < nb; i += gridDim.x) {
        const Bucket b = wk.buckets[p][i];
        if (!b.scatter || b.len > static_cast<uint64_t>(IpCfg<K>::kSmemCap)) continue;  // block-uniform
        const DigitGeo g = digit_geo(b, wk.radix_bits);
        const int len = static_cast<int>(b.len);
        K *base = keys + b.start;
        for (int j = threadIdx.x; j < len; j += T) keys_s[j] = b.raw ? encode_key(base[j], wk.codec) : base[j];
        for (uint32_t d = threadIdx.x; d < kBins; d += T)
            cur[d] = d <= g.mask ? wk.bucket_base[static_cast<size_t>(i) * wk.bins + d] : 0u;
        __syncthreads();
        bool bad = false;
        for (int j = threadIdx.x; j < len; j += T) {
            const K k = keys_s[j];
            const uint32_t pos = atomicAdd(&cur[digit_of(k, g)], 1u);
            if (pos < static_cast<uint32_t>(len)) base[pos] = k;
            else bad = true;
        }
        if (bad) ip_error(wk, kErrBounds);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Stripe classification.  Shared memory: the tile, the tile in digit order,
// per-digit block buffers [kBins][B], and per-digit counters.
template <typename K>
struct StripeSmem {
    static constexpr int B = IpCfg<K>::B, TILE = IpCfg<K>::kTile;
    static constexpr size_t kTileK = 0;
    static constexpr size_t kSorted = kTileK + sizeof(K) * TILE;
    static constexpr size_t kBuf = kSorted + sizeof(K) * TILE;
    static constexpr size_t kCnt = kBuf + sizeof(K) * kBins * B;  // tile digit counts
    static constexpr size_t kStart = kCnt + 4 * kBins;            // tile digit starts, then placement cursors
    static constexpr size_t kFill = kStart + 4 * kBins;           // keys in each digit buffer
    static constexpr size_t kBlk = kFill + 4 * kBins;             // block slot base of each digit in this tile
    static constexpr size_t kNFull = kBlk + 4 * kBins;            // full blocks of each digit in the stripe
    static constexpr size_t kScan = kNFull + 4 * kBins;
    static constexpr size_t kBmap = kScan + 4 * (kIpStripeThreads / 32 + 1);  // digit of each block of a tile
    static constexpr int kMaxTileBlocks = (TILE + kBins * (B - 1)) / B;
    static constexpr size_t kEnd = kBmap + kMaxTileBlocks;
};

template <int THREADS>
__device__ __forceinline__ uint32_t ip_block_scan(uint32_t v, uint32_t *tmp, uint32_t &total) {
    constexpr int WARPS = THREADS / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFullMask, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) tmp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t s = lane < WARPS ? tmp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFullMask, s, o);
            if (lane >= o) s += y;
        }
        if (lane < WARPS) tmp[lane] = s;
    }
    __syncthreads();
    const uint32_t r = (warp ? tmp[warp - 1] : 0) + x - v;
    total = tmp[WARPS - 1];
    __syncthreads();
    return r;
}

template <typename K>
__global__ void __launch_bounds__(kIpStripeThreads, 2) k_ip_stripe(Work wk, int level) {
    using S = StripeSmem<K>;
    constexpr int B = S::B, TILE = S::TILE, T = kIpStripeThreads;
    K *tile = reinterpret_cast<K *>(g_ip_smem + S::kTileK);
    K *sorted = reinterpret_cast<K *>(g_ip_smem + S::kSorted);
    K *buf = reinterpret_cast<K *>(g_ip_smem + S::kBuf);
    uint32_t *cnt = reinterpret_cast<uint32_t *>(g_ip_smem + S::kCnt);
    uint32_t *tstart = reinterpret_cast<uint32_t *>(g_ip_smem + S::kStart);
    uint32_t *fill = reinterpret_cast<uint32_t *>(g_ip_smem + S::kFill);
    uint32_t *blk = reinterpret_cast<uint32_t *>(g_ip_smem + S::kBlk);
    uint32_t *nfull = reinterpret_cast<uint32_t *>(g_ip_smem + S::kNFull);
    uint8_t *bmap = reinterpret_cast<uint8_t *>(g_ip_smem + S::kBmap);
    uint32_t *scan_tmp = reinterpret_cast<uint32_t *>(g_ip_smem + S::kScan);
    const int t = threadIdx.x;
    const int p = level & 1;
    if (wk.ctl->error) return;
    const uint32_t ns = min(wk.ctl->n_stripes, wk.max_stripes);
    K *keys = static_cast<K *>(wk.keys);
    for (uint32_t si = blockIdx.x; si < ns; si += gridDim.x) {
        const IpStripe s = wk.ip_stripes[si];
        const IpBig big = wk.ip_big[s.big];
        const Bucket b = wk.buckets[p][big.bucket];
        const DigitGeo g = digit_geo(b, wk.radix_bits);
        K *base = keys + s.start;
        for (int d = t; d < kBins; d += T) {
            fill[d] = 0;
            nfull[d] = 0;
        }
        uint32_t wp = 0;  // blocks written at the front of the stripe
        for (uint32_t t0 = 0; t0 < s.len; t0 += TILE) {
            const int tlen = static_cast<int>(min(static_cast<uint32_t>(TILE), s.len - t0));
            for (int j = t; j < tlen; j += T) tile[j] = b.raw ? encode_key(base[t0 + j], wk.codec) : base[t0 + j];
            for (int d = t; d < kBins; d += T) cnt[d] = 0;
            __syncthreads();
            for (int j = t; j < tlen; j += T) atomicAdd(&cnt[digit_of(tile[j], g)], 1u);
            __syncthreads();
            // tile digit starts (thread d < kBins), block counts per digit, slot bases
            uint32_t nbk = 0, c = 0, f = 0;
            if (t < kBins) {
                c = cnt[t];
                f = fill[t];
                nbk = (f + c) / B;
            }
            uint32_t tot_keys, tot_blocks;
            const uint32_t st = ip_block_scan<T>(t < kBins ? c : 0u, scan_tmp, tot_keys);
            const uint32_t bs = ip_block_scan<T>(nbk, scan_tmp, tot_blocks);
            if (t < kBins) {
                tstart[t] = st;
                blk[t] = wp + bs;
            }
            __syncthreads();
            // tile in digit order (tstart becomes the placement cursor, then is restored)
            for (int j = t; j < tlen; j += T) {
                const K k = tile[j];
                sorted[atomicAdd(&tstart[digit_of(k, g)], 1u)] = k;
            }
            __syncthreads();
            if (t < kBins) tstart[t] = st;
            __syncthreads();
            // full blocks of every digit go to the stripe front: block bi of
            // this tile (slot wp + bi) belongs to digit bmap[bi]; one thread
            // per key, so consecutive threads write consecutive addresses
            if (t < kBins) {
                for (uint32_t kb = 0; kb < nbk; ++kb) bmap[blk[t] - wp + kb] = static_cast<uint8_t>(t);
            }
            __syncthreads();
            for (uint32_t i = t; i < tot_blocks * B; i += T) {
                const uint32_t bi = i / B, e = i % B;
                const uint32_t d = bmap[bi];
                const uint32_t kb = bi - (blk[d] - wp);
                const uint32_t idx = kb * B + e, fd = fill[d];
                const K v = idx < fd ? buf[d * B + idx] : sorted[tstart[d] + idx - fd];
                const uint64_t pos = static_cast<uint64_t>(wp + bi) * B + e;
                if (pos < t0 + static_cast<uint64_t>(tlen)) base[pos] = v;  // never past what was read
                else ip_error(wk, kErrBounds);
                if (e == 0)
                    wk.ip_state[big.state0 + s.slot0 + wp + bi] = kSlotFull | (d << 22) | (nfull[d] + kb);
            }
            __syncthreads();
            // the rest of each digit's stream becomes its buffer
            for (uint32_t i = t; i < static_cast<uint32_t>(kBins * B); i += T) {
                const uint32_t d = i / B, r = i % B;
                const uint32_t fd = fill[d], totd = fd + cnt[d], nb = totd / B;
                const uint32_t idx = nb * B + r;  // stream index of the new buffer entry r
                if (idx < totd && idx >= fd) buf[d * B + r] = sorted[tstart[d] + idx - fd];
            }
            __syncthreads();
            if (t < kBins) {
                fill[t] = f + c - nbk * B;
                nfull[t] += nbk;
            }
            wp += tot_blocks;
            __syncthreads();
        }
        // stripe summary: full-block counts, partial blocks, slot states.
        // This stripe's blocks of digit d take the digit's slots [P, P + nfull)
        // past its slot base A_d = ceil(D_d / B), P claimed here in any order of
        // the stripes; each full slot's word then names its block's destination.
        uint32_t *pref = cnt;     // reuse: per-digit claimed share
        uint32_t *abase = tstart; // reuse: per-digit slot base
        for (int d = t; d < kBins; d += T) {
            pref[d] = nfull[d] ? atomicAdd(&wk.ip_ncnt[static_cast<size_t>(s.big) * kBins + d], nfull[d]) : 0u;
            abase[d] = static_cast<uint32_t>((dbase(wk, big.bucket, g, d, big.len) + B - 1) / B);
            wk.ip_rem[static_cast<size_t>(si) * kBins + d] = static_cast<uint8_t>(fill[d]);
        }
        __syncthreads();
        for (uint32_t j = t; j < wp; j += T) {
            uint32_t *w = &wk.ip_state[big.state0 + s.slot0 + j];
            const uint32_t v = *w, d = (v >> 22) & 0xFFu;
            *w = kSlotFull | (abase[d] + pref[d] + (v & 0x3FFFFFu));
        }
        K *part = static_cast<K *>(wk.ip_part) + static_cast<size_t>(si) * kBins * B;
        for (int i = t; i < kBins * B; i += T) {
            const int d = i / B, e = i % B;
            if (static_cast<uint32_t>(e) < fill[d]) part[i] = buf[i];
        }
        const uint32_t nslots = (s.len + B - 1) / B;
        for (uint32_t j = wp + t; j < nslots; j += T) wk.ip_state[big.state0 + s.slot0 + j] = kSlotHole;
        if (t == 0) wk.ip_stripes[si].nfull = wp;
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Block permutation.  A group of 8 lanes carries one block: lane gl of the
// group holds keys gl, gl + 8, gl + 16, ... of it (B / 8 keys), so every
// access of the group covers 32 contiguous bytes.  A warp runs four groups,
// each with its own chain, so four carries are in flight per warp.

constexpr int kGroup = 8;

template <typename K>
struct Carry {
    static constexpr int B = IpCfg<K>::B, E = B / kGroup;  // keys per lane
    const Work &wk;
    const IpBig &big;
    uint32_t bb;
    DigitGeo g;
    K *keys;
    K *ovf;
    const uint64_t *dend;  // [kBins] D_{d+1}, relative to the bucket start (shared memory)

    // Reads the block in slot `slot` (keys past the bucket's end, in its last
    // partial slot, are not read).
    __device__ void load(uint32_t slot, int gl, K (&v)[E]) const {
        const uint64_t p0 = static_cast<uint64_t>(slot) * B + gl;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const uint64_t pos = p0 + e * kGroup;
            v[e] = pos < big.len ? keys[big.start + pos] : K(0);
        }
    }

    // Writes a block of digit d into slot `slot`; keys past D_{d+1} go to the
    // digit's overflow buffer.
    __device__ void put(uint32_t d, uint32_t slot, const K (&v)[E], int gl) const {
        const uint64_t end = dend[d];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const uint64_t pos = static_cast<uint64_t>(slot) * B + gl + e * kGroup;
            if (pos < end) keys[big.start + pos] = v[e];
            else if (pos - end < static_cast<uint64_t>(B))
                ovf[(static_cast<size_t>(bb) * kBins + d) * B + (pos - end)] = v[e];
            else ip_error(wk, kErrBounds);
        }
    }
};

template <typename K>
__global__ void __launch_bounds__(kIpPermuteThreads) k_ip_permute(Work wk, int level) {
    using C = Carry<K>;
    constexpr int B = C::B, E = C::E, GROUPS = kIpPermuteThreads / kGroup;
    const int lane = threadIdx.x & 31, gl = lane & (kGroup - 1);
    const int grp = threadIdx.x / kGroup;  // group of this CTA
    const int leader = lane & ~(kGroup - 1);
    const unsigned gmask = 0xFFu << leader;
    const int p = level & 1;
    __shared__ uint64_t dend[kBins];
    if (wk.ctl->error) return;
    const uint32_t ns = min(wk.ctl->n_stripes, wk.max_stripes);
    K *keys = static_cast<K *>(wk.keys);
    K *ovf = static_cast<K *>(wk.ip_ovf);
    for (uint32_t si = blockIdx.x; si < ns; si += gridDim.x) {
        const IpStripe s = wk.ip_stripes[si];
        const IpBig big = wk.ip_big[s.big];
        const Bucket b = wk.buckets[p][big.bucket];
        __syncthreads();  // the previous stripe's groups are done with dend
        for (int d = threadIdx.x; d < kBins; d += kIpPermuteThreads)
            dend[d] = dbase(wk, big.bucket, digit_geo(b, wk.radix_bits), d + 1, big.len);
        __syncthreads();
        const C cy{wk, big, s.big, digit_geo(b, wk.radix_bits), keys, ovf, dend};
        uint32_t *state = wk.ip_state + big.state0;
        const uint32_t nslots = static_cast<uint32_t>((big.len + B - 1) / B);
        bool fail = false;
        for (uint32_t j = grp; j < s.nfull && !fail; j += GROUPS) {
            const uint32_t seed = s.slot0 + j;
            uint32_t old = kSlotHole;
            if (gl == 0) old = atomicOr(&state[seed], kSlotTaken);
            old = __shfl_sync(gmask, old, leader);
            if ((old & kSlotStateMask) != kSlotFull) continue;
            // take the seed block out, then free its slot
            K x[E];
            cy.load(seed, gl, x);
            __syncwarp(gmask);
            if (gl == 0) {
                __threadfence();
                atomicOr(&state[seed], kSlotHole);
            }
            uint32_t xw = old;  // the carried block's state word: its destination
            // carry until the block lands on a slot that holds nothing to take
            for (int hop = 0;; ++hop) {
                const uint32_t d = digit_of(__shfl_sync(gmask, x[0], leader), cy.g);
                const uint32_t dst = xw & ~kSlotStateMask;
                if (dst >= nslots || hop > (1 << 26)) {
                    if (gl == 0) ip_error(wk, kErrBounds);
                    fail = true;
                    break;
                }
                // take whatever dst holds and read it in the same round trip
                // (the read is used only if the slot was full: a full slot
                // changes only when its one destination writer -- this group
                // -- writes it)
                K y[E];
                cy.load(dst, gl, y);
                uint32_t dw = 0;
                if (gl == 0) dw = atomicOr(&state[dst], kSlotTaken);
                dw = __shfl_sync(gmask, dw, leader);
                if ((dw & kSlotStateMask) == kSlotFull) {
                    __syncwarp(gmask);
                    cy.put(d, dst, x, gl);
#pragma unroll
                    for (int e = 0; e < E; ++e) x[e] = y[e];
                    xw = dw;
                    continue;
                }
                if ((dw & kSlotStateMask) == kSlotTaken) {
                    // a seeding group is reading the block at dst out
                    uint32_t ready = 0;
                    if (gl == 0) ready = bounded_wait(&state[dst], kSlotStateMask, kSlotHole);
                    if (!__shfl_sync(gmask, ready, leader)) {
                        if (gl == 0) ip_error(wk, kErrTimeout);
                        fail = true;
                        break;
                    }
                }
                cy.put(d, dst, x, gl);
                break;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Cleanup: per (big bucket, digit), the keys outside the digit's full slots.
template <typename K>
__global__ void __launch_bounds__(kIpCleanupThreads) k_ip_cleanup(Work wk, int level) {
    constexpr int B = IpCfg<K>::B, WARPS = kIpCleanupThreads / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int p = level & 1;
    if (wk.ctl->error) return;
    const uint32_t nbig = min(wk.ctl->n_big, wk.max_big);
    K *keys = static_cast<K *>(wk.keys);
    const K *part = static_cast<const K *>(wk.ip_part);
    const K *ovf = static_cast<const K *>(wk.ip_ovf);
    const uint64_t items = static_cast<uint64_t>(nbig) * kBins;
    for (uint64_t it = static_cast<uint64_t>(blockIdx.x) * WARPS + warp; it < items;
         it += static_cast<uint64_t>(gridDim.x) * WARPS) {
        const uint32_t bb = static_cast<uint32_t>(it / kBins), d = static_cast<uint32_t>(it % kBins);
        const IpBig big = wk.ip_big[bb];
        const Bucket b = wk.buckets[p][big.bucket];
        const DigitGeo g = digit_geo(b, wk.radix_bits);
        if (d > g.mask) continue;
        const uint64_t D0 = dbase(wk, big.bucket, g, d, big.len), D1 = dbase(wk, big.bucket, g, d + 1, big.len);
        const uint64_t N = wk.ip_ncnt[it];
        const uint64_t A = (D0 + B - 1) / B;
        // positions of the digit's range outside its full slots: [D0, h1) then [t0, D1)
        uint64_t h1, t0, o;
        if (N == 0) {
            h1 = D1;
            t0 = D1;
            o = 0;
        } else {
            h1 = A * B;
            const uint64_t e = (A + N) * B;
            t0 = e < D1 ? e : D1;
            o = e > D1 ? e - D1 : 0;
        }
        const uint64_t need = (h1 - D0) + (D1 - t0);
        auto position = [&](uint64_t k) { return k < h1 - D0 ? D0 + k : t0 + (k - (h1 - D0)); };
        uint64_t k0 = 0;
        for (uint32_t s0 = 0; s0 < big.num_stripes; s0 += 32) {
            const uint32_t si = big.first_stripe + s0 + lane;
            const uint32_t r = s0 + lane < big.num_stripes ? wk.ip_rem[static_cast<size_t>(si) * kBins + d] : 0u;
            uint32_t incl = r;
#pragma unroll
            for (int sh = 1; sh < 32; sh <<= 1) {
                const uint32_t y = __shfl_up_sync(kFullMask, incl, sh);
                if (lane >= sh) incl += y;
            }
            const uint32_t total = __shfl_sync(kFullMask, incl, 31);
            const uint64_t my0 = k0 + incl - r;
            // lane l copies stripe s0 + l's partial block of digit d
            for (uint32_t e = 0; e < r; ++e) {
                const uint64_t k = my0 + e;
                if (k < need) keys[big.start + position(k)] = part[(static_cast<size_t>(si) * kBins + d) * B + e];
            }
            k0 += total;
        }
        for (uint32_t e = lane; e < o; e += 32) {
            const uint64_t k = k0 + e;
            if (k < need) keys[big.start + position(k)] = ovf[(static_cast<size_t>(bb) * kBins + d) * B + e];
        }
        if (lane == 0 && k0 + o != need) ip_error(wk, kErrBounds);
    }
}

// Auxiliary bytes this level used (largest level kept).
template <typename K>
__global__ void k_ip_account(Work wk) {
    const unsigned long long used =
        static_cast<unsigned long long>(min(wk.ctl->n_stripes, wk.max_stripes)) * (kBins * kIpBlockBytes + kBins) +
        static_cast<unsigned long long>(min(wk.ctl->n_big, wk.max_big)) * (kBins * kIpBlockBytes + 4 * kBins) +
        static_cast<unsigned long long>(min(wk.ctl->n_slots, wk.max_slots)) * 4;
    atomicMax(&wk.ctl->aux_used, used);
}

}  // namespace

template <typename K>
void ip_prepare() {
    static const bool attrs = [] {
        cudaFuncSetAttribute(k_ip_smem<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(sizeof(K) * IpCfg<K>::kSmemCap + 4 * kBins));
        cudaFuncSetAttribute(k_ip_stripe<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(StripeSmem<K>::kEnd));
        return true;
    }();
    (void)attrs;
}

template <typename K>
void launch_ip_level(const Work &wk, cudaStream_t st, Recorder &rec, int num_sms, int level) {
    rec.begin(BSORT_K_SCATTER, level);
    cudaMemsetAsync(&wk.ctl->n_big, 0, 3 * sizeof(uint32_t), st);
    k_ip_plan<K><<<num_sms * 2, 256, 0, st>>>(wk, level);
    k_ip_smem<K><<<num_sms, kIpSmemThreads, sizeof(K) * IpCfg<K>::kSmemCap + 4 * kBins, st>>>(wk, level);
    k_ip_stripe<K><<<num_sms * 2, kIpStripeThreads, StripeSmem<K>::kEnd, st>>>(wk, level);
    k_ip_permute<K><<<num_sms * 8, kIpPermuteThreads, 0, st>>>(wk, level);
    k_ip_cleanup<K><<<num_sms * 4, kIpCleanupThreads, 0, st>>>(wk, level);
    k_ip_account<K><<<1, 1, 0, st>>>(wk);
    rec.more(5);  // the group's other five kernels
    rec.end();
}

void launch_wait_selftest(uint32_t *flag_and_err, cudaStream_t st) {
    k_wait_selftest<<<1, 32, 0, st>>>(flag_and_err, flag_and_err + 1);
}

template void ip_prepare<uint32_t>();
template void ip_prepare<uint64_t>();
template void launch_ip_level<uint32_t>(const Work &, cudaStream_t, Recorder &, int, int);
template void launch_ip_level<uint64_t>(const Work &, cudaStream_t, Recorder &, int, int);

}  // namespace bsort
