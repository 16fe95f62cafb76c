// Shared device-side definitions of the bsort CUDA library (sm_103a).
//
// The sort works on "encoded" keys: an order-preserving bijection maps every
// dtype onto unsigned words whose ascending order is the requested order
// (Sec. III of the paper: the sign pass of Algs. 3/4 runs in the inverted
// direction, and the negative float half in the inverted direction on its
// exponent and mantissa bits).  Encoding costs a select and a xor:
//     encode(x) = x ^ (msb(x) ? F1 : F0),   decode(k) = k ^ (msb(k) ? D1 : D0)
// with the constants of codec_for().  After encoding, the r-bit MSD digit
// passes are r consecutive binary partitions of Alg. 1 on masks
// 1 << (s - i), fused: binary splits refine lexicographically (Thm. 3's
// induction), so one stable r-bit split equals r successive bit splits.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace bsort {

constexpr int kRadixBits = 8;              // default digit width of the MSD levels
constexpr int kBins = 1 << kRadixBits;     // digits of an 8-bit pass (narrow tables, LSD finish passes)
constexpr int kMinRadixBits = 1;           // narrowest tunable digit width (1: one bit partition per pass)
constexpr int kMaxRadixBits = 11;          // widest tunable digit width (ping-pong levels)
constexpr int kWideBins = 1 << kMaxRadixBits;  // table stride of the digit widths above kRadixBits
constexpr int kMaxLevels = 64;             // ceil(64 / kMinRadixBits)

// device error word bits
constexpr uint32_t kErrCapacity = 1u;
constexpr uint32_t kErrTimeout = 2u;
constexpr uint32_t kErrBounds = 4u;  // a device-side bounds check refused a store

struct Codec {
    uint64_t f0, f1;  // encode: x ^ (msb ? f1 : f0)
    uint64_t d0, d1;  // decode: k ^ (msb ? d1 : d0)
};

// One MSD bucket: keys [start, start+len) of buffer `src` agree on every bit
// at or above position h; bits [0, h) are not partitioned yet.
struct Bucket {
    uint64_t start;
    uint64_t len;
    uint32_t first_chunk;
    uint32_t num_chunks;
    int32_t h;
    uint8_t src;      // 0: caller's keys buffer, 1: alternate buffer
    uint8_t raw;      // keys in src still in the caller's encoding
    uint8_t scatter;  // classify: this bucket is scattered at this level
    uint8_t pad;
};

// A contiguous piece of one bucket, processed by one CTA in the histogram and
// scatter kernels (same decomposition in both, so per-chunk offsets match).
struct Chunk {
    uint64_t start;
    uint32_t len;
    uint32_t bucket;
};

// A run of keys (one or several adjacent small buckets) sorted entirely in
// shared memory and written, decoded, to its final place.  Its keys agree on
// every bit at or above `vbits` (0: not known).
struct Unit {
    uint64_t start;
    uint32_t len;
    uint8_t src;
    uint8_t raw;
    uint8_t vbits;
    uint8_t pad;
};

// A run of identical keys written without reading (value is encoded; its
// bits 64..127 in value_hi for 16-byte keys).
struct Fill {
    uint64_t start;
    uint64_t value;
    uint64_t value_hi;
    uint32_t len;
    uint32_t src;  // key-value sorting: the buffer parity the run's values sit in
};

// In-place mode: a bucket of this level too large for the whole-bucket
// shared-memory pass, and one stripe (a contiguous, block-aligned piece of
// it that one CTA classifies into blocks).
struct IpBig {
    uint64_t start;
    uint64_t len;
    uint32_t bucket;        // index in this level's bucket list
    uint32_t first_stripe;  // its stripes are [first_stripe, first_stripe + num_stripes)
    uint32_t num_stripes;
    uint32_t state0;        // index of its slot 0 in the slot-state array
};

struct IpStripe {
    uint64_t start;  // absolute key index (bucket start + slot0 * block keys)
    uint32_t len;
    uint32_t big;
    uint32_t slot0;  // first slot, relative to the bucket start
    uint32_t nfull;  // full blocks at the stripe's start after classification
};

struct Ctl {
    uint32_t n_buckets[2];
    uint32_t n_chunks[2];
    uint32_t n_units;
    uint32_t n_fills;
    uint32_t error;
    uint32_t n_fb;  // units handed from the comparison finish to the LSD finish
    unsigned long long hist_keys[kMaxLevels];     // keys read by the histogram of a level
    unsigned long long scatter_keys[kMaxLevels];  // keys moved by the scatter of a level
    unsigned long long finish_keys;
    unsigned long long fill_keys;
    unsigned long long raw_reads;                 // keys read while still raw (diagnostic)
    unsigned long long fin_counting, fin_compare; // finish units by method (diagnostic)
    unsigned long long fin_fast;                  // of fin_counting: the vector-load counting pass
    uint32_t n_big, n_stripes, n_slots, ip_pad;   // in-place lists of the current level
    unsigned long long aux_used;                  // in-place: largest auxiliary bytes any level used
};

// Everything a launch needs, passed by value.
struct Work {
    Ctl *ctl;
    Bucket *buckets[2];
    Chunk *chunks[2];
    uint32_t *hist;         // [bins][max_chunks], digit-major; excl. prefix after the scan
    uint64_t *chunk_and;    // [max_chunks] (16-byte keys: two words per chunk, low word first)
    uint64_t *chunk_or;     // [max_chunks] (likewise)
    uint32_t *bucket_base;  // [max_buckets][bins]: digit totals, then digit bases relative to the bucket start
    Unit *units;
    Unit *fb_units;  // [max_units] skewed units for the LSD finish
    Fill *fills;
    void *keys;
    void *alt;
    uint64_t n;
    Codec codec;
    uint32_t max_buckets, max_chunks, max_units, max_fills;
    uint32_t chunk_keys;  // keys per chunk (multiple of the scatter tile)
    uint32_t unit_cap;    // largest run the shared-memory finish sorts
    uint32_t merge_cap;   // adjacent small buckets merge while their sum stays <= this
    int32_t w;            // key bits
    int32_t radix_bits;   // digit width of the MSD levels (kMinRadixBits..kMaxRadixBits)
    uint32_t bins;        // row stride of hist / bucket_base: kBins up to 8-bit digits, kWideBins above
    int32_t levels;       // host-launched MSD levels: ceil(w / radix_bits)
    int32_t stop_level;   // levels actually run (levels, or fewer for an intermediate state)
    bool keys_vec_ok;     // caller's buffer is 16-byte aligned (vector loads)
    // in-place mode (digit permutation inside the caller's buffer)
    bool inplace;
    // key-value sorting (stable): values travel beside the keys, in buffers of
    // the same parity (vals beside `keys`, vals_alt beside `alt`)
    int32_t kv;             // 0: keys only; else the value bytes (4 or 8)
    bool kv_positions;      // the values are the input positions (argsort), made at the first read
    void *vals;
    void *vals_alt;
    void *out_vals;         // where the sorted values go (the caller's values, or u32 positions)
    int64_t *out_idx;       // argsort: int64 positions written beside (may be null)
    IpBig *ip_big;          // [max_big]
    IpStripe *ip_stripes;   // [max_stripes]
    uint32_t *ip_ncnt;      // [max_big][kBins] full blocks per digit
    uint8_t *ip_rem;        // [max_stripes][kBins] keys left in a partial block
    void *ip_part;          // [max_stripes][kBins][block keys] partial blocks
    void *ip_ovf;           // [max_big][kBins][block keys] overflow of a digit's last block
    uint32_t *ip_state;     // [max_slots] slot states
    uint32_t max_big, max_stripes, max_slots;
};

constexpr uint32_t kFillPiece = 1u << 16;  // keys per fill work item

template <typename K>
__device__ __forceinline__ K encode_key(K x, const Codec &c) {
    constexpr int W = sizeof(K) * 8;
    return x ^ static_cast<K>((x >> (W - 1)) ? c.f1 : c.f0);
}

template <typename K>
__device__ __forceinline__ K decode_key(K k, const Codec &c) {
    constexpr int W = sizeof(K) * 8;
    return k ^ static_cast<K>((k >> (W - 1)) ? c.d1 : c.d0);
}

// 16-byte keys are integers only: the transform is one xor with a constant
// whose low word is f0 (d0) and high word f1 (d1) -- all ones for a
// descending sort, the sign bit for signed keys.
typedef unsigned __int128 u128;

template <>
__device__ __forceinline__ u128 encode_key<u128>(u128 x, const Codec &c) {
    return x ^ ((static_cast<u128>(c.f1) << 64) | c.f0);
}

template <>
__device__ __forceinline__ u128 decode_key<u128>(u128 k, const Codec &c) {
    return k ^ ((static_cast<u128>(c.d1) << 64) | c.d0);
}

// Warp shuffle of a key of any width.
template <typename K>
__device__ __forceinline__ K shfl_xor_k(K v, int m) {
    return __shfl_xor_sync(0xffffffffu, v, m);
}

template <>
__device__ __forceinline__ u128 shfl_xor_k<u128>(u128 v, int m) {
    const unsigned long long lo = __shfl_xor_sync(0xffffffffu, static_cast<unsigned long long>(v), m);
    const unsigned long long hi = __shfl_xor_sync(0xffffffffu, static_cast<unsigned long long>(v >> 64), m);
    return (static_cast<u128>(hi) << 64) | lo;
}

// Positions of the highest and the lowest set bit of x (x != 0).
template <typename K>
__device__ __forceinline__ int msb_pos(K x) {
    return 63 - __clzll(static_cast<unsigned long long>(x));
}

template <>
__device__ __forceinline__ int msb_pos<u128>(u128 x) {
    const unsigned long long hi = static_cast<unsigned long long>(x >> 64);
    return hi ? 127 - __clzll(hi) : 63 - __clzll(static_cast<unsigned long long>(x));
}

template <typename K>
__device__ __forceinline__ int lsb_pos(K x) {
    return __ffsll(static_cast<long long>(static_cast<unsigned long long>(x))) - 1;
}

template <>
__device__ __forceinline__ int lsb_pos<u128>(u128 x) {
    const unsigned long long lo = static_cast<unsigned long long>(x);
    return lo ? __ffsll(static_cast<long long>(lo)) - 1
              : 64 + __ffsll(static_cast<long long>(static_cast<unsigned long long>(x >> 64))) - 1;
}

// Keys with bits [0, h) cleared (h >= width: no bit kept).
template <typename K>
__device__ __forceinline__ K high_bits(K x, int h) {
    return h >= static_cast<int>(sizeof(K) * 8) ? K(0) : static_cast<K>(x & (~K(0) << h));
}

// The AND and OR of a chunk's keys in the chunk_and / chunk_or words.
template <typename K>
__device__ __forceinline__ void store_and_or(uint64_t *wa, uint64_t *wo, size_t c, K a, K o) {
    if constexpr (sizeof(K) > 8) {
        wa[2 * c] = static_cast<uint64_t>(a);
        wa[2 * c + 1] = static_cast<uint64_t>(a >> 64);
        wo[2 * c] = static_cast<uint64_t>(o);
        wo[2 * c + 1] = static_cast<uint64_t>(o >> 64);
    } else {
        wa[c] = a;
        wo[c] = o;
    }
}

template <typename K>
__device__ __forceinline__ K load_word_k(const uint64_t *w, size_t c) {
    if constexpr (sizeof(K) > 8) return (static_cast<K>(w[2 * c + 1]) << 64) | w[2 * c];
    else return static_cast<K>(w[c]);
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ void set_error(Ctl *ctl, uint32_t bits) { atomicOr(&ctl->error, bits); }

// Chunk records of the buckets of list q (the ones a level's classify just
// opened), written by the whole grid: one warp per bucket, its chunks in
// order.  A bucket's first chunk starts at the bucket; the others start on
// the chunk grid of the 16-byte-aligned base of the bucket (128 / w keys per
// 16 bytes), so every chunk after the first is an aligned window.
__device__ __forceinline__ void write_child_chunks(const Work &wk, int q) {
    const uint32_t nb = min(wk.ctl->n_buckets[q], wk.max_buckets);
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    const uint64_t vk = 128u / static_cast<uint32_t>(wk.w);
    for (uint32_t i = gw; i < nb; i += nw) {
        const Bucket b = wk.buckets[q][i];
        const uint64_t base = b.start - b.start % vk;
        const uint64_t end = b.start + b.len;
        for (uint32_t k = lane; k < b.num_chunks; k += 32) {
            if (b.first_chunk + k >= wk.max_chunks) break;
            const uint64_t cs = k == 0 ? b.start : base + static_cast<uint64_t>(k) * wk.chunk_keys;
            const uint64_t ce_lim = base + static_cast<uint64_t>(k + 1) * wk.chunk_keys;
            Chunk ch;
            ch.start = cs;
            ch.len = static_cast<uint32_t>((ce_lim < end ? ce_lim : end) - cs);
            ch.bucket = i;
            wk.chunks[q][b.first_chunk + k] = ch;
        }
    }
}

}  // namespace bsort
