// Host-side launch interface between the C ABI (api.cu) and the kernel files.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "bsort.h"
#include "bsort_device.cuh"

namespace bsort {

// Records a CUDA event pair around each launch group when profiling is on
// (accumulating over calls until read), and counts launches always.
struct Recorder {
    struct Rec {
        int kind;
        int level;
        int call;
        cudaEvent_t a, b;
    };
    bool enabled = false;
    bool active = false;  // this call is being recorded
    int count = 0;        // records held
    int calls = 0;        // calls held
    int launches = 0;     // launches of the last call
    int held_launches = 0;
    cudaStream_t stream = nullptr;
    Rec rec[BSORT_PROFILE_MAX];

    void begin(int kind, int level) {
        ++launches;
        ++held_launches;
        if (!active || count >= BSORT_PROFILE_MAX) return;
        rec[count].kind = kind;
        rec[count].level = level;
        rec[count].call = calls;
        cudaEventRecord(rec[count].a, stream);
    }
    // Counts kernels of the current group beyond the one begin() counted.
    void more(int kernels) {
        launches += kernels;
        held_launches += kernels;
    }
    void end() {
        if (!active || count >= BSORT_PROFILE_MAX) return;
        cudaEventRecord(rec[count].b, stream);
        ++count;
    }
};

// Per-key-width tuning of the MSD path.
struct MsdShape {
    uint32_t tile;       // keys per scatter tile (threads x items)
    uint32_t chunk;      // keys per chunk (1 or 2 tiles)
    uint32_t unit_cap;   // largest bucket finished in shared memory
    uint32_t merge_cap;  // adjacent small buckets merge up to this many keys
    int levels;          // host-side level launches (ceil(w / radix bits))
    int radix_bits;      // digit width
    uint32_t bins;       // row stride of the per-digit tables (kBins or kWideBins)
};

// Most tiles per chunk (the scatter stages a whole chunk in shared memory).
constexpr int kMaxChunkTiles = 2;

// Runtime tuning of the MSD path (0 fields: defaults).  Digit width 1..11
// bits (the in-place mode caps it at 8; 1 is the paper's one partition per
// bit, kept for measuring what fusing bits saves); finish threshold between 256 keys
// and the compile-time tile; merge threshold between 64 keys and the finish
// threshold; chunk of 1 or 2 scatter tiles.
struct Tuning {
    int radix_bits = 0;
    int unit_keys = 0;
    int merge_keys = 0;
    int chunk_tiles = 0;
};

// false: a field is out of range.
bool tuning_valid(int key_bytes, const Tuning &t);
// kv_bytes: 0 for keys only, else the value bytes of the stable key-value
// sort (4 or 8), which has its own shape (its finish capacity depends on n
// for 4-byte keys with 8-byte values).
MsdShape msd_shape(int key_bytes, const Tuning &t = Tuning(), bool inplace = false, int kv_bytes = 0,
                   uint64_t n = 0);

// Launches the whole MSD pipeline for 4- or 8-byte keys.
template <typename K>
void launch_msd(const Work &wk, cudaStream_t st, Recorder &rec, int num_sms);

// Segmented form: segments [off[s], off[s+1]) (device offsets) are sorted
// independently in one launch sequence.
template <typename K>
void launch_msd_segmented(const Work &wk, const uint64_t *d_offsets, uint32_t nseg, cudaStream_t st, Recorder &rec,
                          int num_sms);

// Stable key-value sort of 4- or 8-byte keys K with 4- or 8-byte values V
// (Work.kv set): values travel with their keys through every level.
template <typename K, typename V>
void launch_msd_kv(const Work &wk, cudaStream_t st, Recorder &rec, int num_sms);

// Sets kernel attributes (call before stream capture).
template <typename K>
void msd_prepare();

// Key-value sorting of 1- and 2-byte keys: wide[i] = the key's order code
// (descending folded in) as a 32-bit word, and back.  One kernel each.
void launch_widen(const void *keys, int key_bytes, uint64_t n, const Codec &codec, uint32_t *wide, cudaStream_t st,
                  int num_sms);
void launch_narrow(const uint32_t *wide, int key_bytes, uint64_t n, const Codec &codec, void *keys, cudaStream_t st,
                   int num_sms);
// dst[i] = src[idx[i]], elements of elem_bytes (1, 2, 4 or 8); an idx entry
// >= n sets kErrBounds in ctl.  One kernel.
void launch_gather(const void *src, int elem_bytes, const uint32_t *idx, uint64_t n, void *dst, Ctl *ctl,
                   cudaStream_t st, int num_sms);

// In-place mode: one level's digit permutation inside the caller's buffer
// (replaces the ping-pong scatter of that level).
constexpr int kIpBlockBytes = 128;                 // block of the permutation
constexpr int kIpSmemCapBytes = 192 * 1024;        // buckets up to this size go through shared memory whole
constexpr uint64_t kIpStripeBytes = 1ull << 20;    // stripe classified by one CTA
template <typename K>
void ip_prepare();
// One bounded device wait on flag_and_err[0] (which nothing sets); the timeout
// lands in flag_and_err[1].
void launch_wait_selftest(uint32_t *flag_and_err, cudaStream_t st);
template <typename K>
void launch_ip_level(const Work &wk, cudaStream_t st, Recorder &rec, int num_sms, int level);

// Counting sort of 1- or 2-byte keys: histogram of all key bits, bin starts,
// and a write-only fill of the output.  Scratch comes from `ws`.
struct CountWork {
    void *keys;
    uint64_t n;
    Codec codec;
    unsigned long long *hist;     // [bins] global counts
    unsigned long long *rstart;   // [bins + 1] output start of each nonempty bin's run, then n
    uint32_t *rval;               // [bins] the nonempty bins, ascending
    uint32_t *nruns;              // number of nonempty bins
    unsigned long long *btot;     // 16-bit: [256] keys of each group of 256 bins
    uint32_t *bnnz;               // 16-bit: [256] nonempty bins of each group
    uint32_t *partial;            // 16-bit: [grid][65536] per-CTA counts
    uint32_t grid16;              // CTAs of the 16-bit histogram (at most one per SM)
};

// Multi-GPU sort of one array: counts[d] += number of keys whose encoded
// top `bits` bits equal d (1 <= bits <= kDigitCountsMaxBits, bits <= key
// bits); `counts` holds 2^bits entries, zeroed by the caller.
constexpr int kDigitCountsMaxBits = 12;
void launch_digit_counts(const void *keys, int key_bytes, uint64_t n, const Codec &codec, int bits,
                         unsigned long long *counts, cudaStream_t st, int num_sms);

void launch_count8(const CountWork &cw, cudaStream_t st, Recorder &rec, int num_sms);
void launch_count16(const CountWork &cw, cudaStream_t st, Recorder &rec, int num_sms);

}  // namespace bsort
