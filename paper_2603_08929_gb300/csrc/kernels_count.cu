// Counting path of the bsort library for 1- and 2-byte keys (sm_103a).
//
// With w <= 16 one histogram covers every key bit, so all w bit partitions
// of the method are settled by the counts alone: the output is the encoded
// bins in ascending order, each repeated by its count.  Keys with identical
// bits are indistinguishable, so writing the runs from the counts gives the
// same bytes as moving the keys.  Traffic: one read and one write of n keys.
//
//   count_hist8   256 bins, one shared-memory row per warp
//   count_hist16  65536 bins as packed 16-bit shared-memory counters (128 KB
//                 per CTA, one CTA per SM); a half that wraps is carried into
//                 a global correction word, so counts stay exact at any skew
//   count_reduce  sums the per-CTA 16-bit partials
//   count_scan    exclusive bin starts
//   count_fill    position-driven fill: each CTA owns an output span, finds
//                 the bins overlapping it and writes the decoded values
#include "bsort_launch.h"

namespace bsort {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__host__ __device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }
constexpr int kHist8Threads = 512;
constexpr int kHist16Threads = 1024;
constexpr int kFillThreads = 256;
constexpr int kFillPerThread = 32;  // consecutive output keys per thread
constexpr int kFillSpan = kFillThreads * kFillPerThread;
constexpr int kFillWindow = 4096;   // bin starts staged in shared memory

__global__ void __launch_bounds__(kHist8Threads) k_count_hist8(const uint8_t *keys, uint64_t n, Codec codec,
                                                               unsigned long long *hist) {
    constexpr int WARPS = kHist8Threads / 32;
    __shared__ uint32_t sh[WARPS * 256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < WARPS * 256; i += kHist8Threads) sh[i] = 0;
    __syncthreads();
    uint32_t *row = sh + warp * 256;
    // 16 keys per 16-byte load over the aligned middle, bytes at both ends
    const uintptr_t addr = reinterpret_cast<uintptr_t>(keys);
    uint64_t head = (16 - (addr & 15)) & 15;
    if (head > n) head = n;
    const uint64_t nvec = (n - head) / 16;
    const uint64_t tail0 = head + nvec * 16;
    const uint64_t gtid = blockIdx.x * static_cast<uint64_t>(kHist8Threads) + threadIdx.x;
    const uint64_t gstride = static_cast<uint64_t>(gridDim.x) * kHist8Threads;
    if (gtid < head) atomicAdd(&row[encode_key(keys[gtid], codec)], 1u);
    const uint4 *vec = reinterpret_cast<const uint4 *>(keys + head);
    for (uint64_t v = gtid; v < nvec + (gstride - nvec % gstride) % gstride; v += gstride) {
        const bool valid = v < nvec;
        uint4 q = valid ? vec[v] : make_uint4(0, 0, 0, 0);
        const uint32_t words[4] = {q.x, q.y, q.z, q.w};
        // uniform warp (sorted / constant data): one add per word position
        const uint32_t w0 = __shfl_sync(kFull, words[0], 0);
        const bool same = __all_sync(kFull, valid && words[0] == w0 && words[1] == w0 && words[2] == w0 &&
                                                words[3] == w0 && (w0 & 0xff) * 0x01010101u == w0);
        if (same) {
            if (lane == 0) atomicAdd(&row[encode_key(static_cast<uint8_t>(w0), codec)], 32u * 16u);
        } else if (valid) {
#pragma unroll
            for (int q4 = 0; q4 < 4; ++q4) {
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const uint8_t x = static_cast<uint8_t>(words[q4] >> (8 * b));
                    atomicAdd(&row[encode_key(x, codec)], 1u);
                }
            }
        }
    }
    for (uint64_t i = tail0 + gtid; i < n; i += gstride) atomicAdd(&row[encode_key(keys[i], codec)], 1u);
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += kHist8Threads) {
        uint32_t s = 0;
#pragma unroll
        for (int w = 0; w < WARPS; ++w) s += sh[w * 256 + d];
        if (s) atomicAdd(&hist[d], static_cast<unsigned long long>(s));
    }
}

// Adds c (< 65536) to bin v of the packed counters; a 16-bit half that
// wraps is accounted for in corr[] (global, +-65536 per wrap / borrow).
__device__ __forceinline__ void count_add16(uint32_t *cnt, uint32_t v, uint32_t c, unsigned long long *corr) {
    const uint32_t sh = (v & 1u) * 16u;
    const uint32_t old = atomicAdd(&cnt[v >> 1], c << sh);
    if (((old >> sh) & 0xffffu) + c > 0xffffu) {
        atomicAdd(&corr[v], 65536ull);
        if (sh == 0) {
            // the low half's carry went into the high half: account for a
            // possible wrap there, then take the carry back out
            if ((old >> 16) == 0xffffu) atomicAdd(&corr[v | 1u], 65536ull);
            const uint32_t old2 = atomicSub(&cnt[v >> 1], 1u << 16);
            if ((old2 >> 16) == 0u) atomicAdd(&corr[v | 1u], static_cast<unsigned long long>(-65536ll));
        }
    }
}

__device__ __forceinline__ void count_one16(uint32_t *cnt, uint32_t v, unsigned long long *corr) {
    count_add16(cnt, v, 1u, corr);
}

__global__ void __launch_bounds__(kHist16Threads) k_count_hist16(const uint16_t *keys, uint64_t n, Codec codec,
                                                                 uint32_t *partial, unsigned long long *corr) {
    extern __shared__ uint32_t cnt[];  // 32768 words = 65536 packed 16-bit counters
    const int lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < 32768; i += kHist16Threads) cnt[i] = 0;
    __syncthreads();
    // contiguous slice per CTA
    const uint64_t per = (n + gridDim.x - 1) / gridDim.x;
    const uint64_t b0 = min(n, per * blockIdx.x), b1 = min(n, b0 + per);
    const uint16_t *s = keys;
    const uintptr_t addr = reinterpret_cast<uintptr_t>(s + b0);
    uint64_t head = ((16 - (addr & 15)) & 15) / 2;
    if (head > b1 - b0) head = b1 - b0;
    for (uint64_t i = b0 + threadIdx.x; i < b0 + head; i += kHist16Threads)
        count_one16(cnt, encode_key(s[i], codec), corr);
    const uint64_t m0 = b0 + head;
    const uint64_t nvec = (b1 - m0) / 8;
    const uint4 *vec = reinterpret_cast<const uint4 *>(s + m0);
    const uint64_t rounds = (nvec + kHist16Threads - 1) / kHist16Threads;
    for (uint64_t r = 0; r < rounds; ++r) {
        const uint64_t v = r * kHist16Threads + threadIdx.x;
        const bool valid = v < nvec;
        const uint4 q = valid ? vec[v] : make_uint4(0, 0, 0, 0);
        const uint32_t words[4] = {q.x, q.y, q.z, q.w};
        const uint32_t w0 = __shfl_sync(kFull, words[0], 0);
        const bool same = __all_sync(kFull, valid && words[0] == w0 && words[1] == w0 && words[2] == w0 &&
                                                words[3] == w0 && (w0 & 0xffffu) * 0x10001u == w0);
        if (same) {
            if (lane == 0) {
                const uint32_t e = encode_key(static_cast<uint16_t>(w0), codec);
                count_add16(cnt, e, 256u, corr);  // 32 lanes x 8 keys
            }
        } else if (valid) {
#pragma unroll
            for (int q4 = 0; q4 < 4; ++q4) {
                count_one16(cnt, encode_key(static_cast<uint16_t>(words[q4]), codec), corr);
                count_one16(cnt, encode_key(static_cast<uint16_t>(words[q4] >> 16), codec), corr);
            }
        }
    }
    for (uint64_t i = m0 + nvec * 8 + threadIdx.x; i < b1; i += kHist16Threads)
        count_one16(cnt, encode_key(s[i], codec), corr);
    __syncthreads();
    uint32_t *out = partial + static_cast<size_t>(blockIdx.x) * 65536;
    for (int i = threadIdx.x; i < 32768; i += kHist16Threads) {
        const uint32_t c = cnt[i];
        out[2 * i] = c & 0xffffu;
        out[2 * i + 1] = c >> 16;
    }
}

__global__ void k_count_reduce16(const uint32_t *partial, int grid, const unsigned long long *corr,
                                 unsigned long long *hist) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= 65536) return;
    unsigned long long s = corr[v];
    for (int g = 0; g < grid; ++g) s += partial[static_cast<size_t>(g) * 65536 + v];
    hist[v] = s;
}

// Exclusive starts of `bins` counts (one CTA of 1024 threads).
__global__ void __launch_bounds__(1024) k_count_scan(const unsigned long long *hist, int bins,
                                                     unsigned long long *starts) {
    __shared__ unsigned long long part[1024];
    const int per = (bins + 1023) / 1024;
    const int b0 = threadIdx.x * per;
    unsigned long long s = 0;
    for (int i = 0; i < per && b0 + i < bins; ++i) s += hist[b0 + i];
    part[threadIdx.x] = s;
    __syncthreads();
    // Hillis-Steele inclusive scan over 1024 partial sums
    for (int o = 1; o < 1024; o <<= 1) {
        const unsigned long long add = threadIdx.x >= o ? part[threadIdx.x - o] : 0ull;
        __syncthreads();
        part[threadIdx.x] += add;
        __syncthreads();
    }
    unsigned long long run = threadIdx.x ? part[threadIdx.x - 1] : 0ull;
    for (int i = 0; i < per && b0 + i < bins; ++i) {
        starts[b0 + i] = run;
        run += hist[b0 + i];
    }
    if (threadIdx.x == 1023) starts[bins] = part[1023];
}

// Largest bin b with starts[b] <= p among [lo, hi] (starts non-decreasing,
// starts[lo] <= p).
__device__ __forceinline__ int bin_of(const unsigned long long *starts, int lo, int hi, unsigned long long p) {
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (starts[mid] <= p) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <typename K>
__global__ void __launch_bounds__(kFillThreads) k_count_fill(K *keys, uint64_t n, const unsigned long long *starts,
                                                             int bins, Codec codec) {
    __shared__ unsigned long long win[kFillWindow + 1];
    __shared__ int sh_v[2];
    const uint64_t nspan = (n + kFillSpan - 1) / kFillSpan;
    for (uint64_t sp = blockIdx.x; sp < nspan; sp += gridDim.x) {
        const uint64_t p0 = sp * kFillSpan;
        const uint64_t p1 = min(n, p0 + kFillSpan);
        if (threadIdx.x == 0) {
            sh_v[0] = bin_of(starts, 0, bins - 1, p0);
            sh_v[1] = bin_of(starts, 0, bins - 1, p1 - 1);
        }
        __syncthreads();
        const int v0 = sh_v[0], v1 = sh_v[1];
        const bool windowed = v1 - v0 + 2 <= kFillWindow + 1;
        if (windowed)
            for (int i = threadIdx.x; i <= v1 - v0 + 1; i += kFillThreads) win[i] = starts[v0 + i];
        __syncthreads();
        const uint64_t q0 = p0 + static_cast<uint64_t>(threadIdx.x) * kFillPerThread;
        if (q0 < p1) {
            int v = windowed ? v0 + bin_of(win, 0, v1 - v0, q0) : bin_of(starts, v0, v1, q0);
            unsigned long long next = windowed ? win[v - v0 + 1] : starts[v + 1];
            const int cnt = static_cast<int>(umin64(kFillPerThread, p1 - q0));
            K vals[kFillPerThread];
#pragma unroll
            for (int i = 0; i < kFillPerThread; ++i) {
                const uint64_t p = q0 + i;
                while (p >= next && v < bins - 1) {
                    ++v;
                    next = windowed ? win[v - v0 + 1] : starts[v + 1];
                }
                vals[i] = decode_key(static_cast<K>(v), codec);
            }
            K *dst = keys + q0;
            constexpr int kVec = 16 / sizeof(K);
            if (cnt == kFillPerThread && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
#pragma unroll
                for (int i = 0; i < kFillPerThread; i += kVec) {
                    uint4 q;
                    memcpy(&q, &vals[i], 16);
                    *reinterpret_cast<uint4 *>(dst + i) = q;
                }
            } else {
                for (int i = 0; i < cnt; ++i) dst[i] = vals[i];
            }
        }
        __syncthreads();
    }
}

}  // namespace

void launch_count8(const CountWork &cw, cudaStream_t st, Recorder &rec, int num_sms) {
    rec.begin(BSORT_K_COUNT_HIST, -1);
    cudaMemsetAsync(cw.hist, 0, 256 * sizeof(unsigned long long), st);
    const uint64_t vec = cw.n / 16 + 1;
    const int grid = static_cast<int>(umin64(static_cast<uint64_t>(num_sms) * 4,
                                                    (vec + kHist8Threads - 1) / kHist8Threads));
    k_count_hist8<<<max(grid, 1), kHist8Threads, 0, st>>>(static_cast<const uint8_t *>(cw.keys), cw.n, cw.codec,
                                                          cw.hist);
    rec.end();
    rec.begin(BSORT_K_COUNT_SCAN, -1);
    k_count_scan<<<1, 1024, 0, st>>>(cw.hist, 256, cw.starts);
    rec.end();
    rec.begin(BSORT_K_COUNT_FILL, -1);
    const uint64_t spans = (cw.n + kFillSpan - 1) / kFillSpan;
    const int fgrid = static_cast<int>(umin64(static_cast<uint64_t>(num_sms) * 8, spans));
    k_count_fill<uint8_t><<<max(fgrid, 1), kFillThreads, 0, st>>>(static_cast<uint8_t *>(cw.keys), cw.n, cw.starts,
                                                                  256, cw.codec);
    rec.end();
}

void launch_count16(const CountWork &cw, cudaStream_t st, Recorder &rec, int num_sms) {
    static const bool attr_set = [] {  // once per process; thread-safe static initialisation
        cudaFuncSetAttribute(k_count_hist16, cudaFuncAttributeMaxDynamicSharedMemorySize, 32768 * 4);
        return true;
    }();
    (void)attr_set;
    rec.begin(BSORT_K_COUNT_HIST, -1);
    unsigned long long *corr = cw.hist;  // corrections accumulate in place, the reduce overwrites
    cudaMemsetAsync(corr, 0, 65536 * sizeof(unsigned long long), st);
    k_count_hist16<<<cw.grid16, kHist16Threads, 32768 * 4, st>>>(static_cast<const uint16_t *>(cw.keys), cw.n,
                                                                 cw.codec, cw.partial, corr);
    k_count_reduce16<<<256, 256, 0, st>>>(cw.partial, static_cast<int>(cw.grid16), corr, cw.hist);
    rec.more(1);
    rec.end();
    rec.begin(BSORT_K_COUNT_SCAN, -1);
    k_count_scan<<<1, 1024, 0, st>>>(cw.hist, 65536, cw.starts);
    rec.end();
    rec.begin(BSORT_K_COUNT_FILL, -1);
    const uint64_t spans = (cw.n + kFillSpan - 1) / kFillSpan;
    const int fgrid = static_cast<int>(umin64(static_cast<uint64_t>(num_sms) * 8, spans));
    k_count_fill<uint16_t><<<max(fgrid, 1), kFillThreads, 0, st>>>(static_cast<uint16_t *>(cw.keys), cw.n,
                                                                   cw.starts, 65536, cw.codec);
    rec.end();
    (void)num_sms;
}

}  // namespace bsort
