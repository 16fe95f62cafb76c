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
//   count_runs    the nonempty bins in ascending order with their output
//                 starts (256 bins per CTA)
//   count_fill    position-driven fill: each CTA owns an output span, finds
//                 the runs overlapping it and writes the decoded values
#include "bsort_launch.h"

namespace bsort {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__host__ __device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }
constexpr int kHist8Threads = 512;
constexpr int kHist16Threads = 1024;
constexpr int kFillThreads = 256;
// Output span of one fill step: a multiple of kFillThreads 16-byte vectors,
// sized so that each CTA gets about two spans (few per-span searches and
// barriers per byte written), at least kFillMinVecs vectors per thread.
constexpr int kFillMinVecs = 4;
constexpr int kFillWindow = 2048;   // run starts and values staged in shared memory

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
    // eight keys of one 16-byte vector (valid: the vector is in range); a
    // warp whose 32 vectors hold one repeated key adds 256 with one atomic
    auto count_vec = [&](const uint4 q, bool valid) {
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
    };
    // whole rounds of U vectors per thread: U loads in flight before counting
    constexpr int U = 4;
    constexpr uint64_t kRound = static_cast<uint64_t>(U) * kHist16Threads;
    uint64_t base = 0;
    for (; base + kRound <= nvec; base += kRound) {
        uint4 q[U];
#pragma unroll
        for (int u = 0; u < U; ++u) q[u] = __ldcs(vec + base + u * kHist16Threads + threadIdx.x);
#pragma unroll
        for (int u = 0; u < U; ++u) count_vec(q[u], true);
    }
    for (; base < nvec; base += kHist16Threads) {  // the rest, one vector per thread (trip count block-uniform)
        const uint64_t v = base + threadIdx.x;
        const bool valid = v < nvec;
        count_vec(valid ? __ldcs(vec + v) : make_uint4(0, 0, 0, 0), valid);
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

// Count of bin v = corr[v] + the CTAs' partials (256 CTAs x 256 bins), and
// per CTA the keys and the nonempty bins of its 256 bins.
constexpr int kRunThreads = 256;  // bins per CTA of the reduce and run kernels
__global__ void __launch_bounds__(kRunThreads) k_count_reduce16(const uint32_t *partial, int grid,
                                                                const unsigned long long *corr,
                                                                unsigned long long *hist,
                                                                unsigned long long *btot, uint32_t *bnnz) {
    __shared__ unsigned long long ws_c[kRunThreads / 32];
    __shared__ uint32_t ws_z[kRunThreads / 32];
    const int v = blockIdx.x * kRunThreads + threadIdx.x;  // the grid covers the 65536 bins exactly
    unsigned long long s = corr[v];
    int g = 0;
    for (; g + 4 <= grid; g += 4) {
        const uint32_t a = partial[static_cast<size_t>(g) * 65536 + v];
        const uint32_t b = partial[static_cast<size_t>(g + 1) * 65536 + v];
        const uint32_t c = partial[static_cast<size_t>(g + 2) * 65536 + v];
        const uint32_t d = partial[static_cast<size_t>(g + 3) * 65536 + v];
        s += static_cast<unsigned long long>(a) + b + c + d;
    }
    for (; g < grid; ++g) s += partial[static_cast<size_t>(g) * 65536 + v];
    hist[v] = s;
    unsigned long long c = s;
    uint32_t z = s != 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        c += __shfl_xor_sync(kFull, c, o);
        z += __shfl_xor_sync(kFull, z, o);
    }
    if ((threadIdx.x & 31) == 0) {
        ws_c[threadIdx.x >> 5] = c;
        ws_z[threadIdx.x >> 5] = z;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long tc = 0;
        uint32_t tz = 0;
        for (int w = 0; w < kRunThreads / 32; ++w) {
            tc += ws_c[w];
            tz += ws_z[w];
        }
        btot[blockIdx.x] = tc;
        bnnz[blockIdx.x] = tz;
    }
}

// The output as runs: run r holds `count` copies of bin rval[r] starting at
// rstart[r], for the nonempty bins in ascending order; rstart[nruns] = n and
// *nruns the number of runs.  CTA b owns bins [256 b, 256 b + 256): it sums
// the keys and nonempty bins of the CTAs before it from the reduce's
// per-CTA totals (btot / bnnz; a single CTA needs none), then scans its own.
__global__ void __launch_bounds__(kRunThreads) k_count_runs(const unsigned long long *hist,
                                                            const unsigned long long *btot, const uint32_t *bnnz,
                                                            unsigned long long *rstart, uint32_t *rval,
                                                            uint32_t *nruns) {
    __shared__ unsigned long long red_c[kRunThreads / 32], sc_c[kRunThreads / 32];
    __shared__ uint32_t red_z[kRunThreads / 32], sc_z[kRunThreads / 32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    // keys and runs of the bins before this CTA (one earlier CTA per thread)
    unsigned long long c_before = t < static_cast<int>(blockIdx.x) ? btot[t] : 0ull;
    uint32_t z_before = t < static_cast<int>(blockIdx.x) ? bnnz[t] : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        c_before += __shfl_xor_sync(kFull, c_before, o);
        z_before += __shfl_xor_sync(kFull, z_before, o);
    }
    if (lane == 0) {
        red_c[warp] = c_before;
        red_z[warp] = z_before;
    }
    // this CTA's bins: inclusive warp scans of counts and of nonempty flags
    const int v = blockIdx.x * kRunThreads + t;
    const unsigned long long c = hist[v];
    unsigned long long x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    const unsigned mask = __ballot_sync(kFull, c != 0);
    if (lane == 31) {
        sc_c[warp] = x;
        sc_z[warp] = __popc(mask);
    }
    __syncthreads();
    unsigned long long base_c = 0, all_c = 0;
    uint32_t base_z = 0, all_z = 0;
#pragma unroll
    for (int w = 0; w < kRunThreads / 32; ++w) {
        base_c += red_c[w];
        base_z += red_z[w];
        if (w < warp) {
            base_c += sc_c[w];
            base_z += sc_z[w];
        }
        all_c += sc_c[w];
        all_z += sc_z[w];
    }
    if (c) {
        const uint32_t r = base_z + __popc(mask & ((1u << lane) - 1u));
        rstart[r] = base_c + x - c;
        rval[r] = static_cast<uint32_t>(v);
    }
    if (blockIdx.x == gridDim.x - 1 && t == kRunThreads - 1) {
        // the last CTA knows every count: close the run list
        unsigned long long total = 0;
        uint32_t runs = 0;
        for (int w = 0; w < kRunThreads / 32; ++w) {
            total += red_c[w];
            runs += red_z[w];
        }
        total += all_c;
        runs += all_z;
        rstart[runs] = total;
        *nruns = runs;
    }
}

// The same search by a whole warp: 32 probes per round cut [lo, hi] 32-fold
// (four rounds over 65536 entries).  Every lane returns the index.
__device__ __forceinline__ int bin_of_warp(const unsigned long long *starts, int lo, int hi, unsigned long long p) {
    const int lane = threadIdx.x & 31;
    while (lo < hi) {
        const int step = (hi - lo + 31) / 32;                    // >= 1
        const int probe = lo + (lane + 1) * step;
        const bool ok = probe <= hi && starts[probe] <= p;       // a prefix of the lanes (starts non-decreasing)
        const int k = __popc(__ballot_sync(kFull, ok));
        lo += k * step;
        hi = min(hi, lo + step - 1);
    }
    return lo;
}

// Largest index b with starts[b] <= p among [lo, hi] (starts non-decreasing,
// starts[lo] <= p).
__device__ __forceinline__ int bin_of(const unsigned long long *starts, int lo, int hi, unsigned long long p) {
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (starts[mid] <= p) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Position-driven fill from the runs: each CTA takes output spans of `span`
// keys; warps 0 and 1 find the runs holding the span's first and last key
// (warp search), and the runs' starts and values between them go to shared
// memory when they fit.  The span is written as 16-byte vectors, vector j by
// thread j mod kFillThreads, so each warp store covers 512 contiguous bytes;
// a thread's vectors come in increasing order, so the run of each vector's
// first key is searched from the thread's previous run on, and the other
// keys step through the (nonempty) runs they cross.
template <typename K>
__global__ void __launch_bounds__(kFillThreads) k_count_fill(K *keys, uint64_t n, const unsigned long long *rstart,
                                                             const uint32_t *rval, const uint32_t *nruns_p,
                                                             uint32_t span, Codec codec) {
    __shared__ unsigned long long win[kFillWindow + 1];
    __shared__ uint32_t wval[kFillWindow + 1];
    __shared__ int sh_r[2];
    constexpr int kVec = 16 / sizeof(K);
    const int nr = static_cast<int>(*nruns_p);
    const bool vec_ok = (reinterpret_cast<uintptr_t>(keys) & 15) == 0;  // spans start at multiples of kVec keys
    const uint64_t nspan = (n + span - 1) / span;
    for (uint64_t sp = blockIdx.x; sp < nspan; sp += gridDim.x) {
        const uint64_t p0 = sp * span;
        const uint64_t p1 = min(n, p0 + span);
        if (threadIdx.x < 64) {  // warp 0: the run of the span's first key, warp 1: of its last
            const int r = bin_of_warp(rstart, 0, nr - 1, threadIdx.x < 32 ? p0 : p1 - 1);
            if ((threadIdx.x & 31) == 0) sh_r[threadIdx.x >> 5] = r;
        }
        __syncthreads();
        const int r0 = sh_r[0], r1 = sh_r[1];
        const bool windowed = r1 - r0 + 2 <= kFillWindow + 1;
        if (windowed)
            for (int i = threadIdx.x; i <= r1 - r0 + 1; i += kFillThreads) {
                win[i] = rstart[r0 + i];
                wval[i] = i <= r1 - r0 ? rval[r0 + i] : 0u;
            }
        __syncthreads();
        int r_prev = r0;
        for (uint32_t j = threadIdx.x; j < span / kVec; j += kFillThreads) {
            const uint64_t p = p0 + static_cast<uint64_t>(j) * kVec;
            if (p >= p1) break;  // later vectors of this thread start later still
            const unsigned long long prev_end = windowed ? win[r_prev - r0 + 1] : rstart[r_prev + 1];
            int r = p < prev_end ? r_prev  // still inside the thread's previous run
                    : (windowed ? r0 + bin_of(win, r_prev - r0, r1 - r0, p) : bin_of(rstart, r_prev, r1, p));
            unsigned long long next = windowed ? win[r - r0 + 1] : rstart[r + 1];
            K val = decode_key(static_cast<K>(windowed ? wval[r - r0] : rval[r]), codec);
            auto value_at = [&](uint64_t q) {
                while (q >= next) {  // runs are nonempty: one step per run crossed
                    ++r;
                    next = windowed ? win[r - r0 + 1] : rstart[r + 1];
                    val = decode_key(static_cast<K>(windowed ? wval[r - r0] : rval[r]), codec);
                }
                return val;
            };
            const int cnt = static_cast<int>(umin64(kVec, p1 - p));
            if (vec_ok && cnt == kVec && p + kVec <= next) {  // the whole vector inside one run
                const uint32_t v32 = static_cast<uint32_t>(val) * (sizeof(K) == 1 ? 0x01010101u : 0x00010001u);
                *reinterpret_cast<uint4 *>(keys + p) = make_uint4(v32, v32, v32, v32);
            } else if (vec_ok && cnt == kVec) {
                K vals[kVec];
#pragma unroll
                for (int e = 0; e < kVec; ++e) vals[e] = value_at(p + e);
                uint4 q;
                memcpy(&q, vals, 16);
                *reinterpret_cast<uint4 *>(keys + p) = q;
            } else {
                for (int e = 0; e < cnt; ++e) keys[p + e] = value_at(p + e);
            }
            r_prev = r;
        }
        __syncthreads();
    }
}

// One fill launch: 8 CTAs per SM, spans of ~n / (2 * CTAs) keys (a whole
// number of kFillThreads vectors, at least kFillMinVecs per thread).
template <typename K>
void launch_fill(const CountWork &cw, cudaStream_t st, int num_sms) {
    constexpr uint64_t kVec = 16 / sizeof(K);
    constexpr uint64_t unit = kFillThreads * kVec;
    const uint64_t ctas = static_cast<uint64_t>(num_sms) * 8;
    uint64_t span = (cw.n + 2 * ctas - 1) / (2 * ctas);
    span = (span + unit - 1) / unit * unit;
    if (span < kFillMinVecs * unit) span = kFillMinVecs * unit;
    if (span > (1u << 30)) span = 1u << 30;
    const uint64_t spans = (cw.n + span - 1) / span;
    const int fgrid = static_cast<int>(umin64(ctas, spans));
    k_count_fill<K><<<max(fgrid, 1), kFillThreads, 0, st>>>(static_cast<K *>(cw.keys), cw.n, cw.rstart, cw.rval,
                                                           cw.nruns, static_cast<uint32_t>(span), cw.codec);
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
    k_count_runs<<<1, kRunThreads, 0, st>>>(cw.hist, nullptr, nullptr, cw.rstart, cw.rval, cw.nruns);
    rec.end();
    rec.begin(BSORT_K_COUNT_FILL, -1);
    launch_fill<uint8_t>(cw, st, num_sms);
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
    k_count_reduce16<<<65536 / kRunThreads, kRunThreads, 0, st>>>(cw.partial, static_cast<int>(cw.grid16), corr,
                                                                   cw.hist, cw.btot, cw.bnnz);
    rec.more(1);
    rec.end();
    rec.begin(BSORT_K_COUNT_SCAN, -1);
    k_count_runs<<<65536 / kRunThreads, kRunThreads, 0, st>>>(cw.hist, cw.btot, cw.bnnz, cw.rstart, cw.rval,
                                                               cw.nruns);
    rec.end();
    rec.begin(BSORT_K_COUNT_FILL, -1);
    launch_fill<uint16_t>(cw, st, num_sms);
    rec.end();
    (void)num_sms;
}

}  // namespace bsort
