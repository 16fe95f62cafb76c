// Key-value sorting helpers around the value-carrying MSD pipeline: the
// widening of 1- and 2-byte keys to 32-bit order codes and back, and the
// gather of values along sorted input positions.  All are grid-stride loops
// over n (memory-bound, one pass each).
#include "bsort_device.cuh"
#include "bsort_launch.h"

namespace bsort {
namespace {

constexpr int kPairThreads = 256;

__host__ __device__ inline int pairs_grid(uint64_t n, int num_sms) {
    const uint64_t want = (n + kPairThreads - 1) / kPairThreads;
    const uint64_t cap = static_cast<uint64_t>(num_sms) * 8;
    return static_cast<int>(want < cap ? (want ? want : 1) : cap);
}

// wide[i] = the order code of keys[i] (encode_key, descending folded in),
// zero-extended: the 32-bit words sort, as unsigned integers, in the keys'
// order, equal keys to equal words.
template <typename K>
__global__ void __launch_bounds__(kPairThreads) k_widen(const K *__restrict__ keys, uint64_t n, Codec codec,
                                                        uint32_t *__restrict__ wide) {
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < n; i += stride)
        wide[i] = static_cast<uint32_t>(encode_key(keys[i], codec));
}

// keys[i] = the key whose order code wide[i] holds (its low bits).
template <typename K>
__global__ void __launch_bounds__(kPairThreads) k_narrow(const uint32_t *__restrict__ wide, uint64_t n, Codec codec,
                                                         K *__restrict__ keys) {
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < n; i += stride)
        keys[i] = decode_key(static_cast<K>(wide[i]), codec);
}

// dst[i] = src[idx[i]] (idx < n by construction; a larger entry is refused).
// The reads are random, so each thread keeps eight of them in flight: two
// 16-byte loads of positions, then eight independent element loads (idx is
// 16-byte aligned: it starts a workspace region).
template <typename T>
__global__ void __launch_bounds__(kPairThreads) k_gather(const T *__restrict__ src, const uint32_t *__restrict__ idx,
                                                         uint64_t n, T *__restrict__ dst, Ctl *ctl) {
    constexpr int E = 8;
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    const uint64_t tid = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
    const uint64_t groups = n / E;
    bool bad = false;
    for (uint64_t g = tid; g < groups; g += stride) {
        const uint4 a = reinterpret_cast<const uint4 *>(idx)[2 * g];
        const uint4 b = reinterpret_cast<const uint4 *>(idx)[2 * g + 1];
        uint32_t j[E] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
        T v[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            bad |= j[e] >= n;
            v[e] = src[j[e] < n ? j[e] : 0];
        }
#pragma unroll
        for (int e = 0; e < E; ++e) dst[g * E + e] = v[e];
    }
    for (uint64_t i = groups * E + tid; i < n; i += stride) {
        const uint32_t j = idx[i];
        bad |= j >= n;
        dst[i] = src[j < n ? j : 0];
    }
    if (bad) set_error(ctl, kErrBounds);
}

}  // namespace

void launch_widen(const void *keys, int key_bytes, uint64_t n, const Codec &codec, uint32_t *wide, cudaStream_t st,
                  int num_sms) {
    const int g = pairs_grid(n, num_sms);
    if (key_bytes == 1) k_widen<uint8_t><<<g, kPairThreads, 0, st>>>(static_cast<const uint8_t *>(keys), n, codec, wide);
    else k_widen<uint16_t><<<g, kPairThreads, 0, st>>>(static_cast<const uint16_t *>(keys), n, codec, wide);
}

void launch_narrow(const uint32_t *wide, int key_bytes, uint64_t n, const Codec &codec, void *keys, cudaStream_t st,
                   int num_sms) {
    const int g = pairs_grid(n, num_sms);
    if (key_bytes == 1) k_narrow<uint8_t><<<g, kPairThreads, 0, st>>>(wide, n, codec, static_cast<uint8_t *>(keys));
    else k_narrow<uint16_t><<<g, kPairThreads, 0, st>>>(wide, n, codec, static_cast<uint16_t *>(keys));
}

void launch_gather(const void *src, int elem_bytes, const uint32_t *idx, uint64_t n, void *dst, Ctl *ctl,
                   cudaStream_t st, int num_sms) {
    const int g = pairs_grid(n, num_sms);
    switch (elem_bytes) {
    case 1: k_gather<uint8_t><<<g, kPairThreads, 0, st>>>(static_cast<const uint8_t *>(src), idx, n, static_cast<uint8_t *>(dst), ctl); break;
    case 2: k_gather<uint16_t><<<g, kPairThreads, 0, st>>>(static_cast<const uint16_t *>(src), idx, n, static_cast<uint16_t *>(dst), ctl); break;
    case 4: k_gather<uint32_t><<<g, kPairThreads, 0, st>>>(static_cast<const uint32_t *>(src), idx, n, static_cast<uint32_t *>(dst), ctl); break;
    default: k_gather<uint64_t><<<g, kPairThreads, 0, st>>>(static_cast<const uint64_t *>(src), idx, n, static_cast<uint64_t *>(dst), ctl); break;
    }
}

}  // namespace bsort
