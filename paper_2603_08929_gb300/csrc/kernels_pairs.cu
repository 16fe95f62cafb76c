// Key-value sorting around the 8-byte MSD pipeline.
//
// A stable key-value sort is a sort of distinct words: each key's
// order-preserving code (the same encode_key as the key sort, descending
// folded in) goes to the high half of a 64-bit word and its input position to
// the low half.  Positions make every word unique, so the unstable digit
// passes of the 8-byte pipeline give exactly the stable order.  8-byte keys
// take two such sorts over the halves of their code, low half first (LSD
// order): the second sort's low half is the position in the first sort's
// output, which orders ties of the high half by the low half and then by the
// input position.  The kernels here build the words, turn sorted words into
// input positions, and gather keys and values along them; all are
// grid-stride loops over n (memory-bound, one pass each).
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

// word[i] = code << 32 | i, code = encode(keys[src]) (its low or high 32 bits
// for 8-byte keys; part 0 / 1), src = i or perm[i].  A perm entry >= n is
// refused (bit kErrBounds into *err, key 0 read instead).
template <typename K>
__global__ void __launch_bounds__(kPairThreads) k_pairs_pack(const K *__restrict__ keys, uint64_t n, Codec codec,
                                                             int part, const uint32_t *__restrict__ perm,
                                                             uint64_t *__restrict__ words, uint32_t *err) {
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < n; i += stride) {
        uint64_t src = i;
        if (perm) {
            src = perm[i];
            if (src >= n) {
                atomicOr(err, kErrBounds);
                src = 0;
            }
        }
        const uint64_t k = static_cast<uint64_t>(encode_key(keys[src], codec));
        const uint64_t code = sizeof(K) <= 4 ? k : (part == 0 ? (k & 0xffffffffull) : (k >> 32));
        words[i] = (code << 32) | i;
    }
}

// perm[i] = low half of word[i]; thread 0 also keeps the sort's error bits
// (the next sort clears its control block).
__global__ void __launch_bounds__(kPairThreads) k_pairs_perm(const uint64_t *__restrict__ words, uint64_t n,
                                                             uint32_t *__restrict__ perm, const Ctl *ctl,
                                                             uint32_t *err) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && ctl->error) atomicOr(err, ctl->error);
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < n; i += stride)
        perm[i] = static_cast<uint32_t>(words[i]);
}

// Input position of output element i: the low half of the sorted word (then
// through perm for 8-byte keys).  Writes idx[i], indices[i] (if requested)
// and, for keys of at most 4 bytes, the sorted key itself (decoded from the
// high half).  Folds the earlier error bits into the control block.
template <typename K>
__global__ void __launch_bounds__(kPairThreads) k_pairs_index(const uint64_t *__restrict__ words,
                                                              const uint32_t *__restrict__ perm, uint64_t n,
                                                              K *__restrict__ keys, Codec codec,
                                                              uint32_t *__restrict__ idx, int64_t *__restrict__ indices,
                                                              Ctl *ctl, const uint32_t *err) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && *err) set_error(ctl, *err);
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < n; i += stride) {
        const uint64_t w = words[i];
        uint64_t src = static_cast<uint32_t>(w);
        if (perm) src = src < n ? perm[src] : n;
        if (src >= n) {
            set_error(ctl, kErrBounds);
            src = 0;
        }
        if (idx) idx[i] = static_cast<uint32_t>(src);
        if (indices) indices[i] = static_cast<int64_t>(src);
        if (keys) keys[i] = decode_key(static_cast<K>(w >> 32), codec);
    }
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

void launch_pairs_pack(const void *keys, int key_bytes, uint64_t n, const Codec &codec, int part,
                       const uint32_t *perm, uint64_t *words, uint32_t *err, cudaStream_t st, int num_sms) {
    const int g = pairs_grid(n, num_sms);
    switch (key_bytes) {
    case 1: k_pairs_pack<uint8_t><<<g, kPairThreads, 0, st>>>(static_cast<const uint8_t *>(keys), n, codec, part, perm, words, err); break;
    case 2: k_pairs_pack<uint16_t><<<g, kPairThreads, 0, st>>>(static_cast<const uint16_t *>(keys), n, codec, part, perm, words, err); break;
    case 4: k_pairs_pack<uint32_t><<<g, kPairThreads, 0, st>>>(static_cast<const uint32_t *>(keys), n, codec, part, perm, words, err); break;
    default: k_pairs_pack<uint64_t><<<g, kPairThreads, 0, st>>>(static_cast<const uint64_t *>(keys), n, codec, part, perm, words, err); break;
    }
}

void launch_pairs_perm(const uint64_t *words, uint64_t n, uint32_t *perm, const Ctl *ctl, uint32_t *err,
                       cudaStream_t st, int num_sms) {
    k_pairs_perm<<<pairs_grid(n, num_sms), kPairThreads, 0, st>>>(words, n, perm, ctl, err);
}

void launch_pairs_index(const uint64_t *words, const uint32_t *perm, uint64_t n, void *keys, int key_bytes,
                        const Codec &codec, uint32_t *idx, int64_t *indices, Ctl *ctl, const uint32_t *err,
                        cudaStream_t st, int num_sms) {
    const int g = pairs_grid(n, num_sms);
    switch (key_bytes) {
    case 1: k_pairs_index<uint8_t><<<g, kPairThreads, 0, st>>>(words, perm, n, static_cast<uint8_t *>(keys), codec, idx, indices, ctl, err); break;
    case 2: k_pairs_index<uint16_t><<<g, kPairThreads, 0, st>>>(words, perm, n, static_cast<uint16_t *>(keys), codec, idx, indices, ctl, err); break;
    case 4: k_pairs_index<uint32_t><<<g, kPairThreads, 0, st>>>(words, perm, n, static_cast<uint32_t *>(keys), codec, idx, indices, ctl, err); break;
    default: k_pairs_index<uint64_t><<<g, kPairThreads, 0, st>>>(words, perm, n, static_cast<uint64_t *>(keys), codec, idx, indices, ctl, err); break;
    }
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
