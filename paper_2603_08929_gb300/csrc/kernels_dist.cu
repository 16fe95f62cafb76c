// Digit counts for the multi-GPU sort of one array: how many keys of a shard
// fall in each value of the top `bits` bits of their sort-order code.  The
// code is the library's order-preserving encoding (Sec. III's direction
// rules for the sign and the negative float half), so digit d's keys precede
// digit d+1's in the sorted output and prefix sums of the counts are output
// positions; ranks assign themselves contiguous digit ranges from them.
#include "bsort_launch.h"

namespace bsort {

namespace {

// One shared counter row per CTA (at most 2^12 bins), flushed with one
// global atomic per nonempty bin.  The 16-byte-aligned middle of the array
// is read as vectors, the ragged ends key by key.
template <typename K>
__global__ void __launch_bounds__(256) k_digit_counts(const K *__restrict__ keys, uint64_t n, Codec codec, int shift,
                                                      uint32_t nbins, unsigned long long *__restrict__ counts,
                                                      bool vec_ok) {
    constexpr int V = 16 / static_cast<int>(sizeof(K));
    __shared__ uint32_t h[1u << kDigitCountsMaxBits];
    for (uint32_t i = threadIdx.x; i < nbins; i += blockDim.x) h[i] = 0;
    __syncthreads();
    auto one = [&](K k) {
        const K e = encode_key(k, codec);
        atomicAdd(&h[static_cast<uint32_t>(static_cast<uint64_t>(e) >> shift)], 1u);
    };
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    const uint64_t tid = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    uint64_t m0 = 0, m1 = 0;  // aligned middle [m0, m1)
    if (vec_ok) {
        m0 = (V - reinterpret_cast<uintptr_t>(keys) / sizeof(K) % V) % V;
        if (m0 > n) m0 = n;
        m1 = m0 + (n - m0) / V * V;
    }
    for (uint64_t i = tid; i < m0; i += stride) one(keys[i]);
    for (uint64_t i = m1 + tid; i < n; i += stride) one(keys[i]);
    const uint4 *vec = reinterpret_cast<const uint4 *>(keys + m0);
    const uint64_t nvec = (m1 - m0) / V;
    for (uint64_t q = tid; q < nvec; q += stride) {
        const uint4 v = __ldcs(vec + q);
        K kk[V];
        memcpy(kk, &v, 16);
#pragma unroll
        for (int e = 0; e < V; ++e) one(kk[e]);
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < nbins; i += blockDim.x)
        if (h[i]) atomicAdd(&counts[i], static_cast<unsigned long long>(h[i]));
}

}  // namespace

void launch_digit_counts(const void *keys, int key_bytes, uint64_t n, const Codec &codec, int bits,
                         unsigned long long *counts, cudaStream_t st, int num_sms) {
    const int shift = key_bytes * 8 - bits;
    const uint32_t nbins = 1u << bits;
    const bool vec_ok = true;  // the kernel finds the aligned middle itself
    uint64_t blocks = (n + 256 * 16 - 1) / (256 * 16);
    if (blocks > static_cast<uint64_t>(num_sms) * 8) blocks = static_cast<uint64_t>(num_sms) * 8;
    if (blocks < 1) blocks = 1;
    const dim3 grid(static_cast<unsigned>(blocks));
    switch (key_bytes) {
        case 1:
            k_digit_counts<uint8_t><<<grid, 256, 0, st>>>(static_cast<const uint8_t *>(keys), n, codec, shift, nbins,
                                                         counts, vec_ok);
            break;
        case 2:
            k_digit_counts<uint16_t><<<grid, 256, 0, st>>>(static_cast<const uint16_t *>(keys), n, codec, shift,
                                                          nbins, counts, vec_ok);
            break;
        case 4:
            k_digit_counts<uint32_t><<<grid, 256, 0, st>>>(static_cast<const uint32_t *>(keys), n, codec, shift,
                                                          nbins, counts, vec_ok);
            break;
        default:
            k_digit_counts<uint64_t><<<grid, 256, 0, st>>>(static_cast<const uint64_t *>(keys), n, codec, shift,
                                                          nbins, counts, vec_ok);
            break;
    }
}

}  // namespace bsort
