// Hash of a packed bitstring (1 or 2 uint64 words), shared by the host
// table builders and the device probes so that tables built on one side are
// probed on the other.  Multiply-xorshift mixing (splitmix64-style finaliser).
#pragma once
#include <stdint.h>

#ifdef __CUDACC__
#define NNQS_HD __host__ __device__ __forceinline__
#else
#define NNQS_HD inline
#endif

namespace nnqs {

NNQS_HD uint64_t mix64(uint64_t h) {
    h ^= h >> 30;
    h *= 0xbf58476d1ce4e5b9ull;
    h ^= h >> 27;
    h *= 0x94d049bb133111ebull;
    h ^= h >> 31;
    return h;
}

NNQS_HD uint64_t hash_key1(uint64_t k0) { return mix64(k0 * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull); }

NNQS_HD uint64_t hash_key2(uint64_t k0, uint64_t k1) {
    return mix64((k0 * 0x9E3779B97F4A7C15ull) ^ (k1 * 0xC2B2AE3D27D4EB4Full) ^ 0x632BE59BD9B4E019ull);
}

}  // namespace nnqs
