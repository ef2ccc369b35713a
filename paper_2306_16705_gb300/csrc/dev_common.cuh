// Device helpers shared by the kernels: status recording, bitstring words,
// the open-addressing hash table of packed bitstrings.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "hashfn.h"
#include "internal.h"

namespace nnqs {

constexpr uint64_t kEmpty = ~0ull;  // empty slot (all-ones key never occurs: see nnqs_eloc checks)

__device__ __forceinline__ void record_status(DevStatus *st, int code, long long index) {
    if (st == nullptr) return;
    if (atomicCAS(&st->code, 0, code) == 0) st->index = index;
}

template <int W>
struct Bits {
    uint64_t w[W];
};

template <int W>
__device__ __forceinline__ Bits<W> load_bits(const uint64_t *p, int64_t row) {
    Bits<W> b;
    if constexpr (W == 1) {
        b.w[0] = __ldg(p + row);
    } else {
        ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2 *>(p) + row);
        b.w[0] = v.x;
        b.w[1] = v.y;
    }
    return b;
}

template <int W>
__device__ __forceinline__ uint64_t dhash(const Bits<W> &k) {
    if constexpr (W == 1)
        return hash_key1(k.w[0]);
    else
        return hash_key2(k.w[0], k.w[1]);
}

template <int W>
__device__ __forceinline__ int popc_and(const Bits<W> &a, const Bits<W> &b) {
    int c = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) c += __popcll(a.w[w] & b.w[w]);
    return c;
}

__device__ __forceinline__ void cas128(unsigned long long *addr, unsigned long long c0,
                                       unsigned long long c1, unsigned long long v0,
                                       unsigned long long v1, unsigned long long &o0,
                                       unsigned long long &o1) {
    asm volatile(
        "{\n\t.reg .b128 d, c, v;\n\t"
        "mov.b128 c, {%2, %3};\n\t"
        "mov.b128 v, {%4, %5};\n\t"
        "atom.global.cas.b128 d, [%6], c, v;\n\t"
        "mov.b128 {%0, %1}, d;\n\t}"
        : "=l"(o0), "=l"(o1)
        : "l"(c0), "l"(c1), "l"(v0), "l"(v1), "l"(addr)
        : "memory");
}

// Open-addressing table of packed bitstrings -> int32 value, linear probing,
// capacity a power of two, slots [cap][W] (16-byte aligned for W = 2).
template <int W>
struct HashTab {
    uint64_t *keys;
    int32_t *vals;
    uint64_t mask;

    // value of key k, or -1 if absent; at most cap probes
    __device__ __forceinline__ int32_t find(const Bits<W> &k) const {
        uint64_t i = dhash<W>(k) & mask;
        for (uint64_t probe = 0; probe <= mask; ++probe) {
            if constexpr (W == 1) {
                uint64_t v = __ldg(keys + i);
                if (v == k.w[0]) return __ldg(vals + i);
                if (v == kEmpty) return -1;
            } else {
                ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2 *>(keys) + i);
                if (v.x == k.w[0] && v.y == k.w[1]) return __ldg(vals + i);
                if (v.x == kEmpty && v.y == kEmpty) return -1;
            }
            i = (i + 1) & mask;
        }
        return -1;
    }

    // slot of key k after inserting it if absent.  *fresh = true when this
    // call inserted it.  Returns -1 when every slot was probed (table full).
    __device__ __forceinline__ int64_t insert(const Bits<W> &k, bool *fresh) const {
        uint64_t i = dhash<W>(k) & mask;
        for (uint64_t probe = 0; probe <= mask; ++probe) {
            if constexpr (W == 1) {
                unsigned long long old = atomicCAS(reinterpret_cast<unsigned long long *>(keys + i),
                                                   kEmpty, (unsigned long long)k.w[0]);
                if (old == kEmpty) {
                    *fresh = true;
                    return (int64_t)i;
                }
                if (old == k.w[0]) {
                    *fresh = false;
                    return (int64_t)i;
                }
            } else {
                unsigned long long o0, o1;
                cas128(reinterpret_cast<unsigned long long *>(keys + 2 * i), kEmpty, kEmpty, k.w[0],
                       k.w[1], o0, o1);
                if (o0 == kEmpty && o1 == kEmpty) {
                    *fresh = true;
                    return (int64_t)i;
                }
                if (o0 == k.w[0] && o1 == k.w[1]) {
                    *fresh = false;
                    return (int64_t)i;
                }
            }
            i = (i + 1) & mask;
        }
        return -1;
    }
};

inline int64_t pow2_at_least(int64_t v) {
    int64_t c = 1;
    while (c < v) c <<= 1;
    return c;
}

inline unsigned grid_for(int64_t n, int block) { return (unsigned)((n + block - 1) / block); }

}  // namespace nnqs
