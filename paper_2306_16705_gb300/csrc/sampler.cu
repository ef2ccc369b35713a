// Batch autoregressive sampling (BAS, Sec. 3.1, Fig. bas(b)) with the
// number mask of Sec. 3.3.
//
// The tree of unique prefixes is kept level by level on the device: a level
// is a list of prefixes (packed bitstrings with the first t tokens set) and
// their sample counts.  A step runs the ansatz on every prefix to get
// pi~(. | prefix) -- by default only at the new position, attending over
// the cached keys and values of the prefix's ancestors (each tree node keeps
// its own rows; children point at their parent), so the cost of a step is
// one token per prefix rather than t -- splits each count over the 4 children
// with a multinomial
// draw (sequential binomials), drops zero counts and writes the next level
// in (parent, child) order.  Because children are emitted in token order and
// the first token holds the most significant qubits, the final level comes
// out sorted ascending by key.
//
// Randomness: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) keyed by the
// seed, with counter (prefix index, step, draw index); binomials by inversion
// for small means and by transformed rejection (Hormann 1993, "The
// generation of binomial random variates") otherwise.  Every loop has a fixed
// iteration cap.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "dev_common.cuh"
#include "internal.h"
#include "model.h"

namespace nnqs {
namespace {

// ---------------------------------------------------------------- Philox4x32-10
struct Philox {
    uint32_t k0, k1;
    uint32_t c0, c1, c2, c3;
    uint32_t out[4];
    int used = 4;

    __device__ void next_block() {
        uint32_t x0 = c0, x1 = c1, x2 = c2, x3 = c3, a = k0, b = k1;
#pragma unroll
        for (int r = 0; r < 10; ++r) {
            if (r > 0) {
                a += 0x9E3779B9u;
                b += 0xBB67AE85u;
            }
            const uint32_t hi0 = __umulhi(0xD2511F53u, x0), lo0 = 0xD2511F53u * x0;
            const uint32_t hi1 = __umulhi(0xCD9E8D57u, x2), lo1 = 0xCD9E8D57u * x2;
            const uint32_t n0 = hi1 ^ x1 ^ a, n1 = lo1, n2 = hi0 ^ x3 ^ b, n3 = lo0;
            x0 = n0;
            x1 = n1;
            x2 = n2;
            x3 = n3;
        }
        out[0] = x0;
        out[1] = x1;
        out[2] = x2;
        out[3] = x3;
        used = 0;
        ++c3;  // next block of this stream
    }
    __device__ uint32_t u32() {
        if (used >= 4) next_block();
        return out[used++];
    }
    // uniform in (0, 1), 53 bits
    __device__ double uniform() {
        const uint64_t a = u32() >> 5, b = u32() >> 6;
        return ((double)(a * 67108864ull + b) + 0.5) * (1.0 / 9007199254740992.0);
    }
};

// log(k!) - [(k + 1/2) log(k + 1) - (k + 1) + log(2 pi)/2]: Stirling remainder
__device__ __noinline__ double stirling_tail(double k) {
    if (k < 10.0) {
        return lgamma(k + 1.0) - ((k + 0.5) * log(k + 1.0) - (k + 1.0) + 0.91893853320467274178);
    }
    const double kp = k + 1.0, k2 = kp * kp;
    return (1.0 / 12.0 - (1.0 / 360.0 - (1.0 / 1260.0) / k2) / k2) / kp;
}

// inversion (sequential search from 0) for n p < 14, p <= 1/2
__device__ __noinline__ uint64_t binom_inversion(uint64_t n, double p, Philox &rng, DevStatus *st) {
    const double q = 1.0 - p, s = p / q, a = (double(n) + 1.0) * s;
    const double r0 = exp(double(n) * log1p(-p));
    for (int attempt = 0; attempt < 16; ++attempt) {
        double u = rng.uniform(), r = r0;
        uint64_t k = 0;
        bool done = false;
        for (int it = 0; it < 1000; ++it) {
            if (u <= r) {
                done = true;
                break;
            }
            u -= r;
            ++k;
            if (k > n) break;
            r *= (a / double(k) - s);
        }
        if (done && k <= n) return k;
    }
    record_status(st, NNQS_E_TIMEOUT, -2);
    return (uint64_t)floor(double(n) * p);
}

// Transformed rejection with squeeze (BTRS form) for n p >= 14, p <= 1/2:
// proposal k = floor((2a/us + b) u + c) with u ~ U(-1/2, 1/2); accept
// quickly inside the squeeze, otherwise compare log(v * hat) with the exact
// log f(k)/f(m) written through Stirling's series (f the binomial pmf,
// m its mode).
__device__ __noinline__ uint64_t binom_btrs(uint64_t n_, double p, Philox &rng, DevStatus *st) {
    const double n = (double)n_;
    const double q = 1.0 - p;
    const double m = floor((n + 1.0) * p);
    const double r = p / q;
    const double spq = sqrt(n * p * q);
    const double b = 1.15 + 2.53 * spq;
    const double a = -0.0873 + 0.0248 * b + 0.01 * p;
    const double c = n * p + 0.5;
    const double alpha = (2.83 + 5.1 / b) * spq;
    const double vr = 0.92 - 4.2 / b;
    for (int it = 0; it < 10000; ++it) {
        const double u = rng.uniform() - 0.5;
        double v = rng.uniform();
        const double us = 0.5 - fabs(u);
        const double kf = floor((2.0 * a / us + b) * u + c);
        if (kf < 0.0 || kf > n) continue;
        if (us >= 0.07 && v <= vr) return (uint64_t)kf;
        v = log(v * alpha / (a / (us * us) + b));
        const double bound = (m + 0.5) * log((m + 1.0) / (r * (n - m + 1.0))) +
                             (n + 1.0) * log((n - m + 1.0) / (n - kf + 1.0)) +
                             (kf + 0.5) * log(r * (n - kf + 1.0) / (kf + 1.0)) + stirling_tail(m) +
                             stirling_tail(n - m) - stirling_tail(kf) - stirling_tail(n - kf);
        if (v <= bound) return (uint64_t)kf;
    }
    record_status(st, NNQS_E_TIMEOUT, -3);
    return (uint64_t)m;
}

// The rejection and inversion loops and the Stirling tail are kept out of
// line (and k_split's category loop rolled) so that a thread's up to three
// draws run through one copy of their code: the early steps run a handful of
// threads, whose time is the latency of this FP64 code, instruction fetches
// included.
__device__ uint64_t binomial(uint64_t n, double p, Philox &rng, DevStatus *st) {
    if (n == 0 || !(p > 0.0)) return 0;
    if (p >= 1.0) return n;
    if (n == 1) return rng.uniform() < p ? 1 : 0;  // one draw: Bernoulli(p), no exp/log
    const bool flip = p > 0.5;
    const double pp = flip ? 1.0 - p : p;
    const uint64_t k = (double(n) * pp < 14.0) ? binom_inversion(n, pp, rng, st) : binom_btrs(n, pp, rng, st);
    const uint64_t kk = k > n ? n : k;
    return flip ? n - kk : kk;
}

// multinomial split of each prefix's count; nchild[i] = children with count > 0
// n_dev (optional): the count lives on the device; prefixes are then spread
// block-major (prefix i on block i % gridDim.x), so that the few prefixes of
// the early steps land on different SMs.  The draws depend on i only.
__global__ void k_split(const uint64_t *__restrict__ w, const double *__restrict__ cond, int64_t n, int step,
                        uint64_t seed, uint64_t *__restrict__ counts, int32_t *__restrict__ nchild, DevStatus *st,
                        const int64_t *__restrict__ n_dev, const uint64_t *__restrict__ seed_dev) {
    const int64_t i = n_dev ? blockIdx.x + (int64_t)gridDim.x * threadIdx.x
                            : blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (n_dev) n = *n_dev;
    if (seed_dev) seed = *seed_dev;
    if (i >= n) return;
    Philox rng;
    rng.k0 = (uint32_t)seed;
    rng.k1 = (uint32_t)(seed >> 32);
    rng.c0 = (uint32_t)i;
    rng.c1 = (uint32_t)((uint64_t)i >> 32);
    rng.c2 = (uint32_t)step;
    rng.c3 = 0;
    uint64_t rem = w[i];
    double prem = 1.0;
    int last = -1;  // the last child the mask allows takes what is left
#pragma unroll
    for (int v = 0; v < 4; ++v)
        if (cond[i * 4 + v] > 0.0) last = v;
    if (last < 0 && rem > 0) record_status(st, NNQS_E_SECTOR, i);
    int nc = 0;
#pragma unroll 1
    for (int v = 0; v < 4; ++v) {
        const double pv = cond[i * 4 + v];
        uint64_t k = 0;
        if (v == last) {
            k = rem;
        } else if (v < last && pv > 0.0 && rem > 0) {
            const double q = prem > 0.0 ? fmin(1.0, fmax(0.0, pv / prem)) : 0.0;
            k = binomial(rem, q, rng, st);
        }
        counts[i * 4 + v] = k;
        rem -= k;
        prem -= pv;
        nc += k > 0;
    }
    nchild[i] = nc;
}

// exclusive scan, 1024 per block; block totals to bsum
constexpr int kScan = 1024;
__global__ void k_scan_blocks(const int32_t *__restrict__ in, int64_t n, int64_t *__restrict__ out,
                              int64_t *__restrict__ bsum) {
    __shared__ int64_t sh[kScan];
    const int64_t i = blockIdx.x * (int64_t)kScan + threadIdx.x;
    const int64_t v = i < n ? in[i] : 0;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < kScan; off <<= 1) {
        const int64_t t = threadIdx.x >= off ? sh[threadIdx.x - off] : 0;
        __syncthreads();
        sh[threadIdx.x] += t;
        __syncthreads();
    }
    if (i < n) out[i] = sh[threadIdx.x] - v;
    if (threadIdx.x == kScan - 1) bsum[blockIdx.x] = sh[kScan - 1];
}

// sequential scan of the block totals in one block, chunk by chunk
__global__ void k_scan_sums(int64_t *__restrict__ bsum, int64_t nb, int64_t *__restrict__ total) {
    __shared__ int64_t sh[kScan];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t c0 = 0; c0 < nb; c0 += kScan) {
        const int64_t i = c0 + threadIdx.x;
        const int64_t v = i < nb ? bsum[i] : 0;
        sh[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < kScan; off <<= 1) {
            const int64_t t = threadIdx.x >= off ? sh[threadIdx.x - off] : 0;
            __syncthreads();
            sh[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < nb) bsum[i] = carry + sh[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == kScan - 1) carry += sh[kScan - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan_add(int64_t *__restrict__ out, int64_t n, const int64_t *__restrict__ bsum) {
    const int64_t i = blockIdx.x * (int64_t)kScan + threadIdx.x;
    if (i < n) out[i] += bsum[blockIdx.x];
}

// the same exclusive scan in one CTA for short lists (n <= kScanOne): warp w
// takes a contiguous segment (a multiple of 512); pass 1 sums it 512 elements
// at a time (16 loads in flight per lane), the 32 segment totals are scanned,
// pass 2 walks the segment again the same way with a 32-bit shuffle scan per
// 32 elements (a piece of at most 4 x 32 children) and a running 64-bit carry
// starting at the segment's offset; *total = the sum
constexpr int kScanOne = 65536;
__global__ void __launch_bounds__(1024) k_scan_one(const int32_t *__restrict__ in, int64_t n,
                                                  int64_t *__restrict__ out, int64_t *__restrict__ total,
                                                  const int64_t *__restrict__ n_dev) {
    constexpr int kB = 16;  // 32-element pieces per batch
    __shared__ int64_t wsum[32];
    if (n_dev) n = *n_dev;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t seg = ((n + 31) / 32 + 32 * kB - 1) / (32 * kB) * (32 * kB);  // elements per warp
    const int64_t b = min(n, warp * seg), e = min(n, b + seg);
    int64_t part = 0;
    for (int64_t i0 = b; i0 < e; i0 += 32 * kB) {
        int32_t x[kB];
#pragma unroll
        for (int k = 0; k < kB; ++k) {
            const int64_t i = i0 + 32 * k + lane;
            x[k] = i < e ? in[i] : 0;
        }
        int32_t sx = 0;
#pragma unroll
        for (int k = 0; k < kB; ++k) sx += x[k];
        part += sx;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (lane == 0) wsum[warp] = part;
    __syncthreads();
    if (warp == 0) {
        int64_t w = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t u = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += u;
        }
        wsum[lane] = w;  // inclusive over the segments
    }
    __syncthreads();
    int64_t carry = warp > 0 ? wsum[warp - 1] : 0;
    for (int64_t i0 = b; i0 < e; i0 += 32 * kB) {
        int32_t x[kB];
#pragma unroll
        for (int k = 0; k < kB; ++k) {
            const int64_t i = i0 + 32 * k + lane;
            x[k] = i < e ? in[i] : 0;
        }
#pragma unroll
        for (int k = 0; k < kB; ++k) {
            int32_t v = x[k];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t u = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += u;
            }
            const int64_t i = i0 + 32 * k + lane;
            if (i < e) out[i] = carry + (int64_t)(v - x[k]);
            carry += __shfl_sync(0xffffffffu, v, 31);
        }
    }
    if (threadIdx.x == 0) *total = wsum[31];
}

// children of prefix i in token order at slots off[i] ...
// children of prefix i go to rows off[i].. of the next level; with the
// key/value cache each child's ancestors are its parent's plus the parent's
// own node g_cur + i at depth `step` (the tables are depth-major, [T][cap]:
// a warp's lanes write consecutive entries of one depth)
// end of a step with the counts on the device: cnt[cur ^ 1] = the next
// level's size (the scan's total, clamped to the capacity after recording
// NNQS_E_TABLE_FULL), cnt[2] += this level's size (the first tree node of the
// next level)
__device__ __forceinline__ void advance_counts(int64_t *cnt, int cur, const int64_t *total, int64_t cap,
                                               DevStatus *st) {
    int64_t nn = *total;
    if (nn > cap) {
        record_status(st, NNQS_E_TABLE_FULL, nn);
        nn = cap;
    }
    cnt[2] += cnt[cur];
    cnt[cur ^ 1] = nn;
}

__global__ void k_emit(const uint64_t *__restrict__ pref, const uint64_t *__restrict__ counts,
                       const int64_t *__restrict__ off, int64_t n, int W, int T, int step, int64_t cap,
                       uint64_t *__restrict__ npref, uint64_t *__restrict__ nw, const int32_t *__restrict__ anc,
                       int32_t *__restrict__ nanc, int64_t g_cur, DevStatus *st, const int64_t *__restrict__ n_dev,
                       const int64_t *__restrict__ g_dev, int64_t *adv, int cur, const int64_t *__restrict__ total) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (n_dev) {
        n = *n_dev;
        g_cur = *g_dev;
    }
    if (i < n) {
        int64_t j = off[i];
        const int p = T - 1 - step;  // orbital of this token
        for (int v = 0; v < 4; ++v) {
            const uint64_t c = counts[i * 4 + v];
            if (c == 0) continue;
            if (j >= cap) {
                record_status(st, NNQS_E_TABLE_FULL, i);
                break;
            }
            for (int w = 0; w < W; ++w) npref[j * W + w] = pref[i * W + w];
            if (v & 1) npref[j * W + ((2 * p) >> 6)] |= 1ull << ((2 * p) & 63);
            if (v & 2) npref[j * W + ((2 * p + 1) >> 6)] |= 1ull << ((2 * p + 1) & 63);
            nw[j] = c;
            if (nanc) {
                for (int lev = 0; lev < step; ++lev) nanc[lev * cap + j] = anc[lev * cap + i];
                nanc[step * cap + j] = (int32_t)(g_cur + i);
            }
            ++j;
        }
    }
    if (adv) {
        // device-side counts: the last block to finish advances them (every
        // other block read them before its arrival); adv[3] counts arrivals
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            const unsigned long long done = atomicAdd(reinterpret_cast<unsigned long long *>(adv + 3), 1ull);
            if (done == gridDim.x - 1) {
                __threadfence();
                advance_counts(adv, cur, total, cap, st);
                adv[3] = 0;
            }
        }
    }
}

// level 0 of the device-count walk: the empty prefix holds all n_samples =
// args[0] samples; level sizes {1, 0}, first node 0, no emit arrivals yet
__global__ void k_level0(uint64_t *pref, int W, uint64_t *w, int64_t *cnt, const uint64_t *args) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int k = 0; k < W; ++k) pref[k] = 0;
    w[0] = args[0];
    cnt[0] = 1;
    cnt[1] = 0;
    cnt[2] = 0;
    cnt[3] = 0;
}

struct SLayout {
    uint64_t *pref[2], *w[2], *counts;
    double *cond;
    int32_t *nchild;
    int64_t *off, *bsum, *total;
    int32_t *anc[2];  // key/value cache: ancestor tables [T][cap] of the current and next level
    int64_t *cnt;     // device-side counts: level sizes [2], first node of the current level, k_emit arrivals
    uint64_t *args;   // device copies of n_samples and seed (read by the device-count walk)
    char *region;
    int64_t kv_nodes;
    float *act, *fin;  // NNQS_SAMPLE_KEEP: per tree node the layers' input and mid residual rows, the final residual
};

SLayout slayout(const nnqs_model *M, int64_t cap, int prec, bool cached, Arena &a, bool keep = false) {
    SLayout L{};
    const int W = M->W;
    for (int k = 0; k < 2; ++k) {
        L.pref[k] = a.take<uint64_t>(size_t(cap) * W);
        L.w[k] = a.take<uint64_t>(size_t(cap));
    }
    L.counts = a.take<uint64_t>(size_t(cap) * 4);
    L.cond = a.take<double>(size_t(cap) * 4);
    L.nchild = a.take<int32_t>(size_t(cap));
    L.off = a.take<int64_t>(size_t(cap));
    L.bsum = a.take<int64_t>(size_t((cap + kScan - 1) / kScan + 1));
    L.total = a.take<int64_t>(1);
    L.cnt = a.take<int64_t>(4);
    L.args = a.take<uint64_t>(2);
    L.kv_nodes = cached ? int64_t(M->T) * cap + 1 : 0;
    for (int k = 0; k < 2; ++k) L.anc[k] = cached ? a.take<int32_t>(size_t(cap) * M->T) : nullptr;
    L.region = a.take<char>(cond_workspace(M, cap, prec, L.kv_nodes));
    L.act = keep ? a.take<float>(size_t(L.kv_nodes) * 2 * M->L * M->d) : nullptr;
    L.fin = keep ? a.take<float>(size_t(L.kv_nodes) * M->d) : nullptr;
    return L;
}

}  // namespace
}  // namespace nnqs

namespace nnqs {
namespace {

// The whole walk with the level sizes on the device: every kernel reads the
// level's size (and the seed) from device memory and is sized for the
// capacity, so no step waits for the host, and the sequence -- parameter
// conversion, weight images, level 0, then per step the fused decode layers,
// split, scan, emit and advance -- is the same on every call with the same
// model, parameters, workspace and capacity.  Such repeated calls replay it
// as a CUDA graph (captured on the second call; the first runs the kernels
// directly), which removes most of the per-launch gaps of its ~165 launches.
// With profiling on, the kernels always run directly.
struct GraphKey {
    int dev;
    const nnqs_model *M;
    nnqs_model_cfg cfg;
    const float *params;
    int prec;
    int64_t cap;
    const void *ws;
    size_t ws_bytes;
    bool keep;
    bool operator==(const GraphKey &o) const {
        return dev == o.dev && M == o.M && std::memcmp(&cfg, &o.cfg, sizeof cfg) == 0 && params == o.params &&
               prec == o.prec && cap == o.cap && ws == o.ws && ws_bytes == o.ws_bytes && keep == o.keep;
    }
};
struct GraphEntry {
    GraphKey key;
    int calls = 0;
    cudaGraphExec_t exec = nullptr;
    uint64_t launches = 0;
    uint64_t last_use = 0;
};
constexpr size_t kMaxGraphs = 8;
std::mutex g_graph_mu;
std::vector<GraphEntry> g_graphs;
uint64_t g_graph_clock = 0;

// CUDA-graph replay of the walk, from NNQS_SAMPLE_GRAPH in the environment
// (read once): 0 = always launch the kernels directly (comparisons)
bool sample_graphs_enabled() {
    static const bool on = [] {
        const char *e = std::getenv("NNQS_SAMPLE_GRAPH");
        return !(e && e[0] == '0');
    }();
    return on;
}

nnqs_status walk_kernels(const nnqs_model *M, const float *params, int prec, int64_t cap, const SLayout &L,
                         DevStatus *st, cudaStream_t s) {
    Arena sub(L.region);
    CondCtx *ctx = nullptr;
    nnqs_status rc = cond_create(M, params, prec, cap, L.kv_nodes, sub, &ctx, s);
    const int W = M->W, T = M->T;
    const unsigned sgrid = (unsigned)std::max<int64_t>(num_sms(), (cap + 127) / 128);
    if (rc == NNQS_OK) {
        NNQS_LAUNCH("k_emit", s, k_level0<<<1, 32, 0, s>>>(L.pref[0], W, L.w[0], L.cnt, L.args));
        int cur = 0;
        for (int t = 0; t < T && rc == NNQS_OK; ++t) {
            rc = cond_step_cached_dev(M, ctx, L.pref[cur], L.cnt + cur, L.cnt + 2, cap, t, L.anc[cur], L.cond, st, s,
                                      L.act, L.fin);
            if (rc != NNQS_OK) break;
            NNQS_LAUNCH("k_split", s, k_split<<<sgrid, 128, 0, s>>>(L.w[cur], L.cond, cap, t, 0, L.counts, L.nchild, st,
                                                                    L.cnt + cur, L.args + 1));
            NNQS_LAUNCH("k_scan", s, k_scan_one<<<1, 1024, 0, s>>>(L.nchild, cap, L.off, L.total, L.cnt + cur));
            NNQS_LAUNCH("k_emit", s, k_emit<<<grid_for(cap, 128), 128, 0, s>>>(L.pref[cur], L.counts, L.off, cap, W, T, t,
                                                                              cap, L.pref[cur ^ 1], L.w[cur ^ 1],
                                                                              L.anc[cur], L.anc[cur ^ 1], 0, st,
                                                                              L.cnt + cur, L.cnt + 2, L.cnt, cur,
                                                                              L.total));
            cur ^= 1;
        }
    }
    cond_destroy(ctx);
    return rc;
}

nnqs_status dev_walk(const nnqs_model *M, const float *params, uint64_t n_samples, uint64_t seed, int prec,
                     int64_t cap, const SLayout &L, DevStatus *st, uint64_t *samples_out, uint64_t *weights_out,
                     int64_t *n_unique_out, const void *workspace, size_t workspace_bytes, cudaStream_t s) {
    const uint64_t args[2] = {n_samples, seed};
    NNQS_CUDA_TRY(cudaMemcpyAsync(L.args, args, sizeof args, cudaMemcpyHostToDevice, s));
    nnqs_status rc = NNQS_OK;
    if (profiling_on() || !sample_graphs_enabled()) {
        rc = walk_kernels(M, params, prec, cap, L, st, s);
    } else {
        GraphKey key{};
        NNQS_CUDA_TRY(cudaGetDevice(&key.dev));
        key.M = M;
        key.cfg = M->cfg;
        key.params = params;
        key.prec = prec;
        key.cap = cap;
        key.ws = workspace;
        key.ws_bytes = workspace_bytes;
        key.keep = L.act != nullptr;
        std::unique_lock<std::mutex> lk(g_graph_mu);
        GraphEntry *e = nullptr;
        for (auto &g : g_graphs)
            if (g.key == key) e = &g;
        if (!e) {
            if (g_graphs.size() >= kMaxGraphs) {  // drop the least recently used
                auto old = std::min_element(g_graphs.begin(), g_graphs.end(), [](const GraphEntry &a, const GraphEntry &b) {
                    return a.last_use < b.last_use;
                });
                if (old->exec) cudaGraphExecDestroy(old->exec);
                g_graphs.erase(old);
            }
            g_graphs.push_back(GraphEntry{key});
            e = &g_graphs.back();
        }
        e->last_use = ++g_graph_clock;
        ++e->calls;
        if (e->exec) {
            NNQS_CUDA_TRY(cudaGraphLaunch(e->exec, s));
            note_replay(e->launches);
        } else if (e->calls >= 2) {
            // capture the walk once; any failure falls back to direct launches
            const uint64_t l0 = nnqs_launch_count();
            cudaGraph_t graph = nullptr;
            bool captured = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            if (captured) {
                rc = walk_kernels(M, params, prec, cap, L, st, s);
                captured = cudaStreamEndCapture(s, &graph) == cudaSuccess && rc == NNQS_OK;
            }
            cudaGraphExec_t exec = nullptr;
            if (captured && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess) {
                e->exec = exec;
                e->launches = nnqs_launch_count() - l0;
                NNQS_CUDA_TRY(cudaGraphLaunch(exec, s));
            } else {
                cudaGetLastError();
                rc = walk_kernels(M, params, prec, cap, L, st, s);
            }
            if (graph) cudaGraphDestroy(graph);
        } else {
            rc = walk_kernels(M, params, prec, cap, L, st, s);
        }
    }
    if (rc != NNQS_OK) return rc;
    // after T steps the last level sits at index T % 2
    const int cur = M->T & 1;
    int64_t n_final = 0;
    NNQS_CUDA_TRY(cudaMemcpyAsync(&n_final, L.cnt + cur, 8, cudaMemcpyDeviceToHost, s));
    NNQS_CUDA_TRY(cudaStreamSynchronize(s));
    DevStatus hst{};
    NNQS_CUDA_TRY(cudaMemcpy(&hst, st, sizeof hst, cudaMemcpyDeviceToHost));
    if (hst.code == NNQS_E_TABLE_FULL)
        return set_error(NNQS_E_TABLE_FULL, "a step held " + std::to_string(hst.index) + " prefixes, above max_unique " +
                                                std::to_string(cap));
    NNQS_CUDA_TRY(cudaMemcpyAsync(samples_out, L.pref[cur], size_t(n_final) * M->W * 8, cudaMemcpyDeviceToDevice, s));
    NNQS_CUDA_TRY(cudaMemcpyAsync(weights_out, L.w[cur], size_t(n_final) * 8, cudaMemcpyDeviceToDevice, s));
    *n_unique_out = n_final;
    return NNQS_OK;
}

}  // namespace
}  // namespace nnqs

using namespace nnqs;

namespace nnqs {

bool sample_keep_ok(const nnqs_model *M, int prec, int64_t max_unique) {
    return max_unique >= 1 && max_unique <= kScanOne && cond_dev_walk_ok(M, prec, max_unique);
}

nnqs_status sample_kept(const nnqs_model *M, int prec, int64_t max_unique, const void *ws, size_t ws_bytes,
                        SampleKept *out) {
    if (!ws || reinterpret_cast<uintptr_t>(ws) % 256)
        return set_error(NNQS_E_INVAL, "sampler workspace null or misaligned");
    if (!sample_keep_ok(M, prec, max_unique))
        return set_error(NNQS_E_UNSUPPORTED, "no NNQS_SAMPLE_KEEP walk for this model, precision or max_unique");
    if (ws_bytes < nnqs_sample_workspace_size(M, max_unique, prec, NNQS_SAMPLE_KEEP))
        return set_error(NNQS_E_WORKSPACE, "sampler workspace smaller than an NNQS_SAMPLE_KEEP call's");
    Arena a(const_cast<void *>(ws));
    a.take<char>(kStatusBytes);
    const SLayout L = slayout(M, max_unique, prec, true, a, true);
    const int cur = M->T & 1;  // the last level after T steps
    out->act = L.act;
    out->fin = L.fin;
    out->anc = L.anc[cur];
    out->pref = L.pref[cur];
    out->stride = max_unique;
    return NNQS_OK;
}

}  // namespace nnqs

extern "C" size_t nnqs_sample_workspace_size(const nnqs_model *M, int64_t max_unique, int prec, int flags) {
    if (!M || max_unique < 1) return 0;
    Arena a(nullptr);
    a.take<char>(kStatusBytes);
    slayout(M, max_unique, prec, !(flags & NNQS_SAMPLE_RECOMPUTE), a, (flags & NNQS_SAMPLE_KEEP) != 0);
    return a.used + 1024;
}

extern "C" nnqs_status nnqs_sample(const nnqs_model *M, const float *params, uint64_t n_samples, uint64_t seed,
                                   int prec, int flags, int64_t max_unique, uint64_t *samples_out,
                                   uint64_t *weights_out, int64_t *n_unique_out, void *workspace,
                                   size_t workspace_bytes, nnqs_stream stream) {
    if (!M || !params || !samples_out || !weights_out || !n_unique_out || max_unique < 1)
        return set_error(NNQS_E_INVAL, "null argument or max_unique < 1");
    if (!prec_valid(prec)) return set_error(NNQS_E_INVAL, "bad precision");
    if (flags & ~(NNQS_SAMPLE_RECOMPUTE | NNQS_SAMPLE_KEEP)) return set_error(NNQS_E_INVAL, "unknown sampler flags");
    const bool keep = (flags & NNQS_SAMPLE_KEEP) != 0;
    if (keep && ((flags & NNQS_SAMPLE_RECOMPUTE) || !sample_keep_ok(M, prec, max_unique)))
        return set_error(NNQS_E_UNSUPPORTED, "NNQS_SAMPLE_KEEP needs the cached device walk (BF16 or split BF16, "
                                             "d_model 64, max_unique <= 65536)");
    if (n_samples > (uint64_t(1) << 53)) return set_error(NNQS_E_INVAL, "n_samples above 2^53");
    *n_unique_out = 0;
    const bool cached = !(flags & NNQS_SAMPLE_RECOMPUTE);
    const size_t need = nnqs_sample_workspace_size(M, max_unique, prec, flags);
    if (!workspace || reinterpret_cast<uintptr_t>(workspace) % 256 || workspace_bytes < need)
        return set_error(NNQS_E_WORKSPACE, "workspace null, misaligned or smaller than " + std::to_string(need));
    cudaStream_t s = (cudaStream_t)stream;
    NNQS_CUDA_TRY(cudaMemsetAsync(workspace, 0, sizeof(DevStatus), s));
    Arena a(workspace);
    DevStatus *st = a.take<DevStatus>(kStatusBytes / sizeof(DevStatus));
    const SLayout L = slayout(M, max_unique, prec, cached, a, keep);
    if (L.kv_nodes >= (int64_t(1) << 31))
        return set_error(NNQS_E_UNSUPPORTED, "key/value cache above 2^31 nodes (T * max_unique)");
    if (n_samples == 0) return NNQS_OK;
    if (cached && max_unique <= kScanOne && cond_dev_walk_ok(M, prec, max_unique))
        return dev_walk(M, params, n_samples, seed, prec, max_unique, L, st, samples_out, weights_out, n_unique_out,
                        workspace, workspace_bytes, s);
    Arena sub(L.region);
    CondCtx *ctx = nullptr;
    nnqs_status rc = cond_create(M, params, prec, max_unique, L.kv_nodes, sub, &ctx, s);
    if (rc != NNQS_OK) {
        cond_destroy(ctx);
        return rc;
    }
    const int W = M->W, T = M->T;
    // level 0: the empty prefix holds every sample
    NNQS_CUDA_TRY(cudaMemsetAsync(L.pref[0], 0, size_t(W) * 8, s));
    NNQS_CUDA_TRY(cudaMemcpyAsync(L.w[0], &n_samples, 8, cudaMemcpyHostToDevice, s));
    int64_t n = 1;
    int cur = 0;
    int64_t g_cur = 0;  // tree-node id of the first prefix of the current level
    auto step = [&](int t) -> nnqs_status {
        if (cached)
            NNQS_TRY(cond_step_cached(M, ctx, L.pref[cur], n, t, g_cur, L.anc[cur], L.cond, st, s));
        else
            NNQS_TRY(cond_step(M, ctx, L.pref[cur], n, t + 1, L.cond, st, s));
        // the binomial draws are FP64-bound: few prefixes (the early steps,
        // counts in the thousands) are spread one or a few per block over
        // the SMs instead of sharing one SM's FP64 pipe
        const int split_block = (int)std::min<int64_t>(128, std::max<int64_t>(1, (n + num_sms() - 1) / num_sms()));
        NNQS_LAUNCH("k_split", s, k_split<<<(unsigned)((n + split_block - 1) / split_block), split_block, 0, s>>>(
                                      L.w[cur], L.cond, n, t, seed, L.counts, L.nchild, st, nullptr, nullptr));
        const int64_t nb = (n + kScan - 1) / kScan;
        if (n <= kScanOne) {
            NNQS_LAUNCH("k_scan", s, k_scan_one<<<1, 1024, 0, s>>>(L.nchild, n, L.off, L.total, nullptr));
        } else {
            NNQS_LAUNCH("k_scan_blocks", s, k_scan_blocks<<<(unsigned)nb, kScan, 0, s>>>(L.nchild, n, L.off, L.bsum));
            NNQS_LAUNCH("k_scan_sums", s, k_scan_sums<<<1, kScan, 0, s>>>(L.bsum, nb, L.total));
            NNQS_LAUNCH("k_scan_add", s, k_scan_add<<<(unsigned)nb, kScan, 0, s>>>(L.off, n, L.bsum));
        }
        int64_t next = 0;
        NNQS_CUDA_TRY(cudaMemcpyAsync(&next, L.total, 8, cudaMemcpyDeviceToHost, s));
        NNQS_CUDA_TRY(cudaStreamSynchronize(s));
        if (next > max_unique)
            return set_error(NNQS_E_TABLE_FULL, "step " + std::to_string(t) + " holds " + std::to_string(next) +
                                                    " prefixes, above max_unique " + std::to_string(max_unique));
        NNQS_LAUNCH("k_emit", s, k_emit<<<grid_for(n, 128), 128, 0, s>>>(L.pref[cur], L.counts, L.off, n, W, T, t,
                                                                         max_unique, L.pref[cur ^ 1], L.w[cur ^ 1],
                                                                         L.anc[cur], L.anc[cur ^ 1], g_cur, st,
                                                                         nullptr, nullptr, nullptr, 0, nullptr));
        cur ^= 1;
        g_cur += n;
        n = next;
        return NNQS_OK;
    };
    for (int t = 0; t < T && rc == NNQS_OK; ++t) rc = step(t);
    cond_destroy(ctx);
    if (rc != NNQS_OK) return rc;
    NNQS_CUDA_TRY(cudaMemcpyAsync(samples_out, L.pref[cur], size_t(n) * W * 8, cudaMemcpyDeviceToDevice, s));
    NNQS_CUDA_TRY(cudaMemcpyAsync(weights_out, L.w[cur], size_t(n) * 8, cudaMemcpyDeviceToDevice, s));
    *n_unique_out = n;
    return NNQS_OK;
}
