// Fused forward of the transformer amplitude (Sec. 3.1, Eq. auto; mask of
// Sec. 3.3) for log|psi| of whole samples, on tcgen05 tensor cores.
//
// A persistent CTA of 512 threads per SM walks 128-row tiles of token rows
// (floor(128 / T) samples of T tokens each) and keeps every activation of a
// tile on chip through all decoder layers: the residual rows in shared
// memory (FP32), the A operands as BF16 (split hi/lo) swizzled tiles, the
// accumulators in TMEM, the keys and values of the tile in shared memory for
// the causal attention (a sample's tokens never leave its tile), and the
// weights brought in by bulk asynchronous copies of their pre-swizzled
// images while the previous phase computes:
//   embedding -> [LN1 -> qkv MMA -> attention -> out-projection MMA +
//   residual -> LN2 -> four FFN-in MMAs -> GELU chunks -> FFN-out MMAs +
//   residual] x L -> final LN -> head -> masked log-softmax of each row's
//   token -> log|psi| = 1/2 sum over the sample's rows.
// Per sample only its bitstring is read and one double written; the phase
// MLP runs separately.  The arithmetic is the unfused FP32/BF16 path's up to
// the order of floating-point sums and the GELU's erf (ff_gelu; not
// bit-identical to it).
//
// Shared memory (1024-aligned base):
//   [0, 32K)      A tile hi / lo  (LN output, attention output)
//   [32K, 64K)    G tile hi / lo  (GELU chunk); before the FFN: Wo hi / lo
//   [64K, 128K)   k | v of the tile [128][128] FP32 (attention); then W2
//   [128K, 192K)  Wqkv hi / lo; after the qkv MMA: W1 hi / lo
//   [192K, ...)   residual rows [128][65] FP32, per-row log pi~, barriers
// TMEM (512 columns): q | k | v [0, 192), out-projection [192, 256), the four
// FFN-in chunks [256, 512), FFN-out [0, 64) (over q, consumed by then).
//
// Every wait is bounded (tc::mbar_wait): on a timeout the CTA records
// NNQS_E_TIMEOUT, lets its weight copies land (bounded) and frees its TMEM.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "dev_common.cuh"
#include "fwd_fused.cuh"
#include "tc_gemm.cuh"

namespace nnqs {
namespace {
namespace ff {
constexpr int kThreads = 512, kRows = 128, kD = 64, kQKV = 192, kF = 256;
constexpr int kOffA = 0, kOffA2 = 16384, kOffG = 32768, kOffG2 = 49152;
constexpr int kOffKV = 65536, kOffWB = 131072, kOffH = 196608;
constexpr int kHS = 65;
constexpr int kOffLP = kOffH + kRows * kHS * 4;
constexpr int kOffBar = kOffLP + kRows * 4;
constexpr int kSmem = kOffBar + 64 + 1024;  // 231,488 bytes
constexpr uint32_t kColQ = 0, kColO = 192, kColU = 256, kColY = 0, kTmemCols = 512;
constexpr float kLog2e = 1.44269504088896340736f;
}  // namespace ff

__device__ __forceinline__ void ff_bulk(uint8_t *dst, const void *src, uint32_t bytes, uint32_t mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     tc::smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(mbar)
                 : "memory");
}

__device__ __forceinline__ float ff_ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 16 consecutive floats of a 16-byte aligned parameter vector
__device__ __forceinline__ void ff_ld16(const float *__restrict__ p, float (&v)[16]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float4 a = __ldg(reinterpret_cast<const float4 *>(p) + k);
        v[4 * k] = a.x;
        v[4 * k + 1] = a.y;
        v[4 * k + 2] = a.z;
        v[4 * k + 3] = a.w;
    }
}

// GELU x Phi(x) = x (1 + erf(x / sqrt 2)) / 2 with erf from the rational
// approximation of Abramowitz and Stegun, Handbook of Mathematical Functions
// (1964), eq. 7.1.26: erf(z) = 1 - t (a1 + t (a2 + t (a3 + t (a4 + t a5))))
// e^{-z^2}, t = 1 / (1 + p z) for z >= 0, odd in z, absolute error at most
// 1.5e-7 -- far below the 2^-16 relative resolution of the split-BF16 operand
// the value feeds; branch-free, two special-function instructions.
__device__ __forceinline__ float ff_gelu(float x) {
    const float z = fabsf(x) * 0.70710678118654752f;
    const float t = __fdividef(1.0f, fmaf(0.3275911f, z, 1.0f));
    const float poly =
        t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.061405429f, -1.453152027f), 1.421413741f), -0.284496736f), 0.254829592f);
    const float e = ff_ex2(-(z * z) * 1.44269504088896340736f);
    const float erf_abs = 1.0f - poly * e;
    return 0.5f * x * (1.0f + copysignf(erf_abs, x));
}

// element (r, c) of the tile's k | v rows, r of sample sl of the tile: the
// 16-byte pieces XOR-rotated by (r ^ sl) & 7, so that the lanes of a warp
// reading the same piece of their samples' rows s T + j (one row per sample)
// and the lanes writing consecutive rows of one sample use different banks
__device__ __forceinline__ int kv_at(int r, int c, int sl) {
    return r * 128 + ((((c >> 2) ^ ((r ^ sl) & 7))) << 2) + (c & 3);
}

// 8 values as one granule of a swizzled A-operand tile row (hi, and lo when split)
__device__ __forceinline__ void ff_granule(uint8_t *hi, uint8_t *lo, int r, int c, const float *v, bool split) {
    float x[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) x[e] = v[e];
    const int off = r * 128 + ((c ^ (r & 7)) << 4);
    *reinterpret_cast<uint4 *>(hi + off) = tc::pack8(x);
    if (split) {
        float y[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) y[e] = x[e] - __bfloat162float(__float2bfloat16_rn(x[e]));
        *reinterpret_cast<uint4 *>(lo + off) = tc::pack8(y);
    }
}

// LayerNorm (eps 1e-5) of residual rows by 4 lanes per row: warp w takes rows
// 8 w .. 8 w + 7, lane 4 k + p of row 8 w + k the columns 8 p .. 8 p + 7 and
// 32 + 8 p .. 32 + 8 p + 7 (so that the 32 lanes' reads of the residual rows,
// stride 65, fall in 32 different banks).  y[0..7] and y[8..15] are those
// columns' normalised values; the A tile gets them as BF16 (hi / lo, granules
// p and p + 4) when `hi` is not null.
struct LnOut {
    float y[16];
    float mu, rs;
};

// the 16 columns of LayerNorm part p of a 64-wide vector: 8 p .. and 32 + 8 p ..
__device__ __forceinline__ int ln_col(int p, int c) { return (c < 8 ? 8 * p : 32 + 8 * p - 8) + c; }

// 16 floats of LayerNorm part p from a 16-byte aligned vector
__device__ __forceinline__ void ff_ld_part(const float *__restrict__ vec, int p, float (&v)[16]) {
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const float4 a = __ldg(reinterpret_cast<const float4 *>(vec + 32 * h + 8 * p) + k);
            v[8 * h + 4 * k] = a.x;
            v[8 * h + 4 * k + 1] = a.y;
            v[8 * h + 4 * k + 2] = a.z;
            v[8 * h + 4 * k + 3] = a.w;
        }
}

// 16 floats of LayerNorm part p to a 16-byte aligned row
__device__ __forceinline__ void ff_st_part(float *row, int p, const float *v) {
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int k = 0; k < 2; ++k)
            reinterpret_cast<float4 *>(row + 32 * h + 8 * p)[k] =
                make_float4(v[8 * h + 4 * k], v[8 * h + 4 * k + 1], v[8 * h + 4 * k + 2], v[8 * h + 4 * k + 3]);
}

__device__ __forceinline__ LnOut ff_layernorm(const float *sH, int r, int p, const float *__restrict__ gam,
                                              const float *__restrict__ bet, uint8_t *hi, uint8_t *lo, bool split) {
    LnOut o;
    float v[16];
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < 16; ++c) {
        v[c] = sH[r * ff::kHS + ln_col(p, c)];
        s += v[c];
    }
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    o.mu = s / float(ff::kD);
    float q = 0.f;
#pragma unroll
    for (int c = 0; c < 16; ++c) q += (v[c] - o.mu) * (v[c] - o.mu);
    q += __shfl_xor_sync(0xffffffffu, q, 1);
    q += __shfl_xor_sync(0xffffffffu, q, 2);
    o.rs = 1.0f / sqrtf(q / float(ff::kD) + 1e-5f);
    float gv[16], bv[16];
    ff_ld_part(gam, p, gv);
    ff_ld_part(bet, p, bv);
#pragma unroll
    for (int c = 0; c < 16; ++c) o.y[c] = (v[c] - o.mu) * o.rs * gv[c] + bv[c];
    if (hi) {
        ff_granule(hi, lo, r, p, o.y, split);
        ff_granule(hi, lo, r, p + 4, o.y + 8, split);
    }
    return o;
}

// 16 floats to global memory (16-byte aligned)
__device__ __forceinline__ void ff_st16(float *dst, const float *v) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
        reinterpret_cast<float4 *>(dst)[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
}

// 4 K steps (K = 64) of one 128 x N product into TMEM: with split operands
// lo.hi + hi.lo + hi.hi per step
__device__ __forceinline__ void ff_mma(uint32_t tmem, uint32_t aHi, uint32_t aLo, uint32_t bHi, uint32_t bLo, int N,
                                       bool split, bool acc0) {
    const uint32_t idesc = tc::idesc_bf16(ff::kRows, N);
    const uint64_t da = tc::desc_sw128(aHi), db = tc::desc_sw128(bHi);
    const uint64_t da2 = tc::desc_sw128(aLo), db2 = tc::desc_sw128(bLo);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint32_t acc = (acc0 || k > 0) ? 1u : 0u;
        if (split) {
            tc::mma_bf16(tmem, da2 + uint64_t(2 * k), db + uint64_t(2 * k), idesc, acc);
            tc::mma_bf16(tmem, da + uint64_t(2 * k), db2 + uint64_t(2 * k), idesc, 1u);
            tc::mma_bf16(tmem, da + uint64_t(2 * k), db + uint64_t(2 * k), idesc, 1u);
        } else {
            tc::mma_bf16(tmem, da + uint64_t(2 * k), db + uint64_t(2 * k), idesc, acc);
        }
    }
}

__device__ __forceinline__ int ff_bit(const uint64_t *x, int j) { return (int)((x[j >> 6] >> (j & 63)) & 1ull); }
// token at position t: spatial orbital T-1-t, value y_alpha + 2 y_beta
__device__ __forceinline__ int ff_token(const uint64_t *x, int T, int t) {
    const int p = T - 1 - t;
    return ff_bit(x, 2 * p) + 2 * ff_bit(x, 2 * p + 1);
}

template <bool SPLIT, int DH, int KEEP>
__global__ void __launch_bounds__(ff::kThreads, 1) k_fwd_fused(const __grid_constant__ FusedFwdArgs g) {
    using namespace ff;
    constexpr int H = kD / DH;
    constexpr int HPT = H / 4;  // heads of one thread: its row's 16-column quarter
    static_assert(HPT * DH == 16, "a thread covers 16 columns of q");
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = tc::smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *sb = smem_raw + (base - raw);
    uint8_t *aHi = sb + kOffA, *aLo = sb + kOffA2, *gHi = sb + kOffG, *gLo = sb + kOffG2;
    float *sKV = reinterpret_cast<float *>(sb + kOffKV);
    float *sH = reinterpret_cast<float *>(sb + kOffH);
    float *sLP = reinterpret_cast<float *>(sb + kOffLP);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sb + kOffBar + 32);
    // barriers: MMA completion, weight region B (Wqkv / W1), Wo (G region), W2 (k|v region)
    const uint32_t mb = base + kOffBar, bWB = mb + 8, bWO = mb + 16, bW2 = mb + 24;
    const uint32_t uA = base + kOffA, uA2 = base + kOffA2, uG = base + kOffG, uG2 = base + kOffG2;
    const uint32_t uKV = base + kOffKV, uWB = base + kOffWB;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q4 = warp & 3, cq = warp >> 2, row = 32 * q4 + lane;
    const int T = g.T, rows_used = g.spt * T;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(tslot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int b = 0; b < 4; ++b) tc::mbar_init(mb + 8u * b, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const uint32_t tl = tmem + (uint32_t(32 * q4) << 16);

    bool ok = true;
    uint32_t ph_mma = 0;
    uint32_t n_wb = 0, d_wb = 0, n_wo = 0, d_wo = 0, n_w2 = 0, d_w2 = 0;  // copies issued / waited per barrier
    auto sync_async = [&]() {
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
    };
    auto wait_mma = [&]() {
        ok = __syncthreads_and(tc::mbar_wait(mb, ph_mma) ? 1 : 0) != 0;
        ph_mma ^= 1u;
        tc::fence_after_sync();
    };
    auto wait_bar = [&](uint32_t bar, uint32_t &done) {
        ok = __syncthreads_and(tc::mbar_wait(bar, done & 1u) ? 1 : 0) != 0;
        if (ok) ++done;
    };
    // weight copies (thread 0 issues; every thread counts)
    auto issue_wqkv = [&](int l) {
        constexpr uint32_t q = kQKV * 128;
        if (tid == 0) {
            tc::fence_async_smem();
            tc::mbar_expect(bWB, SPLIT ? 2 * q : q);
            ff_bulk(sb + kOffWB, g.tqkv[l], q, bWB);
            if (SPLIT) ff_bulk(sb + kOffWB + q, static_cast<const __nv_bfloat16 *>(g.tqkv[l]) + kQKV * kD, q, bWB);
        }
        ++n_wb;
    };
    auto issue_w1_wo = [&](int l) {
        constexpr uint32_t b1 = kF * 128, bo = kD * 128;
        if (tid == 0) {
            tc::fence_async_smem();
            tc::mbar_expect(bWB, SPLIT ? 2 * b1 : b1);
            ff_bulk(sb + kOffWB, g.t1[l], b1, bWB);
            if (SPLIT) ff_bulk(sb + kOffWB + b1, static_cast<const __nv_bfloat16 *>(g.t1[l]) + kF * kD, b1, bWB);
            tc::mbar_expect(bWO, SPLIT ? 2 * bo : bo);
            ff_bulk(gHi, g.to[l], bo, bWO);
            if (SPLIT) ff_bulk(gHi + bo, static_cast<const __nv_bfloat16 *>(g.to[l]) + kD * kD, bo, bWO);
        }
        ++n_wb;
        ++n_wo;
    };
    auto issue_w2 = [&](int l) {
        constexpr uint32_t b2 = kD * kF * 2;  // four 8 KB K blocks
        if (tid == 0) {
            tc::fence_async_smem();
            tc::mbar_expect(bW2, SPLIT ? 2 * b2 : b2);
            ff_bulk(sb + kOffKV, g.t2[l], b2, bW2);
            if (SPLIT) ff_bulk(sb + kOffKV + b2, static_cast<const __nv_bfloat16 *>(g.t2[l]) + kD * kF, b2, bW2);
        }
        ++n_w2;
    };

    if (blockIdx.x < g.n_tiles) issue_wqkv(0);
    const float qscale = (1.0f / sqrtf(float(DH))) * kLog2e;  // scores in base-2 units
    for (int64_t tile = blockIdx.x; tile < g.n_tiles && ok; tile += gridDim.x) {
        const int64_t s0 = tile * g.spt;
        // embeddings of the tile's rows (padding rows and samples past n: zero)
        for (int e = tid; e < kRows * (kD / 4); e += kThreads) {
            const int r = e >> 4, c4 = e & 15;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (r < rows_used) {
                const int sl = r / T, t = r - sl * T;
                const int64_t i = s0 + sl;
                if (i < g.n) {
                    const int inp = t == 0 ? 4 : ff_token(g.x + i * g.W, T, t - 1);
                    const float4 te = __ldg(reinterpret_cast<const float4 *>(g.tok + inp * kD) + c4);
                    const float4 pe = __ldg(reinterpret_cast<const float4 *>(g.pos + t * kD) + c4);
                    v = make_float4(te.x + pe.x, te.y + pe.y, te.z + pe.z, te.w + pe.w);
                }
            }
            float *hr = sH + r * kHS + 4 * c4;
            hr[0] = v.x;
            hr[1] = v.y;
            hr[2] = v.z;
            hr[3] = v.w;
        }
        __syncthreads();
        for (int l = 0; l < g.L && ok; ++l) {
            // ---- LN1 -> A; qkv product
            {
                const int lr = 8 * warp + (lane >> 2), lq = lane & 3;
                const LnOut n1 = ff_layernorm(sH, lr, lq, g.ln1g[l], g.ln1b[l], aHi, aLo, SPLIT);
                if constexpr (KEEP >= 1) {
                    const int64_t gr = s0 * T + lr, at = (int64_t)l * g.rows + gr;
                    if (lr < rows_used && gr < g.rows) {
                        float hv[16];
#pragma unroll
                        for (int c = 0; c < 16; ++c) hv[c] = sH[lr * kHS + ln_col(lq, c)];
                        ff_st_part(g.hbuf + at * kD, lq, hv);
                        if constexpr (KEEP >= 2) {
                            ff_st_part(g.a + at * kD, lq, n1.y);
                            if (lq == 0) {
                                g.mean1[at] = n1.mu;
                                g.rstd1[at] = n1.rs;
                            }
                        }
                    }
                }
            }
            wait_bar(bWB, d_wb);
            sync_async();
            if (!ok) break;
            if (tid == 0) {
                ff_mma(tmem + kColQ, uA, uA2, uWB, uWB + kQKV * 128, kQKV, SPLIT, false);
                tc::mma_commit(mb);
            }
            wait_mma();
            if (!ok) break;
            issue_w1_wo(l);  // Wqkv consumed: W1 over it, Wo into the G region
            // ---- k | v + bias into shared memory (thread: 32 columns of its row)
            {
                const float *bq = g.bqkv[l];
#pragma unroll
                for (int hf = 0; hf < 2; ++hf) {
                    const int tc0 = 64 + 32 * cq + 16 * hf;  // TMEM column = bias index
                    uint32_t r16[16];
                    tc::tmem_ld16(tl + tc0, r16);
                    float bv[16];
                    ff_ld16(bq + tc0, bv);
#pragma unroll
                    for (int p = 0; p < 4; ++p) {
                        const int c = tc0 - 64 + 4 * p;  // column of k | v
                        float4 v;
                        v.x = __uint_as_float(r16[4 * p]) + bv[4 * p];
                        v.y = __uint_as_float(r16[4 * p + 1]) + bv[4 * p + 1];
                        v.z = __uint_as_float(r16[4 * p + 2]) + bv[4 * p + 2];
                        v.w = __uint_as_float(r16[4 * p + 3]) + bv[4 * p + 3];
                        *reinterpret_cast<float4 *>(sKV + kv_at(row, c, row / T)) = v;
                        if constexpr (KEEP >= 2) {
                            const int64_t gr = s0 * T + row;
                            if (row < rows_used && gr < g.rows)
                                *reinterpret_cast<float4 *>(g.qkv + ((int64_t)l * g.rows + gr) * kQKV + tc0 + 4 * p) = v;
                        }
                    }
                }
            }
            __syncthreads();
            // ---- causal attention within the row's sample: thread (row,
            // quarter cq) takes heads cq HPT .. + HPT - 1 (q columns 16 cq ..)
            float o[16];
#pragma unroll
            for (int c = 0; c < 16; ++c) o[c] = 0.f;
            {
                uint32_t r16[16];
                tc::tmem_ld16(tl + kColQ + 16 * cq, r16);
                if (row < rows_used) {
                    const float *bq = g.bqkv[l];
                    float qv[16];
                    ff_ld16(bq + 16 * cq, qv);
#pragma unroll
                    for (int c = 0; c < 16; ++c) qv[c] += __uint_as_float(r16[c]);
                    const int sl = row / T, t = row - sl * T, r0 = sl * T;
                    const int64_t gr = s0 * T + row;
                    if constexpr (KEEP >= 2) {
                        if (gr < g.rows) ff_st16(g.qkv + ((int64_t)l * g.rows + gr) * kQKV + 16 * cq, qv);
                    }
#pragma unroll
                    for (int c = 0; c < 16; ++c) qv[c] *= qscale;
                    float m[HPT], ls[HPT];
#pragma unroll
                    for (int h = 0; h < HPT; ++h) {
                        m[h] = -INFINITY;
                        ls[h] = 0.f;
                    }
                    for (int j = 0; j <= t; ++j) {
                        const int rj = r0 + j;
                        float kk[16], vv[16];
#pragma unroll
                        for (int p = 0; p < 4; ++p) {
                            const float4 a = *reinterpret_cast<const float4 *>(sKV + kv_at(rj, 16 * cq + 4 * p, sl));
                            const float4 b =
                                *reinterpret_cast<const float4 *>(sKV + kv_at(rj, 64 + 16 * cq + 4 * p, sl));
                            kk[4 * p] = a.x; kk[4 * p + 1] = a.y; kk[4 * p + 2] = a.z; kk[4 * p + 3] = a.w;
                            vv[4 * p] = b.x; vv[4 * p + 1] = b.y; vv[4 * p + 2] = b.z; vv[4 * p + 3] = b.w;
                        }
#pragma unroll
                        for (int h = 0; h < HPT; ++h) {
                            float sc = 0.f;
#pragma unroll
                            for (int c = 0; c < DH; ++c) sc += qv[h * DH + c] * kk[h * DH + c];
                            const float mn = sc > m[h] ? sc : m[h];
                            const float corr = ff_ex2(m[h] - mn);
                            const float p = ff_ex2(sc - mn);
                            ls[h] = ls[h] * corr + p;
#pragma unroll
                            for (int c = 0; c < DH; ++c) o[h * DH + c] = o[h * DH + c] * corr + p * vv[h * DH + c];
                            m[h] = mn;
                        }
                    }
#pragma unroll
                    for (int h = 0; h < HPT; ++h) {
                        const float inv = 1.0f / ls[h];
#pragma unroll
                        for (int c = 0; c < DH; ++c) o[h * DH + c] *= inv;
                    }
                    if constexpr (KEEP >= 2) {
                        if (gr < g.rows) {
                            ff_st16(g.o + ((int64_t)l * g.rows + gr) * kD + 16 * cq, o);
                            // log-sum-exp of each head's scores, natural units
                            const int64_t i = s0 + sl;
#pragma unroll
                            for (int h = 0; h < HPT; ++h)
                                g.lse[(((int64_t)l * g.n + i) * H + cq * HPT + h) * T + t] =
                                    (m[h] + log2f(ls[h])) * 0.69314718055994530942f;
                        }
                    }
                }
            }
            tc::fence_async_smem();  // (every thread: its generic accesses before the async copy below)
            __syncthreads();         // k | v and q read by everyone
            issue_w2(l);             // the k | v region takes W2
            ff_granule(aHi, aLo, row, 2 * cq, o, SPLIT);
            ff_granule(aHi, aLo, row, 2 * cq + 1, o + 8, SPLIT);
            wait_bar(bWO, d_wo);
            sync_async();
            if (!ok) break;
            // ---- out-projection + residual
            if (tid == 0) {
                ff_mma(tmem + kColO, uA, uA2, uG, uG + kD * 128, kD, SPLIT, false);
                tc::mma_commit(mb);
            }
            wait_mma();
            if (!ok) break;
            {
                uint32_t r16[16];
                tc::tmem_ld16(tl + kColO + 16 * cq, r16);
                float hv[16], bv[16];
                ff_ld16(g.bo[l] + 16 * cq, bv);
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int c = 16 * cq + j;
                    hv[j] = sH[row * kHS + c] + (__uint_as_float(r16[j]) + bv[j]);
                    sH[row * kHS + c] = hv[j];
                }
                if constexpr (KEEP >= 1) {
                    const int64_t gr = s0 * T + row;
                    if (row < rows_used && gr < g.rows) ff_st16(g.hmid + ((int64_t)l * g.rows + gr) * kD + 16 * cq, hv);
                }
            }
            __syncthreads();
            // ---- LN2 -> A; the four FFN-in chunks issued together
            {
                const int lr = 8 * warp + (lane >> 2), lq = lane & 3;
                const LnOut n2 = ff_layernorm(sH, lr, lq, g.ln2g[l], g.ln2b[l], aHi, aLo, SPLIT);
                if constexpr (KEEP >= 2) {
                    const int64_t gr = s0 * T + lr, at = (int64_t)l * g.rows + gr;
                    if (lr < rows_used && gr < g.rows) {
                        ff_st_part(g.a2 + at * kD, lq, n2.y);
                        if (lq == 0) {
                            g.mean2[at] = n2.mu;
                            g.rstd2[at] = n2.rs;
                        }
                    }
                }
            }
            wait_bar(bWB, d_wb);
            sync_async();
            if (!ok) break;
            if (tid == 0) {
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    ff_mma(tmem + kColU + 64 * c, uA, uA2, uWB + 8192 * c, uWB + kF * 128 + 8192 * c, kD, SPLIT,
                           false);
                tc::mma_commit(mb);
            }
            wait_mma();
            if (!ok) break;
            // W1 consumed: the next Wqkv (this tile's next layer, or the first
            // layer of this CTA's next tile) comes in during the FFN
            if (l + 1 < g.L)
                issue_wqkv(l + 1);
            else if (tile + gridDim.x < g.n_tiles)
                issue_wqkv(0);
            wait_bar(bW2, d_w2);
            if (!ok) break;
            // ---- per chunk: GELU(U_c + b1) -> G while the previous FFN-out
            // product runs, then Y += G W2_c^T
            for (int c = 0; c < 4 && ok; ++c) {
                float x[16];
                {
                    uint32_t r16[16];
                    tc::tmem_ld16(tl + kColU + 64 * c + 16 * cq, r16);
                    float uv[16];
                    ff_ld16(g.b1[l] + 64 * c + 16 * cq, uv);
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        uv[j] += __uint_as_float(r16[j]);
                        x[j] = ff_gelu(uv[j]);
                    }
                    if constexpr (KEEP >= 2) {
                        const int64_t gr = s0 * T + row;
                        if (row < rows_used && gr < g.rows) {
                            const int64_t at = ((int64_t)l * g.rows + gr) * kF + 64 * c + 16 * cq;
                            ff_st16(g.u + at, uv);
                            ff_st16(g.gu + at, x);
                        }
                    }
                }
                if (c > 0) {
                    wait_mma();
                    if (!ok) break;
                }
                ff_granule(gHi, gLo, row, 2 * cq, x, SPLIT);
                ff_granule(gHi, gLo, row, 2 * cq + 1, x + 8, SPLIT);
                sync_async();
                if (tid == 0) {
                    ff_mma(tmem + kColY, uG, uG2, uKV + 8192 * c, uKV + kD * kF * 2 + 8192 * c, kD, SPLIT, c > 0);
                    tc::mma_commit(mb);
                }
            }
            if (!ok) break;
            wait_mma();
            if (!ok) break;
            {
                uint32_t r16[16];
                tc::tmem_ld16(tl + kColY + 16 * cq, r16);
                float bv[16];
                ff_ld16(g.b2[l] + 16 * cq, bv);
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int c = 16 * cq + j;
                    sH[row * kHS + c] += __uint_as_float(r16[j]) + bv[j];
                }
            }
            __syncthreads();
        }
        if (!ok) break;
        // ---- final LayerNorm, head logits and the masked log-softmax of the
        // token each row predicts (position t predicts token t): 4 lanes per row
        {
            const int lr = 8 * warp + (lane >> 2), lq = lane & 3;
            const LnOut nf = ff_layernorm(sH, lr, lq, g.lnf_g, g.lnf_b, nullptr, nullptr, false);
            float z[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                float a = 0.f, wv[16];
                ff_ld_part(g.hw + k * kD, lq, wv);
#pragma unroll
                for (int c = 0; c < 16; ++c) a += nf.y[c] * wv[c];
                a += __shfl_xor_sync(0xffffffffu, a, 1);
                a += __shfl_xor_sync(0xffffffffu, a, 2);
                z[k] = a + __ldg(g.hb + k);
            }
            const int sl = lr / T, t = lr - sl * T;
            const int64_t i = s0 + sl, gr = s0 * T + lr;
            const bool valid = lr < rows_used && i < g.n;
            if constexpr (KEEP >= 1) {
                if (valid) {
                    float hv[16];
#pragma unroll
                    for (int c = 0; c < 16; ++c) hv[c] = sH[lr * kHS + ln_col(lq, c)];
                    ff_st_part(g.hbuf + ((int64_t)g.L * g.rows + gr) * kD, lq, hv);
                    ff_st_part(g.hf + gr * kD, lq, nf.y);
                    if (lq == 0) {
                        g.meanf[gr] = nf.mu;
                        g.rstdf[gr] = nf.rs;
                    }
                }
            }
            if (lq == 0) {
                float lp = 0.f;
                if (valid) {
                    const uint64_t *xi = g.x + i * g.W;
                    int ca = 0, cb = 0;  // electrons on the orbitals of tokens < t
                    for (int p2 = T - t; p2 < T; ++p2) {
                        ca += ff_bit(xi, 2 * p2);
                        cb += ff_bit(xi, 2 * p2 + 1);
                    }
                    const int rem = T - 1 - t;
                    bool okv[4];
                    float zmax = -INFINITY;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int a = ca + (k & 1), b = cb + (k >> 1);
                        okv[k] = a <= g.n_alpha && b <= g.n_beta && a + rem >= g.n_alpha && b + rem >= g.n_beta;
                        if (okv[k] && z[k] > zmax) zmax = z[k];
                    }
                    float se = 0.f;
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (okv[k]) se += expf(z[k] - zmax);
                    const float lse = zmax + logf(se);
                    const int tk = ff_token(xi, T, t);
                    lp = okv[tk] ? z[tk] - lse : -INFINITY;
                    if constexpr (KEEP >= 1) {
#pragma unroll
                        for (int k = 0; k < 4; ++k) g.pi[gr * 4 + k] = okv[k] ? expf(z[k] - lse) : 0.f;
                        g.tok_out[gr] = (uint8_t)tk;
                    }
                }
                sLP[lr] = lp;
            }
        }
        __syncthreads();
        if (tid < g.spt) {
            const int64_t i = s0 + tid;
            if (i < g.n) {
                float sum = 0.f;
                bool bad = false;
                for (int t = 0; t < T; ++t) {
                    const float v = sLP[tid * T + t];
                    if (v == -INFINITY)
                        bad = true;
                    else
                        sum += v;
                }
                g.out[i].x = bad ? -(double)INFINITY : 0.5 * (double)sum;
                if (bad) record_status(g.st, NNQS_E_SECTOR, g.row_offset + i);
            }
        }
        __syncthreads();
    }
    if (!ok && tid == 0) {
        if (atomicCAS(&g.st->code, 0, (int)NNQS_E_TIMEOUT) == 0) g.st->index = -13;
        // weight copies still in flight land (bounded) before the CTA ends
        for (; d_wb < n_wb; ++d_wb) tc::mbar_wait(bWB, d_wb & 1u);
        for (; d_wo < n_wo; ++d_wo) tc::mbar_wait(bWO, d_wo & 1u);
        for (; d_w2 < n_w2; ++d_w2) tc::mbar_wait(bW2, d_w2 & 1u);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ff::kTmemCols)
                     : "memory");
    }
}

template <bool SPLIT, int DH, int KEEP>
nnqs_status launch_fused(const FusedFwdArgs &a, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        NNQS_CUDA_TRY(cudaFuncSetAttribute(k_fwd_fused<SPLIT, DH, KEEP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           ff::kSmem));
        attr = true;
    }
    const int64_t grid = std::min<int64_t>(a.n_tiles, num_sms());
    NNQS_LAUNCH("k_fwd_fused", s, (k_fwd_fused<SPLIT, DH, KEEP><<<(unsigned)grid, ff::kThreads, ff::kSmem, s>>>(a)));
    return NNQS_OK;
}

template <int KEEP>
nnqs_status launch_fused_keep(const FusedFwdArgs &a, bool split, int dh, cudaStream_t s) {
    if (split) return dh == 8 ? launch_fused<true, 8, KEEP>(a, s) : launch_fused<true, 16, KEEP>(a, s);
    return dh == 8 ? launch_fused<false, 8, KEEP>(a, s) : launch_fused<false, 16, KEEP>(a, s);
}

}  // namespace

bool fused_fwd_aligned(const FusedFwdArgs &a) {
    auto al = [](const void *p) { return reinterpret_cast<uintptr_t>(p) % 16 == 0; };
    bool ok = al(a.tok) && al(a.pos) && al(a.lnf_g) && al(a.lnf_b) && al(a.hw);
    for (int l = 0; l < a.L; ++l)
        ok = ok && al(a.ln1g[l]) && al(a.ln1b[l]) && al(a.bqkv[l]) && al(a.bo[l]) && al(a.ln2g[l]) &&
             al(a.ln2b[l]) && al(a.b1[l]) && al(a.b2[l]) && al(a.tqkv[l]) && al(a.to[l]) && al(a.t1[l]) &&
             al(a.t2[l]);
    return ok;
}

bool fused_fwd_supported(int d, int F, int dh, int T, int L) {
    return d == ff::kD && F == ff::kF && (dh == 8 || dh == 16) && T >= 1 && T <= 64 && L >= 1 &&
           L <= kFusedMaxLayers;
}

nnqs_status fused_fwd_launch(const FusedFwdArgs &a, bool split, int dh, cudaStream_t s) {
    if (a.n <= 0) return NNQS_OK;
    if (a.spt < 1 || a.spt * a.T > ff::kRows) return set_error(NNQS_E_INVAL, "fused forward: bad tile shape");
    note_work("k_fwd_fused",
              double(a.n) * a.T * a.L * 2.0 * (4.0 * ff::kD * ff::kD + 2.0 * ff::kD * ff::kF),
              double(a.n) * (8.0 * a.W + 8.0));
    if (a.hbuf) return a.a ? launch_fused_keep<2>(a, split, dh, s) : launch_fused_keep<1>(a, split, dh, s);
    return launch_fused_keep<0>(a, split, dh, s);
}

}  // namespace nnqs
