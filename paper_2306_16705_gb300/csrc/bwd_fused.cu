// Fused reverse mode of the decoder layers (Sec. 3.1; the energy gradient of
// Sec. 2.1) on tcgen05 tensor cores.
//
// FFN half of a layer (k_bwd_ffn), per 128-row tile of token rows:
//   a2 = LN2(hmid)                       (recomputed, split BF16 when the forward was)
//   u = a2 W1^T + b1, gu = GELU(u)       (recomputed on the tensor cores)
//   dgu = dy W2, du = dgu * GELU'(u)
//   da2 = du W1, dhmid = dy + LN2'(da2)  (written over dy)
//   dW2 += dy^T gu, dW1 += du^T a2, db1 += sum du, dgamma2 / dbeta2 / dbo
// The FFN width is walked in two halves of 128 so that the weight-gradient
// accumulators (dW1 and dW2^T, 256 TMEM columns) stay in TMEM over every tile
// of the CTA; the weight-gradient products read their operands transposed
// (MN-major descriptors) from the same swizzled tiles the other products read
// K-major, so nothing is copied to transpose it.  Each CTA writes one
// partial; bwd_ffn_reduce adds them in CTA order (deterministic).
//
// Shared memory (1024-aligned base):
//   [0, 32K)      a2 hi / lo            [128][64] BF16, 128-byte swizzle
//   [32K, 48K)    dy                    [128][64] BF16
//   [48K, 80K)    gu of the half        two [128][64] panels
//   [80K, 112K)   du of the half        two [128][64] panels
//   [112K, 176K)  W1 image hi / lo      [256][64]
//   [176K, 208K)  W2 image hi           four [64][64] K blocks
//   [208K, 216K)  row-sum exchange, then the column-sum combine
// TMEM: dW1 [0, 128) (halves 64 columns each), dW2^T [128, 256), u / dgu of
// the half [256, 384), da2 [384, 448).
//
// Every wait is bounded (tc::mbar_wait): on a timeout the CTA records
// NNQS_E_TIMEOUT, lets its weight copies land (bounded) and frees its TMEM.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "bwd_fused.cuh"
#include "dev_common.cuh"
#include "tc_gemm.cuh"

namespace nnqs {
namespace {
namespace fb {
constexpr int kThreads = 512, kRows = 128, kD = 64, kF = 256;
constexpr int kOffA = 0, kOffA2 = 16384, kOffDY = 32768, kOffGU = 49152, kOffDU = 81920;
constexpr int kOffW1 = 114688, kOffW2 = 180224, kOffRed = 212992;
constexpr int kOffBar = kOffRed + 8192;
constexpr int kSmem = kOffBar + 64 + 1024;  // 222,272 bytes
constexpr uint32_t kColW1 = 0, kColW2 = 128, kColU = 256, kColDA = 384, kTmemCols = 512;
constexpr int kCols = 448;  // column sums combined per CTA: db1 256 | dgamma2 64 | dbeta2 64 | dbo 64
}  // namespace fb

__device__ __forceinline__ void fb_bulk(uint8_t *dst, const void *src, uint32_t bytes, uint32_t mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     tc::smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(mbar)
                 : "memory");
}

// bring `bytes` (a multiple of 16, 16-byte aligned) of global memory into L2
__device__ __forceinline__ void fb_prefetch_l2(const void *p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// the saved row of token row gr (see BwdRowSource)
__device__ __forceinline__ const float *fb_row(const float *base, int64_t gr, const BwdRowSource &src) {
    if (!src.anc) return base + gr * 64;
    const int64_t i = gr / src.T;
    const int t = int(gr - i * src.T);
    return base + int64_t(__ldg(src.anc + t * src.anc_stride + i)) * src.node_stride;
}

// the next tile's saved rows [r1, r1 + nr) into L2: one bulk prefetch when
// they are contiguous, else one 256-byte prefetch per row by threads 0 .. nr - 1
__device__ __forceinline__ void fb_prefetch_rows(const float *base, int64_t r1, int64_t nr, const BwdRowSource &src,
                                                 int tid) {
    if (!src.anc) {
        if (tid == 0) fb_prefetch_l2(base + r1 * 64, uint32_t(nr * 64 * 4));
    } else if (tid < nr) {
        fb_prefetch_l2(fb_row(base, r1 + tid, src), 256u);
    }
}

// shared-memory descriptor of an MN-major (transposed) operand, 128-byte
// swizzle: 128-byte rows of 64 BF16 along M (or N), one row per K index,
// 8-row groups along K 1024 bytes apart, 64-wide M (N) blocks `lbo` bytes apart
__device__ __forceinline__ uint64_t desc_mn(uint32_t saddr, uint32_t lbo) {
    uint64_t d = 0;
    d |= uint64_t((saddr >> 4) & 0x3FFFu);
    d |= uint64_t((lbo >> 4) & 0x3FFFu) << 16;
    d |= uint64_t(1024u >> 4) << 32;
    d |= uint64_t(1) << 46;
    d |= uint64_t(2) << 61;
    return d;
}

// kind::f16 instruction descriptor (BF16 in, FP32 out) with the transpose
// (MN-major) flags of A and B
__device__ __forceinline__ uint32_t idesc_t(int M, int N, bool ta, bool tb) {
    return tc::idesc_bf16(M, N) | (uint32_t(ta) << 15) | (uint32_t(tb) << 16);
}

__device__ __forceinline__ float fb_ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// GELU(x) = x Phi(x) and GELU'(x) = Phi(x) + x phi(x), with erf from
// Abramowitz and Stegun (1964) eq. 7.1.26 as in the fused forward (absolute
// error at most 1.5e-7); e^{-x^2 / 2} serves both erf and phi
__device__ __forceinline__ void fb_gelu2(float x, float &g, float &dg) {
    const float z = fabsf(x) * 0.70710678118654752f;
    const float t = __fdividef(1.0f, fmaf(0.3275911f, z, 1.0f));
    const float poly =
        t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.061405429f, -1.453152027f), 1.421413741f), -0.284496736f), 0.254829592f);
    const float e = fb_ex2(-(z * z) * 1.44269504088896340736f);
    const float phi_cdf = 0.5f * (1.0f + copysignf(1.0f - poly * e, x));
    g = x * phi_cdf;
    dg = phi_cdf + x * e * 0.39894228040143267794f;
}

// 16 floats from a 16-byte aligned address (read-only data)
__device__ __forceinline__ void fb_ldg16(const float *__restrict__ p, float (&v)[16]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float4 a = __ldg(reinterpret_cast<const float4 *>(p) + k);
        v[4 * k] = a.x;
        v[4 * k + 1] = a.y;
        v[4 * k + 2] = a.z;
        v[4 * k + 3] = a.w;
    }
}

__device__ __forceinline__ void fb_st16(float *p, const float *v) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
        reinterpret_cast<float4 *>(p)[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
}

// 8 values as granule `gi` of row r of a swizzled [128][64] BF16 panel (hi),
// and their low parts v - bf16(v) in `lo` when given
__device__ __forceinline__ void fb_granule(uint8_t *hi, uint8_t *lo, int r, int gi, const float *v) {
    float x[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) x[e] = v[e];
    const int off = r * 128 + ((gi ^ (r & 7)) << 4);
    *reinterpret_cast<uint4 *>(hi + off) = tc::pack8(x);
    if (lo) {
        float y[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) y[e] = x[e] - __bfloat162float(__float2bfloat16_rn(x[e]));
        *reinterpret_cast<uint4 *>(lo + off) = tc::pack8(y);
    }
}

// Sums over the warp's 32 lanes (one row each) of v[0 .. N): recursive
// halving, each lane keeping the half of the remaining columns its lane bit
// selects and adding the partner's copy of them (N - 1 shuffles).  Lane l
// returns the sum of column l (N = 32) or of column l >> 1 (N = 16).  v is
// consumed.
template <int N>
__device__ __forceinline__ float fb_colsum(float (&v)[N], int lane) {
    static_assert(N == 32 || N == 16, "16 or 32 columns");
#pragma unroll
    for (int half = N / 2, m = 16; half >= 1; half >>= 1, m >>= 1) {
        const bool up = (lane & m) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const float send = up ? v[i] : v[i + half];
            const float keep = up ? v[i + half] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, m);
        }
    }
    float r = v[0];
    if (N == 16) r += __shfl_xor_sync(0xffffffffu, r, 1);
    return r;
}

// ---- Four lanes per row.  The LayerNorm phases touch the rows in global
// memory; with one row per lane (the TMEM lane mapping) a warp's 16-byte
// access spans 32 rows and costs 32 L1 wavefronts.  There, lanes 4 r' .. 4 r' + 3
// of a warp hold tile row tid / 4 instead, lane lq = tid % 4 the float4
// pieces lq + 4 m of it (columns 16 m + 4 lq .. + 3, m = 0..3, v[4 m + e]),
// so one access covers eight whole 256-byte rows.

__device__ __forceinline__ void fb_ld_row4(const float *__restrict__ p, int lq, float (&v)[16]) {
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const float4 a = __ldg(reinterpret_cast<const float4 *>(p) + lq + 4 * m);
        v[4 * m] = a.x;
        v[4 * m + 1] = a.y;
        v[4 * m + 2] = a.z;
        v[4 * m + 3] = a.w;
    }
}

// the same for rows this kernel also writes (no read-only path)
__device__ __forceinline__ void fb_ld_row4_rw(const float *p, int lq, float (&v)[16]) {
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const float4 a = reinterpret_cast<const float4 *>(p)[lq + 4 * m];
        v[4 * m] = a.x;
        v[4 * m + 1] = a.y;
        v[4 * m + 2] = a.z;
        v[4 * m + 3] = a.w;
    }
}

__device__ __forceinline__ void fb_st_row4(float *p, int lq, const float (&v)[16]) {
#pragma unroll
    for (int m = 0; m < 4; ++m)
        reinterpret_cast<float4 *>(p)[lq + 4 * m] = make_float4(v[4 * m], v[4 * m + 1], v[4 * m + 2], v[4 * m + 3]);
}

// sum over the row's four lanes
__device__ __forceinline__ float fb_sum4(float s) {
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    return s;
}

// mean and 1 / sqrt(variance + 1e-5) of a row held in four lanes
__device__ __forceinline__ void fb_ln_stats4(const float (&v)[16], float &mu, float &rs) {
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < 16; ++c) s += v[c];
    mu = fb_sum4(s) * (1.0f / 64);
    float q = 0.f;
#pragma unroll
    for (int c = 0; c < 16; ++c) q += (v[c] - mu) * (v[c] - mu);
    rs = 1.0f / sqrtf(fb_sum4(q) * (1.0f / 64) + 1e-5f);
}

// a lane's four pieces of row r as half granules (4 BF16) of a swizzled
// [128][64] panel: the high part, and the low part v - bf16(v) when lo is set
__device__ __forceinline__ void fb_half_granules(uint8_t *hi, uint8_t *lo, int r, int lq, const float (&v)[16]) {
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int k = lq + 4 * m, c = k >> 1;
        const int off = r * 128 + ((c ^ (r & 7)) << 4) + 8 * (k & 1);
        const __nv_bfloat162 h0 = __floats2bfloat162_rn(v[4 * m], v[4 * m + 1]);
        const __nv_bfloat162 h1 = __floats2bfloat162_rn(v[4 * m + 2], v[4 * m + 3]);
        *reinterpret_cast<uint2 *>(hi + off) =
            make_uint2(*reinterpret_cast<const uint32_t *>(&h0), *reinterpret_cast<const uint32_t *>(&h1));
        if (lo) {
            const __nv_bfloat162 l0 = __floats2bfloat162_rn(v[4 * m] - __low2float(h0), v[4 * m + 1] - __high2float(h0));
            const __nv_bfloat162 l1 =
                __floats2bfloat162_rn(v[4 * m + 2] - __low2float(h1), v[4 * m + 3] - __high2float(h1));
            *reinterpret_cast<uint2 *>(lo + off) =
                make_uint2(*reinterpret_cast<const uint32_t *>(&l0), *reinterpret_cast<const uint32_t *>(&l1));
        }
    }
}

// first of the two columns whose sums fb_colsum8 leaves in lane `lane`
__device__ __forceinline__ int fb_col8(int lane) {
    return 16 * (2 * ((lane >> 4) & 1) + ((lane >> 3) & 1)) + 4 * (lane & 3) + 2 * ((lane >> 2) & 1);
}

// Column sums over the warp's eight rows (the lanes with the same lq) of a
// lane's 16 columns: recursive halving over lane bits 16, 8, 4 (14
// shuffles); the lane returns the sums of columns fb_col8(lane) and + 1.  v is
// consumed.
__device__ __forceinline__ float2 fb_colsum8(float (&v)[16], int lane) {
#pragma unroll
    for (int half = 8, m = 16; half >= 2; half >>= 1, m >>= 1) {
        const bool up = (lane & m) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const float send = up ? v[i] : v[i + half];
            const float keep = up ? v[i + half] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, m);
        }
    }
    return make_float2(v[0], v[1]);
}

// da (a TMEM accumulator, one row per lane) through shared memory [128][68]
// FP32 into the four-lanes-per-row mapping: the TMEM-mapped thread (row,
// columns 16 cq ..) stores, every thread reads its row r4's pieces after the
// barrier the caller places between
constexpr int kDaS = 68;
__device__ __forceinline__ void fb_da_store(float *daS, int row, int cq, const uint32_t (&r16)[16]) {
#pragma unroll
    for (int j = 0; j < 4; ++j)
        *reinterpret_cast<float4 *>(daS + row * kDaS + 16 * cq + 4 * j) =
            make_float4(__uint_as_float(r16[4 * j]), __uint_as_float(r16[4 * j + 1]), __uint_as_float(r16[4 * j + 2]),
                        __uint_as_float(r16[4 * j + 3]));
}
__device__ __forceinline__ void fb_da_load(const float *daS, int r4, int lq, float (&v)[16]) {
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const float4 a = *reinterpret_cast<const float4 *>(daS + r4 * kDaS + 4 * (lq + 4 * m));
        v[4 * m] = a.x;
        v[4 * m + 1] = a.y;
        v[4 * m + 2] = a.z;
        v[4 * m + 3] = a.w;
    }
}

// one 128 x N product over K = 64 (four K = 16 steps) from K-major A and B
// tiles; with split operands lo.hi + hi.lo + hi.hi per step
__device__ __forceinline__ void fb_mma_kmajor(uint32_t tmem, uint32_t aHi, uint32_t aLo, uint32_t bHi, uint32_t bLo,
                                              int N, bool split, bool acc0) {
    const uint32_t idesc = tc::idesc_bf16(fb::kRows, N);
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

// D[M = 128][N] (+)= A^T B over the tile's 128 rows (K): A and B are row-major
// [128 rows][features] swizzled tiles read MN-major; A spans two 64-feature
// panels `lboA` bytes apart, B one
__device__ __forceinline__ void fb_mma_rows(uint32_t tmem, uint32_t a, uint32_t lboA, uint32_t b, int N, bool acc0) {
    const uint32_t idesc = idesc_t(fb::kRows, N, true, true);
#pragma unroll
    for (int k = 0; k < 8; ++k)
        tc::mma_bf16(tmem, desc_mn(a + 2048u * k, lboA), desc_mn(b + 2048u * k, 16384u), idesc,
                     (acc0 || k > 0) ? 1u : 0u);
}

template <bool SPLIT>
__global__ void __launch_bounds__(fb::kThreads, 1) k_bwd_ffn(const __grid_constant__ BwdFfnArgs g) {
    using namespace fb;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = tc::smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *sb = smem_raw + (base - raw);
    float *red = reinterpret_cast<float *>(sb + kOffRed);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sb + kOffBar + 32);
    const uint32_t mb = base + kOffBar, bW = mb + 8;
    const uint32_t uA = base + kOffA, uA2 = base + kOffA2, uDY = base + kOffDY, uGU = base + kOffGU;
    const uint32_t uDU = base + kOffDU, uW1 = base + kOffW1, uW2 = base + kOffW2;
    uint8_t *aHi = sb + kOffA, *aLo = SPLIT ? sb + kOffA2 : nullptr;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q4 = warp & 3, cq = warp >> 2, row = 32 * q4 + lane;
    const int r4 = tid >> 2, lq = tid & 3;
    const int64_t n_tiles = (g.rows + kRows - 1) / kRows;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(tslot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        tc::mbar_init(mb, 1);
        tc::mbar_init(bW, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const uint32_t tl = tmem + (uint32_t(32 * q4) << 16);

    // the weight images, once per CTA
    constexpr uint32_t kWB = kF * kD * 2;  // 32 KB
    if (tid == 0) {
        tc::mbar_expect(bW, (SPLIT ? 3u : 2u) * kWB);
        fb_bulk(sb + kOffW1, g.t1, kWB, bW);
        if (SPLIT) fb_bulk(sb + kOffW1 + kWB, static_cast<const __nv_bfloat16 *>(g.t1) + kF * kD, kWB, bW);
        fb_bulk(sb + kOffW2, g.t2, kWB, bW);
    }
    bool ok = __syncthreads_and(tc::mbar_wait(bW, 0) ? 1 : 0) != 0;
    const bool w_landed = ok;
    uint32_t ph = 0;
    auto sync_async = [&]() {
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
    };
    auto wait_mma = [&]() {
        ok = __syncthreads_and(tc::mbar_wait(mb, ph) ? 1 : 0) != 0;
        ph ^= 1u;
        tc::fence_after_sync();
    };

    float cs_b1a = 0.f, cs_b1b = 0.f;  // column sums of du (db1 halves), one column per lane
    // column sums of the LN2 parameters' gradients and dbo over this warp's
    // rows, columns fb_col8(lane) and + 1
    float2 cs_g = make_float2(0.f, 0.f), cs_b = make_float2(0.f, 0.f), cs_o = make_float2(0.f, 0.f);
    bool first = true;
    for (int64_t tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
        // rows of the four-lanes-per-row phases: tile row r4, global row g4
        const int64_t g4 = tile * kRows + r4;
        const bool ok4 = g4 < g.rows;
        if (tile + gridDim.x < n_tiles) {  // the next tile's rows into L2 meanwhile
            const int64_t r1 = (tile + gridDim.x) * kRows, nr = g.rows - r1 < kRows ? g.rows - r1 : kRows;
            fb_prefetch_rows(g.hmid, r1, nr, g.src, tid);
            if (tid == 0) fb_prefetch_l2(g.dh + r1 * kD, uint32_t(nr * kD * 4));
        }
        // ---- LN2 of the saved residual rows -> a2 (A); dy -> DY (four lanes
        // per row; rows past the end are zero)
        {
            float hv[16], dv[16];
            if (ok4) {
                fb_ld_row4(fb_row(g.hmid, g4, g.src), lq, hv);
                fb_ld_row4_rw(g.dh + g4 * kD, lq, dv);
            } else {
#pragma unroll
                for (int c = 0; c < 16; ++c) hv[c] = dv[c] = 0.f;
            }
            float mu, rs;
            fb_ln_stats4(hv, mu, rs);
            float gv[16], bv[16], y[16];
            fb_ld_row4(g.ln2g, lq, gv);
            fb_ld_row4(g.ln2b, lq, bv);
#pragma unroll
            for (int c = 0; c < 16; ++c) y[c] = ok4 ? (hv[c] - mu) * rs * gv[c] + bv[c] : 0.f;
            fb_half_granules(aHi, aLo, r4, lq, y);
            fb_half_granules(sb + kOffDY, nullptr, r4, lq, dv);
        }
        sync_async();
        if (tid == 0) {
            fb_mma_kmajor(tmem + kColU, uA, uA2, uW1, uW1 + kWB, 128, SPLIT, false);
            tc::mma_commit(mb);
        }
        for (int h = 0; h < 2 && ok; ++h) {
            wait_mma();
            if (!ok) break;
            // ---- GELU of u = U_h + b1 -> gu (BF16); GELU'(u) kept
            float gp[32];
            uint8_t *gpan = sb + kOffGU + (cq >> 1) * 16384;
            uint8_t *dpan = sb + kOffDU + (cq >> 1) * 16384;
            const int gbase = 4 * (cq & 1);
#pragma unroll
            for (int hf = 0; hf < 2; ++hf) {
                uint32_t r16[16];
                tc::tmem_ld16(tl + kColU + 32 * cq + 16 * hf, r16);
                float bv[16], x[16];
                fb_ldg16(g.b1 + 128 * h + 32 * cq + 16 * hf, bv);
#pragma unroll
                for (int j = 0; j < 16; ++j) fb_gelu2(__uint_as_float(r16[j]) + bv[j], x[j], gp[16 * hf + j]);
                fb_granule(gpan, nullptr, row, gbase + 2 * hf, x);
                fb_granule(gpan, nullptr, row, gbase + 2 * hf + 1, x + 8);
            }
            sync_async();
            if (tid == 0) {
                // dgu_h = dy W2[:, half h]: B is the FFN-out image read
                // transposed (K = its 64 rows, N = 128 of its columns)
                const uint32_t id = idesc_t(kRows, 128, false, true);
                const uint64_t dA = tc::desc_sw128(uDY);
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    tc::mma_bf16(tmem + kColU, dA + uint64_t(2 * k), desc_mn(uW2 + 2u * h * 8192u + 2048u * k, 8192u),
                                 id, k > 0 ? 1u : 0u);
                // dW2^T[half h] += gu_h^T dy
                fb_mma_rows(tmem + kColW2 + 64 * h, uGU, 16384u, uDY, kD, !first);
                tc::mma_commit(mb);
            }
            wait_mma();
            if (!ok) break;
            // ---- du = dgu * GELU'(u) -> DU (BF16); column sums for db1
            float du[32];
#pragma unroll
            for (int hf = 0; hf < 2; ++hf) {
                uint32_t r16[16];
                tc::tmem_ld16(tl + kColU + 32 * cq + 16 * hf, r16);
#pragma unroll
                for (int j = 0; j < 16; ++j) du[16 * hf + j] = __uint_as_float(r16[j]) * gp[16 * hf + j];
                fb_granule(dpan, nullptr, row, gbase + 2 * hf, du + 16 * hf);
                fb_granule(dpan, nullptr, row, gbase + 2 * hf + 1, du + 16 * hf + 8);
            }
            const float csu = fb_colsum<32>(du, lane);
            if (h == 0)
                cs_b1a += csu;
            else
                cs_b1b += csu;
            sync_async();
            if (tid == 0) {
                // da2 += du_h W1[half h]: B is the FFN-in image read
                // transposed (K = 128 of its rows, N = its 64 columns)
                const uint32_t id = idesc_t(kRows, kD, false, true);
#pragma unroll
                for (int kb = 0; kb < 2; ++kb) {
                    const uint64_t dA = tc::desc_sw128(uDU + 16384u * kb);
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        tc::mma_bf16(tmem + kColDA, dA + uint64_t(2 * k),
                                     desc_mn(uW1 + uint32_t(128 * h + 64 * kb + 16 * k) * 128u, 16384u), id,
                                     (h | kb | k) ? 1u : 0u);
                }
                // dW1[half h] += du_h^T a2
                fb_mma_rows(tmem + kColW1 + 64 * h, uDU, 16384u, uA, kD, !first);
                // the second half's u (over the first half's dgu, read above)
                if (h == 0) fb_mma_kmajor(tmem + kColU, uA, uA2, uW1 + 16384u, uW1 + kWB + 16384u, 128, SPLIT, false);
                tc::mma_commit(mb);
            }
        }
        if (!ok) break;
        wait_mma();
        if (!ok) break;
        // ---- LN2 backward: dhmid = dy + rs (da2 g - mean(da2 g) - xh mean(da2 g xh)),
        // four lanes per row; da2 leaves TMEM through the (now free) gu | du region
        {
            float *daS = reinterpret_cast<float *>(sb + kOffGU);
            {
                uint32_t r16[16];
                tc::tmem_ld16(tl + kColDA + 16 * cq, r16);
                fb_da_store(daS, row, cq, r16);
            }
            __syncthreads();
            float hv[16], dv[16], gv[16], da[16], xh[16];
            if (ok4) {
                fb_ld_row4(fb_row(g.hmid, g4, g.src), lq, hv);
                fb_ld_row4_rw(g.dh + g4 * kD, lq, dv);
            } else {
#pragma unroll
                for (int c = 0; c < 16; ++c) hv[c] = dv[c] = 0.f;
            }
            fb_da_load(daS, r4, lq, da);
            fb_ld_row4(g.ln2g, lq, gv);
            float mu, rs;
            fb_ln_stats4(hv, mu, rs);
            float s1 = 0.f, s2 = 0.f;
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                xh[c] = ok4 ? (hv[c] - mu) * rs : 0.f;
                const float dx = da[c] * gv[c];
                s1 += dx;
                s2 += dx * xh[c];
            }
            const float m1 = fb_sum4(s1) * (1.0f / kD), m2 = fb_sum4(s2) * (1.0f / kD);
            float out[16], t[16];
#pragma unroll
            for (int c = 0; c < 16; ++c) out[c] = ok4 ? dv[c] + rs * (da[c] * gv[c] - m1 - xh[c] * m2) : 0.f;
            if (ok4) fb_st_row4(g.dh + g4 * kD, lq, out);
#pragma unroll
            for (int c = 0; c < 16; ++c) t[c] = da[c] * xh[c];
            const float2 sg = fb_colsum8(t, lane), sbt = fb_colsum8(da, lane), so = fb_colsum8(out, lane);
            cs_g.x += sg.x;
            cs_g.y += sg.y;
            cs_b.x += sbt.x;
            cs_b.y += sbt.y;
            cs_o.x += so.x;
            cs_o.y += so.y;
        }
        __syncthreads();
        first = false;
    }
    if (ok && !first) {
        // ---- this CTA's partial: the TMEM accumulators, then the column sums
        // of the four row quadrants added in order
        float *part = g.part + (int64_t)blockIdx.x * kBwdFfnPart;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            uint32_t r16[16];
            tc::tmem_ld16(tl + kColW1 + 64 * h + 16 * cq, r16);
            float v[16];
#pragma unroll
            for (int c = 0; c < 16; ++c) v[c] = __uint_as_float(r16[c]);
            fb_st16(part + (128 * h + row) * kD + 16 * cq, v);
            tc::tmem_ld16(tl + kColW2 + 64 * h + 16 * cq, r16);
#pragma unroll
            for (int c = 0; c < 16; ++c) part[kF * kD + (16 * cq + c) * kF + 128 * h + row] = __uint_as_float(r16[c]);
        }
        float *cs = red + q4 * kCols;
        cs[32 * cq + lane] = cs_b1a;
        cs[128 + 32 * cq + lane] = cs_b1b;
        // the LN2 and dbo sums per warp ([16][192] over the free gu region),
        // added in warp order
        float *lnp = reinterpret_cast<float *>(sb + kOffGU);
        const int c8 = fb_col8(lane);
        lnp[warp * 192 + c8] = cs_g.x;
        lnp[warp * 192 + c8 + 1] = cs_g.y;
        lnp[warp * 192 + 64 + c8] = cs_b.x;
        lnp[warp * 192 + 64 + c8 + 1] = cs_b.y;
        lnp[warp * 192 + 128 + c8] = cs_o.x;
        lnp[warp * 192 + 128 + c8 + 1] = cs_o.y;
        __syncthreads();
        for (int e = tid; e < kF; e += kThreads)
            part[2 * kF * kD + e] = ((red[e] + red[kCols + e]) + red[2 * kCols + e]) + red[3 * kCols + e];
        for (int e = tid; e < 192; e += kThreads) {
            float sum = 0.f;
#pragma unroll 4
            for (int w = 0; w < kThreads / 32; ++w) sum += lnp[w * 192 + e];
            part[2 * kF * kD + kF + e] = sum;
        }
    }
    if (!ok && tid == 0) {
        if (atomicCAS(&g.st->code, 0, (int)NNQS_E_TIMEOUT) == 0) g.st->index = -14;
        if (!w_landed) tc::mbar_wait(bW, 0);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(fb::kTmemCols)
                     : "memory");
    }
}

// sum over `grid` CTA partials, in CTA order, added into the gradients
__global__ void k_bwd_ffn_reduce(const float *__restrict__ part, int grid, float *dw1, float *dw2, float *db1,
                                 float *dg2, float *db2, float *dbo) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= kBwdFfnPart) return;
    float s = 0.f;
#pragma unroll 8
    for (int c = 0; c < grid; ++c) s += part[(int64_t)c * kBwdFfnPart + e];
    constexpr int a = 256 * 64, b = 2 * a, c1 = b + 256, c2 = c1 + 64, c3 = c2 + 64;
    float *dst = e < a ? dw1 + e : e < b ? dw2 + (e - a) : e < c1 ? db1 + (e - b) : e < c2 ? dg2 + (e - c1)
                 : e < c3 ? db2 + (e - c2) : dbo + (e - c3);
    *dst += s;
}

// ---------------------------------------------------------------------------
// Attention half of a layer (k_bwd_attn), per tile of floor(128 / T) whole
// samples (a sample's tokens never leave its tile, so the causal attention
// and its reverse mode need no other tile):
//   a = LN1(hin), q | k | v = a Wqkv^T + bqkv    (recomputed; split BF16 when the forward was)
//   do = dhmid Wo                                 (tensor cores)
//   per head: o, log-sum-exp recomputed; D = do . o; P = softmax;
//     dq = scale sum_j P (do . v_j - D) k_j, dk, dv over the later queries  (CUDA cores, FP32)
//   da = dqkv Wqkv, dh_in = dhmid + LN1'(da)     (written over dhmid)
//   dWqkv += dqkv^T a, dWo += dhmid^T o, dbqkv, dgamma1 / dbeta1, sum dh_in
// The heads are walked in two groups of 32 columns of q | k | v | do, whose
// FP32 values go through shared memory for the other rows of the sample; the
// causal loops run token-major (one thread per (token, sample, head)), the
// rest row-major (one thread per (row, head), as TMEM lanes are rows).
//
// Shared memory (1024-aligned base):
//   [0, 32K)       a hi / lo                 [128][64] BF16
//   [32K, 48K)     dhmid                     [128][64] BF16
//   [48K, 64K)     o                         [128][64] BF16 (right after dhmid:
//                                            the second 64-row block of the dWo product's A)
//   [64K, 112K)    dq | dk | dv              three [128][64] panels
//   [112K, 186K)   the group's q | k | v | do, log-sum-exp, D per (row, head),
//                                            FP32 (the qkv image's low part at the start of a tile)
//   [186K, 210K)   qkv image hi              [192][64]
//   [210K, 218K)   out-projection image hi   [64][64]
//   [218K, 224K)   row-sum exchange; the column-sum combine
// TMEM: dWqkv [0, 128) (rows 0..127, then rows 64..191), dWo [128, 192)
// (lanes 0..63), q | k | v [192, 384), do [384, 448), da [448, 512).
namespace fa {
constexpr int kThreads = 512, kRows = 128, kD = 64, kQKV = 192;
constexpr int kOffA = 0, kOffA2 = 16384, kOffDH = 32768, kOffO = 49152, kOffDQ = 65536;
// scratch: per row four head slots of 36 floats (q | k | v | do of head
// dimension 8, then log-sum-exp and D; two slots of 68 for dimension 16) and
// 4 floats of padding, so that the 16-byte pieces the token-major loops read
// (6 samples x 4 heads of one key) fall in different bank groups
constexpr int kOffS = 114688, kSS = 148;
constexpr int kOffWQ = 190464, kOffWO = 215040, kOffRed = 223232;
constexpr int kOffBar = kOffRed + 6144;
constexpr int kSmem = kOffBar + 64 + 1024;  // 230,464 bytes
constexpr uint32_t kColWQ = 0, kColWO = 128, kColQKV = 192, kColDO = 384, kColDA = 448, kTmemCols = 512;
constexpr int kCols = 384;  // column sums per CTA: dbqkv 192 | dgamma1 64 | dbeta1 64 | dsum 64
constexpr float kLog2e = 1.44269504088896340736f;
}  // namespace fa

// DH consecutive TMEM columns of this warp's 32 lanes
template <int DH>
__device__ __forceinline__ void fa_tmem_ld(uint32_t taddr, float (&v)[DH]) {
    if constexpr (DH == 16) {
        uint32_t r[16];
        tc::tmem_ld16(taddr, r);
#pragma unroll
        for (int c = 0; c < 16; ++c) v[c] = __uint_as_float(r[c]);
    } else {
        uint32_t r[8];
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                       "=r"(r[7])
                     : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int c = 0; c < 8; ++c) v[c] = __uint_as_float(r[c]);
    }
}

template <int DH>
__device__ __forceinline__ void fa_ld(const float *p, float (&v)[DH]) {
#pragma unroll
    for (int k = 0; k < DH / 4; ++k) {
        const float4 a = reinterpret_cast<const float4 *>(p)[k];
        v[4 * k] = a.x;
        v[4 * k + 1] = a.y;
        v[4 * k + 2] = a.z;
        v[4 * k + 3] = a.w;
    }
}
template <int DH>
__device__ __forceinline__ void fa_st(float *p, const float (&v)[DH]) {
#pragma unroll
    for (int k = 0; k < DH / 4; ++k)
        reinterpret_cast<float4 *>(p)[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
}
template <int DH>
__device__ __forceinline__ float fa_dot(const float (&a)[DH], const float (&b)[DH]) {
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < DH; ++c) s = fmaf(a[c], b[c], s);
    return s;
}

template <bool SPLIT, int DH>
__global__ void __launch_bounds__(fa::kThreads, 1) k_bwd_attn(const __grid_constant__ BwdAttnArgs g) {
    using namespace fa;
    constexpr int HPG = 32 / DH;  // heads per group of 32 columns
    constexpr int kSlot = 4 * DH + 4;  // q | k | v | do | log-sum-exp, D (base 2), -, -
    static_assert(HPG * DH == 32, "head dimension 8 or 16");
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = tc::smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *sb = smem_raw + (base - raw);
    float *red = reinterpret_cast<float *>(sb + kOffRed);
    float *sS = reinterpret_cast<float *>(sb + kOffS);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sb + kOffBar + 32);
    const uint32_t mb = base + kOffBar, bW = mb + 8, bL = mb + 16;
    const uint32_t uA = base + kOffA, uA2 = base + kOffA2, uDH = base + kOffDH, uO = base + kOffO;
    const uint32_t uDQ = base + kOffDQ, uS = base + kOffS, uWQ = base + kOffWQ, uWO = base + kOffWO;
    uint8_t *aHi = sb + kOffA, *aLo = SPLIT ? sb + kOffA2 : nullptr;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q4 = warp & 3, cq = warp >> 2, row = 32 * q4 + lane;
    const int r4 = tid >> 2, lq = tid & 3;
    const int T = g.T, rows_used = g.spt * T;
    const int64_t rows = g.n * T, n_tiles = (g.n + g.spt - 1) / g.spt;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(tslot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        tc::mbar_init(mb, 1);
        tc::mbar_init(bW, 1);
        tc::mbar_init(bL, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const uint32_t tl = tmem + (uint32_t(32 * q4) << 16);

    constexpr uint32_t kWQB = kQKV * 128, kWOB = kD * 128;  // 24 KB, 8 KB
    if (tid == 0) {
        tc::mbar_expect(bW, kWQB + kWOB);
        fb_bulk(sb + kOffWQ, g.tqkv, kWQB, bW);
        fb_bulk(sb + kOffWO, g.to, kWOB, bW);
    }
    bool ok = __syncthreads_and(tc::mbar_wait(bW, 0) ? 1 : 0) != 0;
    const bool w_landed = ok;
    uint32_t ph = 0, n_lo = 0, d_lo = 0;  // low-part copies issued / waited
    auto sync_async = [&]() {
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
    };
    auto wait_mma = [&]() {
        ok = __syncthreads_and(tc::mbar_wait(mb, ph) ? 1 : 0) != 0;
        ph ^= 1u;
        tc::fence_after_sync();
    };
    const float qscale = (1.0f / sqrtf(float(DH))) * kLog2e;  // scores in base-2 units
    const float scale = 1.0f / sqrtf(float(DH));

    float csq00 = 0.f, csq01 = 0.f, csq10 = 0.f, csq11 = 0.f;  // dbqkv column sums per group (see the flush)
    // column sums of the LN1 parameters' gradients and of dh_in over this
    // warp's rows, columns fb_col8(lane) and + 1
    float2 cs_g = make_float2(0.f, 0.f), cs_b = make_float2(0.f, 0.f), cs_o = make_float2(0.f, 0.f);
    bool first = true;
    for (int64_t tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
        const int64_t s0 = tile * g.spt;
        const bool valid = row < rows_used && s0 * T + row < rows;  // (TMEM-lane mapping)
        // rows of the four-lanes-per-row phases: tile row r4, global row g4
        const int64_t g4 = s0 * T + r4;
        const bool ok4 = r4 < rows_used && g4 < rows;
        if (tile + gridDim.x < n_tiles) {  // the next tile's rows into L2 meanwhile
            const int64_t r1 = (tile + gridDim.x) * g.spt * T, nr = rows - r1 < rows_used ? rows - r1 : rows_used;
            fb_prefetch_rows(g.hin, r1, nr, g.src, tid);
            if (tid == 0) fb_prefetch_l2(g.dh + r1 * kD, uint32_t(nr * kD * 4));
        }
        if (SPLIT && tid == 0) {  // the qkv image's low part into the scratch region
            tc::fence_async_smem();
            tc::mbar_expect(bL, kWQB);
            fb_bulk(sb + kOffS, static_cast<const __nv_bfloat16 *>(g.tqkv) + kQKV * kD, kWQB, bL);
        }
        if (SPLIT) ++n_lo;
        // ---- LN1 of the saved layer input -> a (A); dhmid -> DH (four lanes
        // per row; rows outside the tile's samples are zero)
        {
            float hv[16], dv[16];
            if (ok4) {
                fb_ld_row4(fb_row(g.hin, g4, g.src), lq, hv);
                fb_ld_row4_rw(g.dh + g4 * kD, lq, dv);
            } else {
#pragma unroll
                for (int c = 0; c < 16; ++c) hv[c] = dv[c] = 0.f;
            }
            float mu, rs;
            fb_ln_stats4(hv, mu, rs);
            float gv[16], bv[16], y[16];
            fb_ld_row4(g.ln1g, lq, gv);
            fb_ld_row4(g.ln1b, lq, bv);
#pragma unroll
            for (int c = 0; c < 16; ++c) y[c] = ok4 ? (hv[c] - mu) * rs * gv[c] + bv[c] : 0.f;
            fb_half_granules(aHi, aLo, r4, lq, y);
            fb_half_granules(sb + kOffDH, nullptr, r4, lq, dv);
        }
        if (SPLIT) {
            ok = __syncthreads_and(tc::mbar_wait(bL, d_lo & 1u) ? 1 : 0) != 0;
            if (!ok) break;
            ++d_lo;
        }
        sync_async();
        if (tid == 0) {
            fb_mma_kmajor(tmem + kColQKV, uA, uA2, uWQ, uS, kQKV, SPLIT, false);
            // do = dhmid Wo: B is the out-projection image read transposed
            const uint32_t id = idesc_t(kRows, kD, false, true);
            const uint64_t dA = tc::desc_sw128(uDH);
#pragma unroll
            for (int k = 0; k < 4; ++k)
                tc::mma_bf16(tmem + kColDO, dA + uint64_t(2 * k), desc_mn(uWO + 2048u * k, 8192u), id, k > 0 ? 1u : 0u);
            tc::mma_commit(mb);
        }
        wait_mma();
        if (!ok) break;
        // ---- the heads in two groups of 32 columns of q | k | v | do
        const int ipt = g.spt * HPG;  // work items (sample, head) per token position
#pragma unroll 1
        for (int gq = 0; gq < 2; ++gq) {
            // (1) thread (row, head cq of the group): q | k | v (+ bias) and do
            // from TMEM to the row's slot; rows outside the tile's samples get
            // zero o
            if (cq < HPG) {  // warp-uniform
                const int c0 = DH * (gq * HPG + cq);
                float *slot = sS + row * kSS + cq * kSlot;
                float q[DH], k[DH], v[DH], d[DH], b[DH];
                fa_tmem_ld<DH>(tl + kColQKV + c0, q);
                fa_tmem_ld<DH>(tl + kColQKV + 64 + c0, k);
                fa_tmem_ld<DH>(tl + kColQKV + 128 + c0, v);
                fa_tmem_ld<DH>(tl + kColDO + c0, d);
                fa_ld<DH>(g.bqkv + c0, b);
#pragma unroll
                for (int c = 0; c < DH; ++c) q[c] += b[c];
                fa_ld<DH>(g.bqkv + 64 + c0, b);
#pragma unroll
                for (int c = 0; c < DH; ++c) k[c] += b[c];
                fa_ld<DH>(g.bqkv + 128 + c0, b);
#pragma unroll
                for (int c = 0; c < DH; ++c) v[c] += b[c];
                fa_st<DH>(slot, q);
                fa_st<DH>(slot + DH, k);
                fa_st<DH>(slot + 2 * DH, v);
                fa_st<DH>(slot + 3 * DH, d);
                if (!valid) {
                    const float z[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
                    for (int e = 0; e < DH / 8; ++e) fb_granule(sb + kOffO, nullptr, row, c0 / 8 + e, z);
                }
            }
            __syncthreads();
            // (2) thread = (token position, sample, head), token-major: a warp
            // holds one or two token positions, so the lengths of its causal
            // loops (t + 1 keys for dq, T - t queries for dk and dv) nearly agree
            const int ti = tid / ipt, rem = tid - ti * ipt, sl = rem / HPG, hh = rem - sl * HPG;
            const bool act = ti < T && s0 + sl < g.n;
            const int r0 = sl * T, ri = r0 + ti;
            const int c0 = DH * (gq * HPG + hh);
            float *slot = act ? sS + ri * kSS + hh * kSlot : sS;
            // forward recomputation: o, log-sum-exp (base 2) and D = do . o
            if (act) {
                float qs[DH], o[DH];
                fa_ld<DH>(slot, qs);
#pragma unroll
                for (int c = 0; c < DH; ++c) {
                    qs[c] *= qscale;
                    o[c] = 0.f;
                }
                float m = -INFINITY, l = 0.f;
                for (int j = 0; j <= ti; ++j) {
                    const float *sj = sS + (r0 + j) * kSS + hh * kSlot;
                    float kj[DH], vj[DH];
                    fa_ld<DH>(sj + DH, kj);
                    fa_ld<DH>(sj + 2 * DH, vj);
                    const float sc = fa_dot<DH>(qs, kj);
                    const float mn = sc > m ? sc : m;
                    const float corr = fb_ex2(m - mn), p = fb_ex2(sc - mn);
                    l = l * corr + p;
#pragma unroll
                    for (int c = 0; c < DH; ++c) o[c] = o[c] * corr + p * vj[c];
                    m = mn;
                }
                const float inv = 1.0f / l;
#pragma unroll
                for (int c = 0; c < DH; ++c) o[c] *= inv;
                float dd[DH];
                fa_ld<DH>(slot + 3 * DH, dd);
                slot[4 * DH] = m + log2f(l);
                slot[4 * DH + 1] = fa_dot<DH>(dd, o);
#pragma unroll
                for (int e = 0; e < DH / 8; ++e) fb_granule(sb + kOffO, nullptr, ri, c0 / 8 + e, o + 8 * e);
            }
            __syncthreads();
            // reverse mode: dq over this query's keys, dk and dv over the
            // queries that see this row's key
            float dq[DH], dk[DH], dv[DH];
#pragma unroll
            for (int c = 0; c < DH; ++c) dq[c] = dk[c] = dv[c] = 0.f;
            if (act) {
                {
                    float qs[DH], dd[DH];
                    fa_ld<DH>(slot, qs);
                    fa_ld<DH>(slot + 3 * DH, dd);
#pragma unroll
                    for (int c = 0; c < DH; ++c) qs[c] *= qscale;
                    const float lse = slot[4 * DH], D = slot[4 * DH + 1];
                    for (int j = 0; j <= ti; ++j) {
                        const float *sj = sS + (r0 + j) * kSS + hh * kSlot;
                        float kj[DH], vj[DH];
                        fa_ld<DH>(sj + DH, kj);
                        fa_ld<DH>(sj + 2 * DH, vj);
                        const float p = fb_ex2(fa_dot<DH>(qs, kj) - lse);
                        const float ds = p * (fa_dot<DH>(dd, vj) - D);
#pragma unroll
                        for (int c = 0; c < DH; ++c) dq[c] = fmaf(ds, kj[c], dq[c]);
                    }
                }
                {
                    float ks[DH], vv[DH];
                    fa_ld<DH>(slot + DH, ks);
                    fa_ld<DH>(slot + 2 * DH, vv);
#pragma unroll
                    for (int c = 0; c < DH; ++c) ks[c] *= qscale;
                    for (int j = ti; j < T; ++j) {
                        const float *sj = sS + (r0 + j) * kSS + hh * kSlot;
                        float qj[DH], dj[DH];
                        fa_ld<DH>(sj, qj);
                        fa_ld<DH>(sj + 3 * DH, dj);
                        const float2 ld = *reinterpret_cast<const float2 *>(sj + 4 * DH);  // log-sum-exp, D
                        const float p = fb_ex2(fa_dot<DH>(qj, ks) - ld.x);
                        const float ds = p * (fa_dot<DH>(dj, vv) - ld.y);
#pragma unroll
                        for (int c = 0; c < DH; ++c) {
                            dk[c] = fmaf(ds, qj[c], dk[c]);
                            dv[c] = fmaf(p, dj[c], dv[c]);
                        }
                    }
                }
#pragma unroll
                for (int c = 0; c < DH; ++c) {
                    dq[c] *= scale;
                    dk[c] *= scale;
                }
            }
            __syncthreads();  // every loop has read q | k | v | do
            if (act) {
                fa_st<DH>(slot, dq);
                fa_st<DH>(slot + DH, dk);
                fa_st<DH>(slot + 2 * DH, dv);
            }
            __syncthreads();
            // (3) thread (row, head cq): dq | dk | dv to the BF16 tile (zero
            // outside the samples) and their column sums over the warp's rows
            if (cq < HPG) {
                const int cc = DH * (gq * HPG + cq);
                const float *slot3 = sS + row * kSS + cq * kSlot;
                float a[DH], b[DH], c3[DH];
                if (valid) {
                    fa_ld<DH>(slot3, a);
                    fa_ld<DH>(slot3 + DH, b);
                    fa_ld<DH>(slot3 + 2 * DH, c3);
                } else {
#pragma unroll
                    for (int c = 0; c < DH; ++c) a[c] = b[c] = c3[c] = 0.f;
                }
#pragma unroll
                for (int e = 0; e < DH / 8; ++e) {
                    fb_granule(sb + kOffDQ, nullptr, row, cc / 8 + e, a + 8 * e);
                    fb_granule(sb + kOffDQ + 16384, nullptr, row, cc / 8 + e, b + 8 * e);
                    fb_granule(sb + kOffDQ + 32768, nullptr, row, cc / 8 + e, c3 + 8 * e);
                }
                if constexpr (DH == 8) {
                    float t[32];
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        t[c] = a[c];
                        t[8 + c] = b[c];
                        t[16 + c] = c3[c];
                        t[24 + c] = 0.f;
                    }
                    const float c32 = fb_colsum<32>(t, lane);
                    if (gq == 0)
                        csq00 += c32;
                    else
                        csq10 += c32;
                } else {
                    float t[32], t2[16];
#pragma unroll
                    for (int c = 0; c < 16; ++c) {
                        t[c] = a[c];
                        t[16 + c] = b[c];
                        t2[c] = c3[c];
                    }
                    const float c32 = fb_colsum<32>(t, lane), c16 = fb_colsum<16>(t2, lane);
                    if (gq == 0) {
                        csq00 += c32;
                        csq01 += c16;
                    } else {
                        csq10 += c32;
                        csq11 += c16;
                    }
                }
            }
            __syncthreads();  // the slots are rewritten by the next group
        }
        sync_async();
        if (tid == 0) {
            // da = dqkv Wqkv: B is the qkv image read transposed (K = its 192 rows)
            const uint32_t id = idesc_t(kRows, kD, false, true);
#pragma unroll
            for (int kb = 0; kb < 3; ++kb) {
                const uint64_t dA = tc::desc_sw128(uDQ + 16384u * kb);
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    tc::mma_bf16(tmem + kColDA, dA + uint64_t(2 * k),
                                 desc_mn(uWQ + uint32_t(64 * kb + 16 * k) * 128u, 16384u), id, (kb | k) ? 1u : 0u);
            }
            // dWqkv rows 0..127 and 64..191 += dqkv^T a; dWo += dhmid^T o
            // (rows 64..127 of that product read the o panel after dhmid: unused)
            fb_mma_rows(tmem + kColWQ, uDQ, 16384u, uA, kD, !first);
            fb_mma_rows(tmem + kColWQ + 64, uDQ + 16384u, 16384u, uA, kD, !first);
            fb_mma_rows(tmem + kColWO, uDH, 16384u, uO, kD, !first);
            tc::mma_commit(mb);
        }
        wait_mma();
        if (!ok) break;
        // ---- LN1 backward: dh_in = dhmid + rs (da g - mean(da g) - xh mean(da g xh)),
        // four lanes per row; da leaves TMEM through the (now free) dq | dk | dv region
        {
            float *daS = reinterpret_cast<float *>(sb + kOffDQ);
            {
                uint32_t r16[16];
                tc::tmem_ld16(tl + kColDA + 16 * cq, r16);
                fb_da_store(daS, row, cq, r16);
            }
            __syncthreads();
            float hv[16], dv[16], gv[16], da[16], xh[16];
            if (ok4) {
                fb_ld_row4(fb_row(g.hin, g4, g.src), lq, hv);
                fb_ld_row4_rw(g.dh + g4 * kD, lq, dv);
                fb_da_load(daS, r4, lq, da);
            } else {
#pragma unroll
                for (int c = 0; c < 16; ++c) hv[c] = dv[c] = da[c] = 0.f;
            }
            fb_ld_row4(g.ln1g, lq, gv);
            float mu, rs;
            fb_ln_stats4(hv, mu, rs);
            float s1 = 0.f, s2 = 0.f;
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                xh[c] = ok4 ? (hv[c] - mu) * rs : 0.f;
                const float dx = da[c] * gv[c];
                s1 += dx;
                s2 += dx * xh[c];
            }
            const float m1 = fb_sum4(s1) * (1.0f / kD), m2 = fb_sum4(s2) * (1.0f / kD);
            float out[16], t[16];
#pragma unroll
            for (int c = 0; c < 16; ++c) out[c] = ok4 ? dv[c] + rs * (da[c] * gv[c] - m1 - xh[c] * m2) : 0.f;
            if (ok4) fb_st_row4(g.dh + g4 * kD, lq, out);
#pragma unroll
            for (int c = 0; c < 16; ++c) t[c] = da[c] * xh[c];
            const float2 sg = fb_colsum8(t, lane), sbt = fb_colsum8(da, lane), so = fb_colsum8(out, lane);
            cs_g.x += sg.x;
            cs_g.y += sg.y;
            cs_b.x += sbt.x;
            cs_b.y += sbt.y;
            cs_o.x += so.x;
            cs_o.y += so.y;
        }
        sync_async();  // (the next tile's copy into the scratch region follows these reads)
        first = false;
    }
    if (ok && !first) {
        float *part = g.part + (int64_t)blockIdx.x * kBwdAttnPart;
        {
            uint32_t r16[16];
            float v[16];
            // dWqkv rows 0..127 (lane = row)
            tc::tmem_ld16(tl + kColWQ + 16 * cq, r16);
#pragma unroll
            for (int c = 0; c < 16; ++c) v[c] = __uint_as_float(r16[c]);
            fb_st16(part + row * kD + 16 * cq, v);
            // rows 64..191: lanes 64..127 hold rows 128..191
            tc::tmem_ld16(tl + kColWQ + 64 + 16 * cq, r16);
#pragma unroll
            for (int c = 0; c < 16; ++c) v[c] = __uint_as_float(r16[c]);
            if (row >= 64) fb_st16(part + (64 + row) * kD + 16 * cq, v);
            // dWo (lanes 0..63)
            tc::tmem_ld16(tl + kColWO + 16 * cq, r16);
#pragma unroll
            for (int c = 0; c < 16; ++c) v[c] = __uint_as_float(r16[c]);
            if (row < 64) fb_st16(part + kQKV * kD + row * kD + 16 * cq, v);
        }
        float *cs = red + q4 * kCols;
        for (int e = tid; e < 4 * kCols; e += kThreads) red[e] = 0.f;
        __syncthreads();
        if (cq < HPG) {
#pragma unroll
            for (int gq = 0; gq < 2; ++gq) {
                const int c0 = DH * (gq * HPG + cq);
                const float a0 = gq == 0 ? csq00 : csq10, a1 = gq == 0 ? csq01 : csq11;
                if constexpr (DH == 8) {
                    if (lane < 24) cs[(lane >> 3) * 64 + c0 + (lane & 7)] = a0;
                } else {
                    cs[(lane >> 4) * 64 + c0 + (lane & 15)] = a0;
                    if ((lane & 1) == 0) cs[128 + c0 + (lane >> 1)] = a1;
                }
            }
        }
        // the LN1 and dh_in sums per warp ([16][192] over the free dq | dk | dv
        // region), added in warp order
        float *lnp = reinterpret_cast<float *>(sb + kOffDQ);
        const int c8 = fb_col8(lane);
        lnp[warp * 192 + c8] = cs_g.x;
        lnp[warp * 192 + c8 + 1] = cs_g.y;
        lnp[warp * 192 + 64 + c8] = cs_b.x;
        lnp[warp * 192 + 64 + c8 + 1] = cs_b.y;
        lnp[warp * 192 + 128 + c8] = cs_o.x;
        lnp[warp * 192 + 128 + c8 + 1] = cs_o.y;
        __syncthreads();
        for (int e = tid; e < kQKV; e += kThreads)
            part[kQKV * kD + kD * kD + e] = ((red[e] + red[kCols + e]) + red[2 * kCols + e]) + red[3 * kCols + e];
        for (int e = tid; e < 192; e += kThreads) {
            float sum = 0.f;
#pragma unroll 4
            for (int w = 0; w < kThreads / 32; ++w) sum += lnp[w * 192 + e];
            part[kQKV * kD + kD * kD + kQKV + e] = sum;
        }
    }
    if (!ok && tid == 0) {
        if (atomicCAS(&g.st->code, 0, (int)NNQS_E_TIMEOUT) == 0) g.st->index = -15;
        if (!w_landed) tc::mbar_wait(bW, 0);
        for (; d_lo < n_lo; ++d_lo) tc::mbar_wait(bL, d_lo & 1u);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(fa::kTmemCols)
                     : "memory");
    }
}

__global__ void k_bwd_attn_reduce(const float *__restrict__ part, int grid, float *dwqkv, float *dwo, float *dbqkv,
                                  float *dg1, float *db1, float *dsum) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= kBwdAttnPart) return;
    constexpr int a = 192 * 64, b = a + 64 * 64, c1 = b + 192, c2 = c1 + 64, c3 = c2 + 64;
    float *dst = e < a ? dwqkv + e : e < b ? dwo + (e - a) : e < c1 ? dbqkv + (e - b) : e < c2 ? dg1 + (e - c1)
                 : e < c3 ? db1 + (e - c2) : (dsum ? dsum + (e - c3) : nullptr);
    if (!dst) return;
    float s = 0.f;
#pragma unroll 8
    for (int c = 0; c < grid; ++c) s += part[(int64_t)c * kBwdAttnPart + e];
    *dst += s;
}

template <bool SPLIT, int DH>
nnqs_status launch_attn(const BwdAttnArgs &a, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        NNQS_CUDA_TRY(
            cudaFuncSetAttribute(k_bwd_attn<SPLIT, DH>, cudaFuncAttributeMaxDynamicSharedMemorySize, fa::kSmem));
        attr = true;
    }
    NNQS_LAUNCH("k_bwd_attn", s, (k_bwd_attn<SPLIT, DH><<<(unsigned)bwd_attn_grid(a.n, a.T), fa::kThreads, fa::kSmem, s>>>(a)));
    return NNQS_OK;
}

template <bool SPLIT>
nnqs_status launch_ffn(const BwdFfnArgs &a, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        NNQS_CUDA_TRY(cudaFuncSetAttribute(k_bwd_ffn<SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, fb::kSmem));
        attr = true;
    }
    NNQS_LAUNCH("k_bwd_ffn", s, (k_bwd_ffn<SPLIT><<<(unsigned)bwd_ffn_grid(a.rows), fb::kThreads, fb::kSmem, s>>>(a)));
    return NNQS_OK;
}

}  // namespace

bool bwd_ffn_supported(int d, int F) { return d == fb::kD && F == fb::kF; }

int bwd_ffn_grid(int64_t rows) {
    const int64_t tiles = (rows + fb::kRows - 1) / fb::kRows;
    return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, num_sms()));
}

nnqs_status bwd_ffn_launch(const BwdFfnArgs &a, bool split, cudaStream_t s) {
    if (a.rows <= 0) return NNQS_OK;
    auto al = [](const void *p) { return reinterpret_cast<uintptr_t>(p) % 16 == 0; };
    if (!al(a.hmid) || !al(a.dh) || !al(a.ln2g) || !al(a.ln2b) || !al(a.b1) || !al(a.t1) || !al(a.t2))
        return set_error(NNQS_E_INVAL, "fused FFN reverse mode: operands not 16-byte aligned");
    if (a.src.anc && (a.src.T < 1 || a.src.anc_stride < 1 || a.src.node_stride % 4 != 0))
        return set_error(NNQS_E_INVAL, "fused FFN reverse mode: bad tree row source");
    // method FLOPs: the recomputed FFN-in product and the four reverse products
    note_work("k_bwd_ffn", double(a.rows) * 2.0 * fb::kD * fb::kF * 5.0, double(a.rows) * fb::kD * 4.0 * 3.0);
    return split ? launch_ffn<true>(a, s) : launch_ffn<false>(a, s);
}

nnqs_status bwd_ffn_reduce(const float *part, int grid, float *dw1, float *dw2, float *db1, float *dg2, float *db2,
                           float *dbo, cudaStream_t s) {
    NNQS_LAUNCH("k_bwd_reduce", s, (k_bwd_ffn_reduce<<<(kBwdFfnPart + 255) / 256, 256, 0, s>>>(part, grid, dw1, dw2, db1, dg2, db2, dbo)));
    return NNQS_OK;
}

bool bwd_attn_supported(int d, int dh, int T) { return d == fa::kD && (dh == 8 || dh == 16) && T >= 1 && T <= 64; }

int bwd_attn_grid(int64_t n, int T) {
    const int64_t spt = 128 / std::max(T, 1), tiles = (n + spt - 1) / spt;
    return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, num_sms()));
}

nnqs_status bwd_attn_launch(const BwdAttnArgs &a, bool split, int dh, cudaStream_t s) {
    if (a.n <= 0) return NNQS_OK;
    if (a.T < 1 || a.T > 64 || a.spt != 128 / a.T) return set_error(NNQS_E_INVAL, "fused attention reverse mode: bad tile shape");
    auto al = [](const void *p) { return reinterpret_cast<uintptr_t>(p) % 16 == 0; };
    if (!al(a.hin) || !al(a.dh) || !al(a.ln1g) || !al(a.ln1b) || !al(a.bqkv) || !al(a.tqkv) || !al(a.to))
        return set_error(NNQS_E_INVAL, "fused attention reverse mode: operands not 16-byte aligned");
    if (a.src.anc && (a.src.T != a.T || a.src.anc_stride < 1 || a.src.node_stride % 4 != 0))
        return set_error(NNQS_E_INVAL, "fused attention reverse mode: bad tree row source");
    // method FLOPs: the recomputed qkv product, do, da and the two weight products
    const double rows = double(a.n) * a.T;
    note_work("k_bwd_attn", rows * 2.0 * fa::kD * (3.0 * fa::kQKV + 2.0 * fa::kD), rows * fa::kD * 4.0 * 3.0);
    if (split) return dh == 8 ? launch_attn<true, 8>(a, s) : launch_attn<true, 16>(a, s);
    return dh == 8 ? launch_attn<false, 8>(a, s) : launch_attn<false, 16>(a, s);
}

nnqs_status bwd_attn_reduce(const float *part, int grid, float *dwqkv, float *dwo, float *dbqkv, float *dg1,
                            float *db1, float *dsum, cudaStream_t s) {
    NNQS_LAUNCH("k_bwd_reduce", s, (k_bwd_attn_reduce<<<(kBwdAttnPart + 255) / 256, 256, 0, s>>>(part, grid, dwqkv, dwo, dbqkv, dg1, db1, dsum)));
    return NNQS_OK;
}

}  // namespace nnqs
