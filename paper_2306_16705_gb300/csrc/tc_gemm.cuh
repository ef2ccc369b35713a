// tcgen05 (5th-generation tensor core) GEMM for the ansatz's linear layers:
//   Y[M][N] (epilogue) = X[M][K] W[N][K]^T,  X FP32 -> BF16, W BF16, FP32 accumulate in TMEM.
//
// One CTA of 128 threads computes a 128 x Nt tile (Nt <= 128, a multiple of
// 16; four CTAs share an SM).  K is walked in chunks of 64 BF16 (one 128-byte row per operand row):
// all threads convert/stage the chunk into shared memory in the K-major
// 128-byte-swizzle layout (8-row x 128 B atoms, 16-byte granules XOR-ed by the
// row index within the atom), one thread issues four M=128, K=16 MMAs and
// commits them to an mbarrier, and every thread waits on it before the
// buffer is refilled.  The epilogue reads the accumulator with tcgen05.ld
// (warp w owns TMEM lanes 32w..32w+31 = tile rows) and applies bias /
// activation / residual in FP32.
//
// Every wait is bounded: on a timeout the kernel records NNQS_E_TIMEOUT,
// skips the epilogue and still releases its TMEM.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace nnqs {
namespace tc {

constexpr int kThreads = 128;
constexpr int kTileM = 128;
constexpr int kChunkK = 64;                      // BF16 per 128-byte row
constexpr int kABytes = kTileM * kChunkK * 2;    // 16 KB
constexpr int kMaxN = 128;                       // N per CTA: TMEM 128 columns, 4 CTAs per SM
constexpr int kBBytes = kMaxN * kChunkK * 2;     // 16 KB
// dynamic shared memory: 1024 bytes of alignment slack, the operand buffers
// (kOps), then at kOps + 0 the MMA mbarrier, + 16 the TMEM address, + 24 the
// four epilogue residual-slot mbarriers, + 64 the 512-byte column-sum scratch
constexpr int kSmemBytes = kABytes + kBBytes + 1024 + 64 + 512;
// split operands: high and low BF16 parts of A and B
constexpr int kSmemBytesSplit = 2 * (kABytes + kBBytes) + 1024 + 64 + 512;

// EPI_DGELU / EPI_DRELU (input gradients): Y = acc * act'(Z) with the
// pre-activation Z passed as `resid`
enum { EPI_STORE = 0, EPI_GELU = 1, EPI_RELU = 2, EPI_RESID = 3, EPI_DGELU = 4, EPI_DRELU = 5 };
constexpr int kNumEpi = 6;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), descriptor version 1
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= uint64_t((saddr >> 4) & 0x3FFFu);
    d |= uint64_t(1) << 16;                 // leading byte offset (unused for swizzled K-major)
    d |= uint64_t((1024u >> 4) & 0x3FFFu) << 32;
    d |= uint64_t(1) << 46;
    d |= uint64_t(2) << 61;                 // 128-byte swizzle
    return d;
}

// instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major
__host__ __device__ __forceinline__ uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

// instruction descriptor, kind::f8f6f4: D = F32, A = B = E4M3 (format 0), both K-major
__host__ __device__ __forceinline__ uint32_t idesc_e4m3(int M, int N) {
    return (1u << 4) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

// one M x N x 32 step with E4M3 operands (32 bytes of a 128-byte K row)
__device__ __forceinline__ void mma_e4m3(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}

// bounded wait on an mbarrier phase; false on timeout (~2 s at 2 GHz)
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase) {
    const long long t0 = clock64();
    for (uint32_t it = 0; it < (1u << 26); ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(mbar), "r"(phase)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > 4000000000ll) return false;
    }
    return false;
}

__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// GELU(x) = x Phi(x) with erf of Abramowitz and Stegun (1964), eq. 7.1.26:
// erf(z) = 1 - t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) e^{-z^2}, t = 1 / (1 + p z)
// for z >= 0, odd in z, absolute error at most 1.5e-7 (far below the 2^-16
// relative resolution of the split-BF16 operands the values feed); branch-free,
// two special-function instructions.  The fused forward and reverse mode use
// the same form and operation order.
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// 1 - erf(|x| / sqrt 2), from the polynomial, and e = exp(-x^2 / 2)
__device__ __forceinline__ float erfc_as(float x, float &e) {
    const float z = fabsf(x) * 0.70710678118654752f;
    const float t = __fdividef(1.0f, fmaf(0.3275911f, z, 1.0f));
    const float poly =
        t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.061405429f, -1.453152027f), 1.421413741f), -0.284496736f), 0.254829592f);
    e = ex2_approx(-(z * z) * 1.44269504088896340736f);
    return poly * e;
}
__device__ __forceinline__ float gelu_f(float x) {
    float e;
    const float erf_abs = 1.0f - erfc_as(x, e);
    return 0.5f * x * (1.0f + copysignf(erf_abs, x));
}
// d gelu / dx = Phi(x) + x phi(x)
__device__ __forceinline__ float gelu_grad_f(float x) {
    float e;
    const float phi_cdf = 0.5f * (1.0f + copysignf(1.0f - erfc_as(x, e), x));
    return phi_cdf + x * e * 0.39894228040143267794f;
}

__device__ __forceinline__ uint4 pack8(const float (&v)[8]) {
    uint32_t p[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        __nv_bfloat162 b2 = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
        p[e] = *reinterpret_cast<uint32_t *>(&b2);
    }
    return make_uint4(p[0], p[1], p[2], p[3]);
}

// 16 FP32 values -> 16 E4M3 bytes in element order (round to nearest,
// saturating to +-448)
__device__ __forceinline__ uint4 pack16_e4m3(const float (&v)[16]) {
    uint32_t p[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint32_t a = __nv_cvt_float2_to_fp8x2(make_float2(v[4 * q], v[4 * q + 1]), __NV_SATFINITE, __NV_E4M3);
        const uint32_t b = __nv_cvt_float2_to_fp8x2(make_float2(v[4 * q + 2], v[4 * q + 3]), __NV_SATFINITE, __NV_E4M3);
        p[q] = (a & 0xFFFFu) | (b << 16);
    }
    return make_uint4(p[0], p[1], p[2], p[3]);
}

struct Args {
    const float *X;        // [M][ldx], K valid columns
    int64_t ldx;
    const __nv_bfloat16 *Wt;  // [Npad][Kpad] BF16, zero padded
    const __nv_bfloat16 *Wt2; // SPLIT: low parts W - bf16(W), same layout
    int64_t Kpad;
    const float *bias;     // [N] or null
    const float *resid;    // EPI_RESID: [M][ldy] added; EPI_DGELU/DRELU: pre-activation [M][ldy]
    float *Y;              // [M][ldy]
    float *Y2;             // activation output for GELU/RELU
    int64_t ldy;
    int64_t M, N, K;
    int Nt;                // N per CTA (multiple of 16, <= 256)
    int vec_x;             // X rows (TRANS: X and Xb rows) 16-byte aligned: float4 loads allowed
    const float *Xb;       // TRANS: second operand [K][ldb]
    int64_t ldb;
    int64_t kchunk;        // TRANS: reduction rows per blockIdx.z (multiple of 64)
    int tmem_cols;         // power of two >= max(32, Nt)
    DevStatus *st;
    // TMA epilogue (use_tma): 3-D FP32 tensor maps {N, M, splits} of Y, Y2 and
    // the residual / pre-activation, 128 x 32 boxes with the 128-byte swizzle
    int use_tma;
    CUtensorMap tmY, tmY2, tmR;
    // TMA epilogue, optional: column sums of this CTA's 128 output rows,
    // colpart[row tile][N] (for the bias gradient of the layer whose input
    // gradient Y is)
    float *colpart;
    // warp-specialised kernel (k_tc_gemm_ws): N tiles, epilogue bytes per
    // warpgroup, and X as a 3-D FP32 tensor map {K, M, 1} with 32 x 128 boxes
    // and the 128-byte swizzle
    int p_ntiles;
    int p_wg_epi;
    CUtensorMap tmX;
    // FP8 (E4M3) forward: W8 [Npad][Kpad8] bytes, each output row n scaled by
    // a power of two s_n, and wsinv[n] = 1 / s_n applied to the accumulator
    const uint8_t *W8;
    int64_t Kpad8;
    const float *wsinv;
};

// TMA: one 32-column x 128-row FP32 box between shared memory (1024-byte
// aligned, 128-byte swizzled) and global memory
__device__ __forceinline__ void tma_store_box(const CUtensorMap *tm, uint32_t smem, int x, int y, int z) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
                     reinterpret_cast<uint64_t>(tm)),
                 "r"(smem), "r"(x), "r"(y), "r"(z)
                 : "memory");
}
__device__ __forceinline__ void tma_load_box(uint32_t smem, const CUtensorMap *tm, int x, int y, int z, uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z), "r"(mbar)
        : "memory");
}
__device__ __forceinline__ void mbar_expect(uint32_t mbar, uint32_t bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(mbar),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// at most N of this thread's latest bulk store groups still reading shared memory
template <int N>
__device__ __forceinline__ void bulk_wait_read_n() {
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}

// TRANS = false: Y = X W^T (X FP32 [M][ldx], W BF16 [N][Kpad]).
// TRANS = true : Y = A^T B over a long K (weight gradients): A(m,k) =
//   X[k*ldx + m], B(n,k) = Xb[k*ldb + n], both FP32 and staged transposed;
//   blockIdx.z takes rows [z*kchunk, (z+1)*kchunk) of the reduction.
// SPLIT (TRANS = false only): X = Xh + Xl and W = Wh + Wl with BF16 parts
//   (Xh = bf16(X), Xl = bf16(X - Xh)) and Y = Xh Wh + Xh Wl + Xl Wh: three
//   MMAs per K step, operands good to about 16 bits instead of 8, the same
//   global traffic.  Three CTAs per SM (64 KB of operand buffers each).
// FP8 (TRANS = false, SPLIT = false only): X and W in E4M3, K chunks of 128
//   (one 128-byte row per operand row), kind::f8f6f4 MMAs of K = 32; W rows
//   carry a power-of-two scale that the epilogue divides out.
template <int EPI, bool TRANS, bool SPLIT = false, bool FP8 = false>
__global__ void __launch_bounds__(kThreads, SPLIT ? 3 : 4) k_tc_gemm(const __grid_constant__ Args g) {
    static_assert(!(TRANS && SPLIT), "split operands are for the forward layers only");
    static_assert(!(FP8 && (TRANS || SPLIT)), "E4M3 operands are for the plain forward layers only");
    constexpr int kCK = FP8 ? 128 : kChunkK;  // K elements per chunk: one 128-byte row
    constexpr int kOps = (SPLIT ? 2 : 1) * (kABytes + kBBytes);
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;  // swizzle atoms want 1024-byte alignment
    uint8_t *sbase = smem_raw + (base - raw);
    uint8_t *sA = sbase;
    uint8_t *sB = sbase + kABytes;
    uint8_t *sA2 = sbase + kABytes + kBBytes;  // SPLIT: low parts
    uint8_t *sB2 = sA2 + kABytes;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sbase + kOps);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sbase + kOps + 16);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // N tiles vary fastest so the CTAs sharing an A tile run together (A is
    // then read from HBM once and from L2 after)
    const int64_t m0 = blockIdx.y * (int64_t)kTileM;
    const int64_t n0 = blockIdx.x * (int64_t)g.Nt;
    const int Nt = g.Nt;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(g.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(smem_u32(mbar), 1);
        for (int k = 0; k < 4; ++k) mbar_init(smem_u32(sbase + kOps + 24 + 8 * k), 1);  // epilogue residual slots
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    const uint32_t idesc = FP8 ? idesc_e4m3(kTileM, Nt) : idesc_bf16(kTileM, Nt);
    const uint32_t mb = smem_u32(mbar);

    bool ok = true;
    uint32_t phase = 0;
    const int64_t kbeg = TRANS ? blockIdx.z * g.kchunk : 0;
    const int64_t kend = TRANS ? min(g.K, kbeg + g.kchunk) : g.K;
    const int nchunks = (int)((kend - kbeg + kCK - 1) / kCK);
    // operand granules of one K chunk, held in registers as packed BF16:
    // 8 A granules and up to 8 B granules per thread
    uint4 ra[8], rb[8], ra2[8], rb2[8];  // ra2/rb2: low parts (SPLIT)
    // TRANS with 16-byte rows (vec_x): a thread loads float4s of 4 consecutive
    // m (or n) for the 8 k of one granule and transposes them in registers
    // into 4 granules; granule i = 4q + j is row 4 (tid & 31) + j, k-granule
    // (tid >> 5) + 4q of A, and row 4 (p % (Nt/4)) + j, k-granule p / (Nt/4)
    // with p = tid + 128 q of B
    const bool tvec = TRANS && g.vec_x;
    auto load4x8 = [&](const float *src, int64_t ld, int64_t lim, int64_t c0i, int64_t k0g, float (&v)[4][8]) {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int64_t k = k0g + e;
            float4 f = make_float4(0.f, 0.f, 0.f, 0.f);
            if (k < kend) {
                if (c0i + 3 < lim) {
                    f = __ldg(reinterpret_cast<const float4 *>(src + k * ld + c0i));
                } else {
                    if (c0i < lim) f.x = __ldg(src + k * ld + c0i);
                    if (c0i + 1 < lim) f.y = __ldg(src + k * ld + c0i + 1);
                    if (c0i + 2 < lim) f.z = __ldg(src + k * ld + c0i + 2);
                }
            }
            v[0][e] = f.x;
            v[1][e] = f.y;
            v[2][e] = f.z;
            v[3][e] = f.w;
        }
    };
    auto load_chunk = [&](int64_t k0) {
        if constexpr (FP8) {
            // A: 8 consecutive threads cover one row's 128 values, 16 each
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int it = tid + i * kThreads;
                const int r = it >> 3, c = it & 7;
                const int64_t m = m0 + r;
                const int64_t k = k0 + c * 16;
                float v[16];
                if (m < g.M && g.vec_x && k + 16 <= g.K) {
                    const float4 *src = reinterpret_cast<const float4 *>(g.X + m * g.ldx + k);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float4 f = __ldg(src + q);
                        v[4 * q] = f.x; v[4 * q + 1] = f.y; v[4 * q + 2] = f.z; v[4 * q + 3] = f.w;
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < 16; ++e) v[e] = (m < g.M && k + e < g.K) ? g.X[m * g.ldx + k + e] : 0.f;
                }
                ra[i] = pack16_e4m3(v);
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                if (i * kThreads >= Nt * 8) break;
                const int it = tid + i * kThreads;
                const int r = it >> 3, c = it & 7;
                const int64_t n = n0 + r;
                rb[i] = n < g.N ? __ldg(reinterpret_cast<const uint4 *>(g.W8 + n * g.Kpad8 + k0 + c * 16))
                                : make_uint4(0u, 0u, 0u, 0u);
            }
            return;
        }
        if (tvec) {
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                float v[4][8];
                load4x8(g.X, g.ldx, g.M, m0 + 4 * (tid & 31), k0 + 8 * ((tid >> 5) + 4 * q), v);
#pragma unroll
                for (int j = 0; j < 4; ++j) ra[4 * q + j] = pack8(v[j]);
            }
            const int nq = Nt / 4;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int pidx = tid + kThreads * q;
                if (pidx >= 8 * nq) break;
                float v[4][8];
                load4x8(g.Xb, g.ldb, g.N, n0 + 4 * (pidx % nq), k0 + 8 * (pidx / nq), v);
#pragma unroll
                for (int j = 0; j < 4; ++j) rb[4 * q + j] = pack8(v[j]);
            }
            return;
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            float v[8];
            if (TRANS) {
                // A(m, k) = X[k][m]: a warp's 32 threads read 32 consecutive m of one row
                const int it = tid + i * kThreads;
                const int r = it & (kTileM - 1), c = it >> 7;
                const int64_t m = m0 + r;
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int64_t k = k0 + c * 8 + e;
                    v[e] = (m < g.M && k < kend) ? __ldg(g.X + k * g.ldx + m) : 0.f;
                }
            } else {
                // A rows: 8 consecutive threads cover one row's 64 FP32 values
                const int it = tid + i * kThreads;
                const int r = it >> 3, c = it & 7;
                const int64_t m = m0 + r;
                const int64_t k = k0 + c * 8;
                if (m < g.M && g.vec_x && k + 8 <= g.K) {
                    const float4 *src = reinterpret_cast<const float4 *>(g.X + m * g.ldx + k);
                    const float4 a = __ldg(src), b = __ldg(src + 1);
                    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
                    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
                } else {
#pragma unroll
                    for (int e = 0; e < 8; ++e) v[e] = (m < g.M && k + e < g.K) ? g.X[m * g.ldx + k + e] : 0.f;
                }
            }
            ra[i] = pack8(v);
            if (SPLIT) {
                float lo[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) lo[e] = v[e] - __bfloat162float(__float2bfloat16_rn(v[e]));
                ra2[i] = pack8(lo);
            }
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (i * kThreads >= Nt * 8) break;  // Nt/16 granule rounds
            const int it = tid + i * kThreads;
            if (TRANS) {
                const int r = it % Nt, c = it / Nt;
                const int64_t n = n0 + r;
                float v[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int64_t k = k0 + c * 8 + e;
                    v[e] = (n < g.N && k < kend) ? __ldg(g.Xb + k * g.ldb + n) : 0.f;
                }
                rb[i] = pack8(v);
            } else {
                const int r = it >> 3, c = it & 7;
                const int64_t n = n0 + r;
                rb[i] = n < g.N ? __ldg(reinterpret_cast<const uint4 *>(g.Wt + n * g.Kpad + k0 + c * 8))
                                : make_uint4(0u, 0u, 0u, 0u);
                if (SPLIT)
                    rb2[i] = n < g.N ? __ldg(reinterpret_cast<const uint4 *>(g.Wt2 + n * g.Kpad + k0 + c * 8))
                                     : make_uint4(0u, 0u, 0u, 0u);
            }
        }
    };
    auto store_chunk = [&]() {
        if (tvec) {
            const int nq = Nt / 4;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int r = 4 * (tid & 31) + (i & 3), c = (tid >> 5) + 4 * (i >> 2);
                *reinterpret_cast<uint4 *>(sA + r * 128 + ((c ^ (r & 7)) << 4)) = ra[i];
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int pidx = tid + kThreads * (i >> 2);
                if (pidx >= 8 * nq) break;
                const int r = 4 * (pidx % nq) + (i & 3), c = pidx / nq;
                *reinterpret_cast<uint4 *>(sB + r * 128 + ((c ^ (r & 7)) << 4)) = rb[i];
            }
            return;
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int it = tid + i * kThreads;
            const int r = TRANS ? (it & (kTileM - 1)) : (it >> 3), c = TRANS ? (it >> 7) : (it & 7);
            *reinterpret_cast<uint4 *>(sA + r * 128 + ((c ^ (r & 7)) << 4)) = ra[i];
            if (SPLIT) *reinterpret_cast<uint4 *>(sA2 + r * 128 + ((c ^ (r & 7)) << 4)) = ra2[i];
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (i * kThreads >= Nt * 8) break;
            const int it = tid + i * kThreads;
            const int r = TRANS ? (it % Nt) : (it >> 3), c = TRANS ? (it / Nt) : (it & 7);
            *reinterpret_cast<uint4 *>(sB + r * 128 + ((c ^ (r & 7)) << 4)) = rb[i];
            if (SPLIT) *reinterpret_cast<uint4 *>(sB2 + r * 128 + ((c ^ (r & 7)) << 4)) = rb2[i];
        }
    };
    if (nchunks > 0) load_chunk(kbeg);
    for (int kc = 0; kc < nchunks && ok; ++kc) {
        store_chunk();
        fence_async_smem();
        fence_before_sync();
        __syncthreads();
        fence_after_sync();
        if (tid == 0) {
            const uint64_t da = desc_sw128(smem_u32(sA)), db = desc_sw128(smem_u32(sB));
            const uint64_t da2 = desc_sw128(smem_u32(sA2)), db2 = desc_sw128(smem_u32(sB2));
#pragma unroll
            for (int k = 0; k < kChunkK / 16; ++k) {  // +32 bytes per K=16 step inside the swizzle atom
                if (FP8) {
                    mma_e4m3(tmem, da + uint64_t(2 * k), db + uint64_t(2 * k), idesc, (kc > 0 || k > 0) ? 1u : 0u);
                } else if (SPLIT) {  // small terms first
                    mma_bf16(tmem, da2 + uint64_t(2 * k), db + uint64_t(2 * k), idesc, (kc > 0 || k > 0) ? 1u : 0u);
                    mma_bf16(tmem, da + uint64_t(2 * k), db2 + uint64_t(2 * k), idesc, 1u);
                    mma_bf16(tmem, da + uint64_t(2 * k), db + uint64_t(2 * k), idesc, 1u);
                } else {
                    mma_bf16(tmem, da + uint64_t(2 * k), db + uint64_t(2 * k), idesc, (kc > 0 || k > 0) ? 1u : 0u);
                }
            }
            mma_commit(mb);
        }
        // the next chunk's loads are in flight while the MMAs run
        if (kc + 1 < nchunks) load_chunk(kbeg + int64_t(kc + 1) * kCK);
        // every thread saw the MMAs retire (or gave up) before the buffers are
        // reused; the flag is made CTA-uniform so no barrier below diverges
        ok = __syncthreads_and(mbar_wait(mb, phase) ? 1 : 0) != 0;
        phase ^= 1u;
    }
    fence_after_sync();
    if (!ok) {
        if (tid == 0) {
            if (atomicCAS(&g.st->code, 0, (int)NNQS_E_TIMEOUT) == 0) g.st->index = -10;
        }
    } else if (g.use_tma && Nt % 32 == 0) {  // whole boxes inside this CTA's columns
        // 32-column boxes: TMEM -> registers (thread = row) -> epilogue ->
        // shared memory in the TMA layout (row r at 128 r bytes, 16-byte chunk
        // q at q ^ (r & 7)) -> one bulk tensor store per box.  The boxes cycle
        // through the free operand buffers (two-output epilogues through pairs
        // (Y, activation)), so a box is computed while the stores of the
        // previous ones drain; a slot is rewritten once its store has read it.
        // Residual / pre-activation boxes are loaded by TMA into their slots
        // ahead of use (all of them at once when every box has its own slot).
        // Rows and columns outside the tensor are dropped by the store (zeros
        // on the load).
        constexpr bool kNeedR = EPI == EPI_RESID || EPI == EPI_DGELU || EPI == EPI_DRELU;
        constexpr bool kTwo = EPI == EPI_GELU || EPI == EPI_RELU;
        constexpr int kSlots = kOps / 16384;
        // boxes whose slots are in use at once (at most the 4 residual barriers)
        constexpr int kCyc = (kTwo ? kSlots / 2 : kSlots) < 4 ? (kTwo ? kSlots / 2 : kSlots) : 4;
        const int nbox = Nt / 32;
        const int row = warp * 32 + lane;
        const uint32_t lane_base = tmem + (uint32_t(warp * 32) << 16);
        const int zc = TRANS ? (int)blockIdx.z : 0;
        float *cpart = reinterpret_cast<float *>(sbase + kOps + 64);
        const uint32_t rb0 = smem_u32(sbase + kOps + 24);  // residual barrier of slot k at rb0 + 8 k
        auto ybox = [&](int c) { return sbase + (kTwo ? 2 * (c % kCyc) : c % kCyc) * 16384; };
        int r_issued = 0, r_done = 0;
        auto issue_r = [&](int c) {
            const uint32_t rb = rb0 + 8u * uint32_t(c % kCyc);
            mbar_expect(rb, 16384u);
            tma_load_box(smem_u32(ybox(c)), &g.tmR, (int)(n0 + 32 * c), (int)m0, zc, rb);
            r_issued = c + 1;
        };
        if (kNeedR && tid == 0)
            for (int c = 0; c < kCyc && c < nbox; ++c) issue_r(c);
        for (int c = 0; c < nbox && ok; ++c) {
            uint8_t *box = ybox(c), *box2 = box + 16384;
            if (!kNeedR && tid == 0 && c >= kCyc) bulk_wait_read_n<kCyc - 1>();  // box c - kCyc's store has read it
            bool good = true;
            if (kNeedR) good = mbar_wait(rb0 + 8u * uint32_t(c % kCyc), uint32_t((c / kCyc) & 1));
            ok = __syncthreads_and(good ? 1 : 0) != 0;
            if (!ok) break;
            if (kNeedR) r_done = c + 1;
            uint32_t r[32];
            tmem_ld16(lane_base + uint32_t(32 * c), *reinterpret_cast<uint32_t(*)[16]>(r));
            tmem_ld16(lane_base + uint32_t(32 * c + 16), *reinterpret_cast<uint32_t(*)[16]>(r + 16));
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int off = row * 128 + ((q ^ (row & 7)) << 4);
                float v[4], y[4], y2[4];
                float4 rv = make_float4(0.f, 0.f, 0.f, 0.f);
                if (kNeedR) rv = *reinterpret_cast<const float4 *>(box + off);
                const float rr[4] = {rv.x, rv.y, rv.z, rv.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int64_t n = n0 + 32 * c + 4 * q + e;
                    const float bias_v = (g.bias && n < g.N) ? __ldg(g.bias + n) : 0.f;
                    float a = __uint_as_float(r[4 * q + e]);
                    if (FP8) a *= n < g.N ? __ldg(g.wsinv + n) : 0.f;
                    v[e] = a + bias_v;
                    if (EPI == EPI_STORE) {
                        y[e] = v[e];
                    } else if (EPI == EPI_GELU) {
                        y[e] = v[e];
                        y2[e] = gelu_f(v[e]);
                    } else if (EPI == EPI_RELU) {
                        y[e] = v[e];
                        y2[e] = v[e] > 0.f ? v[e] : 0.f;
                    } else if (EPI == EPI_RESID) {
                        y[e] = rr[e] + v[e];
                    } else if (EPI == EPI_DGELU) {
                        y[e] = v[e] * gelu_grad_f(rr[e]);
                    } else {
                        y[e] = rr[e] > 0.f ? v[e] : 0.f;
                    }
                }
                *reinterpret_cast<float4 *>(box + off) = make_float4(y[0], y[1], y[2], y[3]);
                if (kTwo) *reinterpret_cast<float4 *>(box2 + off) = make_float4(y2[0], y2[1], y2[2], y2[3]);
            }
            fence_async_smem();
            __syncthreads();
            if (!kTwo && g.colpart) {
                // column tid & 31 over rows 32 (tid >> 5) .. + 31 of the box, in
                // order (rows past M are left out); the four row groups are
                // added in order below
                const int rmax = (int)min((int64_t)kTileM, g.M - m0);
                const int cl = tid & 31, q = cl >> 2, e = cl & 3, rg = tid >> 5;
                float cs = 0.f;
                for (int rr = 32 * rg; rr < min(32 * rg + 32, rmax); ++rr)
                    cs += *reinterpret_cast<const float *>(box + rr * 128 + ((q ^ (rr & 7)) << 4) + 4 * e);
                cpart[rg * 32 + cl] = cs;
            }
            if (tid == 0) {
                tma_store_box(&g.tmY, smem_u32(box), (int)(n0 + 32 * c), (int)m0, zc);
                if (kTwo) tma_store_box(&g.tmY2, smem_u32(box2), (int)(n0 + 32 * c), (int)m0, zc);
                bulk_commit();
            }
            if (!kTwo && g.colpart) {
                __syncthreads();  // also: no thread reads the box any more
                if (tid < 32 && n0 + 32 * c + tid < g.N)
                    g.colpart[blockIdx.y * g.N + n0 + 32 * c + tid] =
                        ((cpart[tid] + cpart[32 + tid]) + cpart[64 + tid]) + cpart[96 + tid];
            }
            if (kNeedR && tid == 0 && c + kCyc < nbox) {
                // the slot takes box c + kCyc's residual once every thread is
                // done with it (the barrier above, or the one before the
                // store) and the store has read it
                bulk_wait_read();
                issue_r(c + kCyc);
            }
        }
        if (tid == 0) {
            if (!ok) {
                if (atomicCAS(&g.st->code, 0, (int)NNQS_E_TIMEOUT) == 0) g.st->index = -12;
                // residual loads still in flight land (bounded)
                for (int c = r_done; c < r_issued; ++c)
                    mbar_wait(rb0 + 8u * uint32_t(c % kCyc), uint32_t((c / kCyc) & 1));
            }
            asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");  // stores complete
        }
    } else {
        // 64-column slabs: TMEM -> shared (thread = row) -> global (a warp
        // writes consecutive floats of a row), epilogue applied on the way
        // out.  The operand buffers (32 KB) are free once the MMAs retired; the
        // slab [128][64] is XOR-swizzled by the row so both phases are free of
        // bank conflicts.  Residual and bias values of a batch are loaded before
        // any of its stores: Y may alias the residual, and batching keeps the
        // loads in flight together instead of one dependent round trip each.
        float *slab = reinterpret_cast<float *>(sbase);
        const int row = warp * 32 + lane;
        const uint32_t lane_base = tmem + (uint32_t(warp * 32) << 16);
        const int64_t zoff = TRANS ? int64_t(blockIdx.z) * g.M * g.ldy : 0;
        for (int c0 = 0; c0 < Nt; c0 += 64) {
            const int sw = min(64, Nt - c0);  // slab width, a multiple of 16
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (16 * q >= sw) break;
                uint32_t r[16];
                tmem_ld16(lane_base + uint32_t(c0 + 16 * q), r);
#pragma unroll
                for (int j = 0; j < 16; ++j) slab[row * 64 + ((16 * q + j) ^ (row & 31))] = __uint_as_float(r[j]);
            }
            __syncthreads();
            // thread -> one column (tid % sw) of the slab and the rows r0,
            // r0 + rp, ... with r0 = tid / sw and rp = 128 / sw row phases:
            // consecutive threads store consecutive floats of a row, and a
            // narrow slab spreads its rows over more threads
            const int rp = kThreads / sw;
            const int cc = tid % sw, r0 = tid / sw;
            const int64_t n = n0 + c0 + cc;
            const bool col_ok = (r0 < rp) && (n < g.N);
            const float bias_v = (g.bias && col_ok) ? __ldg(g.bias + n) : 0.f;
            const float ws_v = (FP8 && col_ok) ? __ldg(g.wsinv + n) : 1.f;
            const int nrow = (kTileM + rp - 1) / rp;
            for (int b = 0; 16 * b < nrow; ++b) {
                float rv[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int rr = r0 + rp * (16 * b + j);
                    const int64_t m = m0 + rr;
                    rv[j] = ((EPI == EPI_RESID || EPI == EPI_DGELU || EPI == EPI_DRELU) && col_ok && rr < kTileM &&
                             m < g.M)
                                ? g.resid[zoff + m * g.ldy + n]
                                : 0.f;
                }
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int rr = r0 + rp * (16 * b + j);
                    const int64_t m = m0 + rr;
                    if (!col_ok || rr >= kTileM || m >= g.M) continue;
                    const float v = (FP8 ? slab[rr * 64 + (cc ^ (rr & 31))] * ws_v : slab[rr * 64 + (cc ^ (rr & 31))]) +
                                    bias_v;
                    const int64_t o = zoff + m * g.ldy + n;
                    if (EPI == EPI_STORE) {
                        g.Y[o] = v;
                    } else if (EPI == EPI_GELU) {
                        g.Y[o] = v;
                        g.Y2[o] = gelu_f(v);
                    } else if (EPI == EPI_RELU) {
                        g.Y[o] = v;
                        g.Y2[o] = v > 0.f ? v : 0.f;
                    } else if (EPI == EPI_RESID) {
                        g.Y[o] = rv[j] + v;
                    } else if (EPI == EPI_DGELU) {
                        g.Y[o] = v * gelu_grad_f(rv[j]);
                    } else {
                        g.Y[o] = rv[j] > 0.f ? v : 0.f;
                    }
                }
            }
            __syncthreads();
        }
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        fence_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(g.tmem_cols) : "memory");
    }
}

}  // namespace tc
}  // namespace nnqs
