// Warp-specialised tcgen05 GEMM for the non-transposed layers with K = 64
// (one 64-wide K chunk per tile): Y[M][N] (epilogue) = X[M][64] W[N][64]^T.
//
// One CTA of 14 warps per SM keeps one N tile (n0, Nt columns, its weights
// resident in shared memory) and walks M tiles m = blockIdx.x / n_tiles,
// + gridDim.x / n_tiles, ...  The warps run concurrently, joined by
// mbarrier rings (full / empty pairs, two slots each):
//   warp 0      TMA producer: tile i's FP32 rows (two 32 x 128 boxes,
//               128-byte swizzle) into stage i % 2;
//   warps 1-4   converters: stage -> BF16 operand tile (high and, split, low
//               parts) in the MMA's swizzled layout, operand buffer i % 2;
//   warp 5      MMA issuer: the tile's MMAs into TMEM accumulator i % 2,
//               committed to the operand's empty and the accumulator's full
//               barriers;
//   warps 6-13  epilogue, two warpgroups splitting the 32-column boxes (warp w
//               reads TMEM lanes 32 (w % 4)..): TMEM -> registers -> shared
//               boxes -> TMA stores; the residual / pre-activation box comes
//               in by TMA into the output box first.
// Per element the arithmetic is k_tc_gemm's (same BF16 split, same MMA order,
// same epilogue expressions), so both kernels give identical results.
//
// Measured on a 40-qubit step (ncu, four launches each): the split forward
// with a plain store (qkv) 412 -> 320 us; with two outputs (FFN-in + GELU)
// 742 -> 826 us and with a pre-activation input (GELU' input gradient)
// 800 -> 1,217 us, since one epilogue role per SM then waits on its boxes'
// stores and loads that three interleaved k_tc_gemm CTAs hide.  The library
// uses it for the first case only.
//
// Every wait is bounded and also gives up when another warp has recorded a
// failure (shared abort flag); the kernel then records NNQS_E_TIMEOUT, lets
// its copies and MMAs in flight land (bounded) and frees its TMEM.
#pragma once
#include "tc_gemm.cuh"

namespace nnqs {
namespace tc {

constexpr int kWsWarps = 14, kWsThreads = 32 * kWsWarps;
constexpr int kWsStage = 32768;     // FP32 tile: 128 rows x 64 columns
constexpr int kWsSmemMax = 232448;  // 227 KB opt-in per CTA
constexpr int kWsFixed = 2048 + 1024;  // barriers, flags, column-sum scratch; alignment slack

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(mbar) : "memory");
}

// bounded wait that also stops once *abort is set
__device__ __forceinline__ bool mbar_wait_ab(uint32_t mbar, uint32_t parity, const volatile int *abort) {
    const long long t0 = clock64();
    for (uint32_t it = 0; it < (1u << 26); ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (ok) return true;
        if ((it & 31u) == 31u && (*abort || clock64() - t0 > 4000000000ll)) return false;
    }
    return false;
}

__device__ __forceinline__ void ws_named_sync(int id, int n) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// named barrier that also ANDs a predicate over its n threads
__device__ __forceinline__ bool ws_named_and(int id, int n, bool pred) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(r)
        : "r"(pred ? 1u : 0u), "r"(id), "r"(n)
        : "memory");
    return r != 0;
}

template <int EPI, bool SPLIT>
__global__ void __launch_bounds__(kWsThreads, 1) k_tc_gemm_ws(const __grid_constant__ Args g) {
    constexpr bool kNeedR = EPI == EPI_RESID || EPI == EPI_DGELU || EPI == EPI_DRELU;
    constexpr bool kTwo = EPI == EPI_GELU || EPI == EPI_RELU;
    constexpr int kOpBytes = (SPLIT ? 2 : 1) * kABytes;  // one operand buffer (high [, low])
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *sbase = smem_raw + (base - raw);

    const int Nt = g.Nt;
    const int w_bytes = (SPLIT ? 2 : 1) * Nt * 128;  // one K chunk of the weights
    uint8_t *sW = sbase;
    uint8_t *sSt = sbase + ((w_bytes + 1023) / 1024) * 1024;  // 2 FP32 stages
    uint8_t *sOp = sSt + 2 * kWsStage;                         // 2 operand buffers
    uint8_t *sE = sOp + 2 * kOpBytes;                           // 2 warpgroups x p_wg_epi
    uint8_t *sBar = sE + 2 * g.p_wg_epi;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sBar);
    // barrier slots: full[2] empty[2] ofull[2] oempty[2] afull[2] aempty[2] epir[2]
    const uint32_t b0 = smem_u32(bars);
    auto bar = [&](int kind, int k) { return b0 + 8u * uint32_t(2 * kind + k); };
    enum { FULL = 0, EMPTY = 1, OFULL = 2, OEMPTY = 3, AFULL = 4, AEMPTY = 5, EPIR = 6 };
    volatile int *abort_flag = reinterpret_cast<volatile int *>(sBar + 128);
    int *counts = reinterpret_cast<int *>(sBar + 136);  // loads issued, loads taken, MMAs issued, MMAs taken
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sBar + 160);
    float *cpart_all = reinterpret_cast<float *>(sBar + 1024);  // [2 warpgroups][128]

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntiles = g.p_ntiles;
    const int64_t n0 = int64_t(blockIdx.x % ntiles) * Nt;
    const int64_t m_first = blockIdx.x / ntiles, m_stride = gridDim.x / ntiles;
    const int64_t m_tiles = (g.M + kTileM - 1) / kTileM;
    const int64_t t_local = m_first < m_tiles ? (m_tiles - m_first + m_stride - 1) / m_stride : 0;
    auto m0_of = [&](int64_t i) { return (m_first + i * m_stride) * kTileM; };

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(g.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int k = 0; k < 2; ++k) {
            mbar_init(bar(FULL, k), 1);
            mbar_init(bar(EMPTY, k), 4);
            mbar_init(bar(OFULL, k), 4);
            mbar_init(bar(OEMPTY, k), 1);
            mbar_init(bar(AFULL, k), 1);
            mbar_init(bar(AEMPTY, k), 8);
            mbar_init(bar(EPIR, k), 1);
        }
        *abort_flag = 0;
        counts[0] = counts[1] = counts[2] = counts[3] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // the N tile's weights (high then low part) in the MMA layout
    for (int it = tid; it < Nt * 8; it += kWsThreads) {
        const int r = it >> 3, q = it & 7;
        const int64_t n = n0 + r;
        const int off = r * 128 + ((q ^ (r & 7)) << 4);
        *reinterpret_cast<uint4 *>(sW + off) =
            n < g.N ? __ldg(reinterpret_cast<const uint4 *>(g.Wt + n * g.Kpad + q * 8)) : make_uint4(0u, 0u, 0u, 0u);
        if (SPLIT)
            *reinterpret_cast<uint4 *>(sW + Nt * 128 + off) =
                n < g.N ? __ldg(reinterpret_cast<const uint4 *>(g.Wt2 + n * g.Kpad + q * 8))
                        : make_uint4(0u, 0u, 0u, 0u);
    }
    fence_async_smem();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tslot;

    if (warp == 0) {
        // ---- producer
        if (lane == 0) {
            for (int64_t i = 0; i < t_local; ++i) {
                const int s = (int)(i & 1);
                const uint32_t u = uint32_t(i >> 1);
                if (!mbar_wait_ab(bar(EMPTY, s), (u & 1u) ^ 1u, abort_flag)) {
                    *abort_flag = 1;
                    break;
                }
                const uint32_t dst = smem_u32(sSt + s * kWsStage);
                mbar_expect(bar(FULL, s), uint32_t(kWsStage));
                tma_load_box(dst, &g.tmX, 0, (int)m0_of(i), 0, bar(FULL, s));
                tma_load_box(dst + 16384, &g.tmX, 32, (int)m0_of(i), 0, bar(FULL, s));
                counts[0] = (int)(i + 1);
            }
        }
    } else if (warp <= 4) {
        // ---- converters (128 threads)
        const int ct = tid - 32;
        for (int64_t i = 0; i < t_local; ++i) {
            const int s = (int)(i & 1), o = (int)(i & 1);
            const uint32_t u = uint32_t(i >> 1);
            bool got = mbar_wait_ab(bar(FULL, s), u & 1u, abort_flag);
            got = got && mbar_wait_ab(bar(OEMPTY, o), (u & 1u) ^ 1u, abort_flag);
            if (!__all_sync(0xffffffffu, got)) {  // warp-uniform: the lanes leave together
                if (lane == 0) *abort_flag = 1;
                break;
            }
            if (ct == 0) counts[1] = (int)(i + 1);
            uint8_t *opA = sOp + o * kOpBytes, *opA2 = opA + kABytes;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int it = ct + 128 * k;
                const int r = it >> 3, c = it & 7, ph = r & 7;
                const uint8_t *bx = sSt + s * kWsStage + (c >> 2) * 16384 + r * 128;
                const int q0 = (c & 3) * 2;
                const float4 a = *reinterpret_cast<const float4 *>(bx + ((q0 ^ ph) << 4));
                const float4 b = *reinterpret_cast<const float4 *>(bx + (((q0 + 1) ^ ph) << 4));
                const float v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
                const int off = r * 128 + ((c ^ ph) << 4);
                *reinterpret_cast<uint4 *>(opA + off) = pack8(v);
                if (SPLIT) {
                    float lo[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) lo[e] = v[e] - __bfloat162float(__float2bfloat16_rn(v[e]));
                    *reinterpret_cast<uint4 *>(opA2 + off) = pack8(lo);
                }
            }
            fence_async_smem();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(bar(EMPTY, s));
                mbar_arrive(bar(OFULL, o));
            }
        }
    } else if (warp == 5) {
        // ---- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(kTileM, Nt);
            const uint64_t db = desc_sw128(smem_u32(sW)), db2 = desc_sw128(smem_u32(sW + Nt * 128));
            for (int64_t i = 0; i < t_local; ++i) {
                const int o = (int)(i & 1), a = (int)(i & 1);
                const uint32_t u = uint32_t(i >> 1);
                if (!mbar_wait_ab(bar(OFULL, o), u & 1u, abort_flag) ||
                    !mbar_wait_ab(bar(AEMPTY, a), (u & 1u) ^ 1u, abort_flag)) {
                    *abort_flag = 1;
                    break;
                }
                fence_after_sync();
                const uint32_t dt = tmem + uint32_t(a) * uint32_t(Nt);
                const uint64_t da = desc_sw128(smem_u32(sOp + o * kOpBytes));
                const uint64_t da2 = desc_sw128(smem_u32(sOp + o * kOpBytes + kABytes));
#pragma unroll
                for (int k = 0; k < kChunkK / 16; ++k) {
                    if (SPLIT) {  // small terms first, as k_tc_gemm
                        mma_bf16(dt, da2 + uint64_t(2 * k), db + uint64_t(2 * k), idesc, k > 0 ? 1u : 0u);
                        mma_bf16(dt, da + uint64_t(2 * k), db2 + uint64_t(2 * k), idesc, 1u);
                        mma_bf16(dt, da + uint64_t(2 * k), db + uint64_t(2 * k), idesc, 1u);
                    } else {
                        mma_bf16(dt, da + uint64_t(2 * k), db + uint64_t(2 * k), idesc, k > 0 ? 1u : 0u);
                    }
                }
                mma_commit(bar(OEMPTY, o));
                mma_commit(bar(AFULL, a));
                counts[2] = (int)(i + 1);
            }
        }
    } else {
        // ---- epilogue (256 threads, two warpgroups)
        const int et = tid - 192, wg = et >> 7, q4 = warp & 3, row = 32 * q4 + lane;
        const bool leader = (et & 127) == 0;
        const int nb = Nt / 32, nmine = (nb - wg + 1) / 2;  // boxes b = wg, wg + 2, ...
        uint8_t *obuf = sE + wg * g.p_wg_epi;
        float *cpart = cpart_all + wg * 128;
        for (int64_t i = 0; i < t_local; ++i) {
            const int a = (int)(i & 1);
            const uint32_t u = uint32_t(i >> 1);
            const int64_t m0 = m0_of(i);
            bool good = true;
            if (!kTwo) {
                // my output boxes free (the previous tile's stores have read
                // them), then the residual / pre-activation boxes into them
                if (leader) {
                    bulk_wait_read();
                    if (kNeedR && nmine > 0) {
                        mbar_expect(bar(EPIR, wg), uint32_t(16384 * nmine));
                        for (int j = 0; j < nmine; ++j)
                            tma_load_box(smem_u32(obuf + j * 16384), &g.tmR, (int)(n0 + 32 * (wg + 2 * j)), (int)m0,
                                         0, bar(EPIR, wg));
                    }
                }
            }
            good = mbar_wait_ab(bar(AFULL, a), u & 1u, abort_flag);
            if (good && kNeedR && nmine > 0) good = mbar_wait_ab(bar(EPIR, wg), uint32_t(i & 1), abort_flag);
            // the warpgroup leaves together when any thread failed or saw the abort flag
            if (!ws_named_and(1 + wg, 128, good && *abort_flag == 0)) {
                if (leader) *abort_flag = 1;
                break;
            }
            if (leader && wg == 0) counts[3] = (int)(i + 1);
            fence_after_sync();
            const uint32_t lane_base = tmem + (uint32_t(32 * q4) << 16) + uint32_t(a) * uint32_t(Nt);
            if (!kTwo) {
                for (int j = 0; j < nmine; ++j) {
                    const int b = wg + 2 * j;
                    uint8_t *box = obuf + j * 16384;
                    uint32_t r[32];
                    tmem_ld16(lane_base + uint32_t(32 * b), *reinterpret_cast<uint32_t(*)[16]>(r));
                    tmem_ld16(lane_base + uint32_t(32 * b + 16), *reinterpret_cast<uint32_t(*)[16]>(r + 16));
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int off = row * 128 + ((q ^ (row & 7)) << 4);
                        float4 rv = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (kNeedR) rv = *reinterpret_cast<const float4 *>(box + off);
                        const float rr[4] = {rv.x, rv.y, rv.z, rv.w};
                        float y[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int64_t n = n0 + 32 * b + 4 * q + e;
                            const float bias_v = (g.bias && n < g.N) ? __ldg(g.bias + n) : 0.f;
                            const float v = __uint_as_float(r[4 * q + e]) + bias_v;
                            if (EPI == EPI_STORE)
                                y[e] = v;
                            else if (EPI == EPI_RESID)
                                y[e] = rr[e] + v;
                            else if (EPI == EPI_DGELU)
                                y[e] = v * gelu_grad_f(rr[e]);
                            else
                                y[e] = rr[e] > 0.f ? v : 0.f;
                        }
                        *reinterpret_cast<float4 *>(box + off) = make_float4(y[0], y[1], y[2], y[3]);
                    }
                }
                // the accumulator is read: the MMA warp may refill it
                fence_before_sync();
                __syncwarp();
                if (lane == 0) mbar_arrive(bar(AEMPTY, a));
                fence_async_smem();
                ws_named_sync(1 + wg, 128);
                if (g.colpart) {
                    const int rmax = (int)min((int64_t)kTileM, g.M - m0);
                    for (int j = 0; j < nmine; ++j) {
                        const int b = wg + 2 * j;
                        const uint8_t *box = obuf + j * 16384;
                        const int t = et & 127, cl = t & 31, q = cl >> 2, e = cl & 3, rg = t >> 5;
                        float cs = 0.f;
                        for (int rr2 = 32 * rg; rr2 < min(32 * rg + 32, rmax); ++rr2)
                            cs += *reinterpret_cast<const float *>(box + rr2 * 128 + ((q ^ (rr2 & 7)) << 4) + 4 * e);
                        cpart[rg * 32 + cl] = cs;
                        ws_named_sync(1 + wg, 128);
                        if (t < 32 && n0 + 32 * b + t < g.N)
                            g.colpart[(m0 / kTileM) * g.N + n0 + 32 * b + t] =
                                ((cpart[t] + cpart[32 + t]) + cpart[64 + t]) + cpart[96 + t];
                        ws_named_sync(1 + wg, 128);
                    }
                }
                if (leader) {
                    for (int j = 0; j < nmine; ++j)
                        tma_store_box(&g.tmY, smem_u32(obuf + j * 16384), (int)(n0 + 32 * (wg + 2 * j)), (int)m0, 0);
                    bulk_commit();
                }
            } else {
                // two outputs, one box at a time through the pair (Y, activation)
                for (int j = 0; j < nmine; ++j) {
                    const int b = wg + 2 * j;
                    uint8_t *box = obuf, *box2 = obuf + 16384;
                    if (leader) bulk_wait_read();
                    ws_named_sync(1 + wg, 128);
                    uint32_t r[32];
                    tmem_ld16(lane_base + uint32_t(32 * b), *reinterpret_cast<uint32_t(*)[16]>(r));
                    tmem_ld16(lane_base + uint32_t(32 * b + 16), *reinterpret_cast<uint32_t(*)[16]>(r + 16));
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int off = row * 128 + ((q ^ (row & 7)) << 4);
                        float y[4], y2[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int64_t n = n0 + 32 * b + 4 * q + e;
                            const float bias_v = (g.bias && n < g.N) ? __ldg(g.bias + n) : 0.f;
                            const float v = __uint_as_float(r[4 * q + e]) + bias_v;
                            y[e] = v;
                            y2[e] = EPI == EPI_GELU ? gelu_f(v) : (v > 0.f ? v : 0.f);
                        }
                        *reinterpret_cast<float4 *>(box + off) = make_float4(y[0], y[1], y[2], y[3]);
                        *reinterpret_cast<float4 *>(box2 + off) = make_float4(y2[0], y2[1], y2[2], y2[3]);
                    }
                    fence_async_smem();
                    ws_named_sync(1 + wg, 128);
                    if (leader) {
                        tma_store_box(&g.tmY, smem_u32(box), (int)(n0 + 32 * b), (int)m0, 0);
                        tma_store_box(&g.tmY2, smem_u32(box2), (int)(n0 + 32 * b), (int)m0, 0);
                        bulk_commit();
                    }
                }
                fence_before_sync();
                __syncwarp();
                if (lane == 0) mbar_arrive(bar(AEMPTY, a));
            }
        }
        if (leader) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");  // stores complete
    }
    fence_before_sync();
    __syncthreads();
    if (*abort_flag && tid == 0) {
        if (atomicCAS(&g.st->code, 0, (int)NNQS_E_TIMEOUT) == 0) g.st->index = -14;
        // loads and MMAs still in flight land (bounded) before the CTA ends
        for (int i = counts[1]; i < counts[0]; ++i) mbar_wait(bar(FULL, i & 1), uint32_t((i >> 1) & 1));
        for (int i = counts[3]; i < counts[2]; ++i) mbar_wait(bar(AFULL, i & 1), uint32_t((i >> 1) & 1));
    }
    __syncthreads();
    if (warp == 0) {
        fence_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(g.tmem_cols)
                     : "memory");
    }
}

}  // namespace tc
}  // namespace nnqs
