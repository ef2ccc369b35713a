// Host side of the tcgen05 linear layers used by NNQS_MIXED and NNQS_BF16X3:
// BF16 copies of the weight matrices (K padded to 64 with zeros) and their
// low parts, and the launch of tc::k_tc_gemm.
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "dev_common.cuh"
#include "tc_gemm.cuh"
#include "tc_gemm_ws.cuh"
#include "tc_gemm.h"

namespace nnqs {
namespace {

// every conversion of one tc_weights_prepare in one launch; job y is one of
//   kind 0: W [N][K] -> dst [N][pad] BF16 and dst_lo = bf16(W - bf16(W))
//   kind 1: W^T -> dst [K][pad] (rows = K, cols = N)
//   kind 2: the swizzled shared-memory image of W [N][pad]: K block kc is
//           N rows of 128 bytes at kc * N * 64 elements, granule c of row r
//           stored at granule c ^ (r & 7); low parts in dst_lo
struct ConvJob {
    int64_t src, rows, cols, pad;
    __nv_bfloat16 *dst, *dst_lo;
    int kind;
};
constexpr int kMaxConvJobs = 64;
struct ConvTab {
    int n;
    ConvJob j[kMaxConvJobs];
};

__global__ void k_to_bf16_all(const float *__restrict__ params, ConvTab tab) {
    const ConvJob jb = tab.j[blockIdx.y];
    const int64_t total = jb.rows * jb.pad;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t r, c;
        if (jb.kind == 2) {
            const int64_t blk = jb.rows * 64;
            const int64_t kc = i / blk, q = i % blk;
            r = q / 64;
            const int pos = (int)(q % 64);
            c = kc * 64 + (((pos >> 3) ^ (int)(r & 7)) << 3) + (pos & 7);
        } else {
            r = i / jb.pad;
            c = i % jb.pad;
        }
        float v = 0.f;
        if (c < jb.cols) v = jb.kind == 1 ? params[jb.src + c * jb.rows + r] : params[jb.src + r * jb.cols + c];
        const __nv_bfloat16 hi = __float2bfloat16_rn(v);
        jb.dst[i] = hi;
        if (jb.dst_lo) jb.dst_lo[i] = __float2bfloat16_rn(v - __bfloat162float(hi));
    }
}

// E4M3 copy of one forward matrix per blockIdx.y (slot job), one warp per
// row: s_n = 2^k with k the largest integer such that max_k |W[n][k]| 2^k <=
// 448 (1 for an all-zero row), dst[n][c] = e4m3(W[n][c] s_n) (zero past K),
// inv[n] = 2^-k
struct Fp8Job {
    int64_t src, rows, cols, pad;
    uint8_t *dst;
    float *inv;
};
struct Fp8Tab {
    int n;
    Fp8Job j[64];
};

__global__ void k_to_fp8_all(const float *__restrict__ params, Fp8Tab tab) {
    const Fp8Job jb = tab.j[blockIdx.y];
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t r = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); r < jb.rows; r += warps) {
        const float *w = params + jb.src + r * jb.cols;
        float amax = 0.f;
        for (int64_t c = lane; c < jb.cols; c += 32) amax = fmaxf(amax, fabsf(w[c]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
        int k = 0;
        if (amax > 0.f && isfinite(amax)) {
            int e;
            frexpf(448.f / amax, &e);  // 448 / amax = f 2^e with f in [0.5, 1)
            k = e - 1;                 // 2^k <= 448 / amax < 2^(k+1)
            for (int it = 0; it < 4 && ldexpf(amax, k) > 448.f; ++it) --k;  // rounding of the quotient
            k = max(-120, min(120, k));  // 2^k and 2^-k stay finite normal floats
        }
        const float sc = ldexpf(1.f, k);
        for (int64_t c = lane; c < jb.pad; c += 32) {
            const float v = c < jb.cols ? w[c] * sc : 0.f;
            jb.dst[r * jb.pad + c] = (uint8_t)(__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3));
        }
        if (lane == 0) jb.inv[r] = ldexpf(1.f, -k);
    }
}

// dW[o][i] += sum_z partial[z][.], splits in order; partial is [z][out][in],
// or [z][in][out] when the GEMM ran transposed (trans)
__global__ void k_tc_reduce(const float *__restrict__ partial, int64_t splits, int64_t out_n, int64_t in_n, int trans,
                            float *__restrict__ dW) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t n = out_n * in_n;
    if (i >= n) return;
    const int64_t src = trans ? (i % in_n) * out_n + i / in_n : i;
    float acc = 0.f;
    for (int64_t z = 0; z < splits; ++z) acc += partial[z * n + src];
    dW[i] += acc;
}

// the same sum with more threads: a block takes 128 consecutive partial
// elements (a lane: 4 of them as float4), its 32 warps split the splits (warp
// w: z = w, w + 32, ...), and the 32 warp sums are added in warp order
__global__ void __launch_bounds__(1024) k_tc_reduce4(const float *__restrict__ partial, int64_t splits, int64_t out_n,
                                                     int64_t in_n, int trans, float *__restrict__ dW) {
    __shared__ float4 sh[32][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t n = out_n * in_n;
    const int64_t e0 = blockIdx.x * 128 + 4 * lane;  // first of this lane's 4 elements
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    if (e0 < n) {
        int64_t z = warp;
        for (; z + 96 < splits; z += 128) {
            const float4 a = __ldg(reinterpret_cast<const float4 *>(partial + z * n + e0));
            const float4 b = __ldg(reinterpret_cast<const float4 *>(partial + (z + 32) * n + e0));
            const float4 c = __ldg(reinterpret_cast<const float4 *>(partial + (z + 64) * n + e0));
            const float4 d = __ldg(reinterpret_cast<const float4 *>(partial + (z + 96) * n + e0));
            acc.x += a.x; acc.y += a.y; acc.z += a.z; acc.w += a.w;
            acc.x += b.x; acc.y += b.y; acc.z += b.z; acc.w += b.w;
            acc.x += c.x; acc.y += c.y; acc.z += c.z; acc.w += c.w;
            acc.x += d.x; acc.y += d.y; acc.z += d.z; acc.w += d.w;
        }
        for (; z < splits; z += 32) {
            const float4 a = __ldg(reinterpret_cast<const float4 *>(partial + z * n + e0));
            acc.x += a.x; acc.y += a.y; acc.z += a.z; acc.w += a.w;
        }
    }
    sh[warp][lane] = acc;
    __syncthreads();
    if (warp == 0 && e0 < n) {
        float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int w = 0; w < 32; ++w) {
            const float4 v = sh[w][lane];
            t.x += v.x; t.y += v.y; t.z += v.z; t.w += v.w;
        }
        const float tv[4] = {t.x, t.y, t.z, t.w};
        for (int k = 0; k < 4; ++k) {
            const int64_t src = e0 + k;
            if (src >= n) break;
            // partial is [out][in], or [in][out] when transposed
            const int64_t dst = trans ? (src % out_n) * in_n + src / out_n : src;
            dW[dst] += tv[k];
        }
    }
}

// ---- tensor maps for the TMA epilogue
using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
    static EncodeTiled fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

// FP32 [Z][M][ld] (N valid columns) as a 3-D tensor with 32 x 128 x 1 boxes and
// the 128-byte swizzle; false when the layout does not meet the TMA rules
// (16-byte aligned base and row stride)
bool make_box_map(CUtensorMap *tm, const float *base, int64_t N, int64_t M, int64_t Z, int64_t ld) {
    EncodeTiled fn = encode_fn();
    if (!fn || !base || reinterpret_cast<uintptr_t>(base) % 16 != 0 || (ld * 4) % 16 != 0 || N < 1 || M < 1 ||
        Z < 1)
        return false;
    const cuuint64_t dims[3] = {(cuuint64_t)N, (cuuint64_t)M, (cuuint64_t)Z};
    const cuuint64_t strides[2] = {(cuuint64_t)(ld * 4), (cuuint64_t)(M * ld * 4)};
    const cuuint32_t box[3] = {32, (cuuint32_t)tc::kTileM, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return fn(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// turns on the TMA epilogue of g when every tensor it touches has a map
void setup_tma(tc::Args &g, int epi, int64_t Z) {
    g.use_tma = 0;
    if (!make_box_map(&g.tmY, g.Y, g.N, g.M, Z, g.ldy)) return;
    if ((epi == tc::EPI_GELU || epi == tc::EPI_RELU) && !make_box_map(&g.tmY2, g.Y2, g.N, g.M, Z, g.ldy)) return;
    if ((epi == tc::EPI_RESID || epi == tc::EPI_DGELU || epi == tc::EPI_DRELU) &&
        !make_box_map(&g.tmR, g.resid, g.N, g.M, Z, g.ldy))
        return;
    g.use_tma = 1;
}

int64_t kpad_of(int64_t K) { return (K + tc::kChunkK - 1) / tc::kChunkK * tc::kChunkK; }

// (N, K, source offset) of every slot
void slot_shapes(const nnqs_model *M, int slot, int64_t &N, int64_t &K, int64_t &src) {
    const int l = slot / 4, which = slot % 4;
    const int64_t d = M->d, F = M->F;
    if (l == M->L) {
        N = M->P;
        K = M->P;
        src = M->lay.ph_w2;
        return;
    }
    const auto &lo = M->lay.layer[l];
    switch (which) {
        case 0: N = 3 * d; K = d; src = lo.wqkv; break;
        case 1: N = d; K = d; src = lo.wo; break;
        case 2: N = F; K = d; src = lo.w1; break;
        default: N = d; K = F; src = lo.w2; break;
    }
}

bool g_attr_set[2][2][2][tc::kNumEpi] = {};

template <int EPI, bool TRANS = false, bool SPLIT = false, bool FP8 = false>
nnqs_status launch(const tc::Args &g, int64_t n_tiles_n, cudaStream_t s, int64_t splits = 1) {
    constexpr int smem = SPLIT ? tc::kSmemBytesSplit : tc::kSmemBytes;
    if (!g_attr_set[TRANS][SPLIT][FP8][EPI]) {
        NNQS_CUDA_TRY(cudaFuncSetAttribute(tc::k_tc_gemm<EPI, TRANS, SPLIT, FP8>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        g_attr_set[TRANS][SPLIT][FP8][EPI] = true;
    }
    dim3 grid((unsigned)n_tiles_n, (unsigned)((g.M + tc::kTileM - 1) / tc::kTileM), (unsigned)splits);
    NNQS_LAUNCH("k_tc_gemm", s, (tc::k_tc_gemm<EPI, TRANS, SPLIT, FP8><<<grid, tc::kThreads, smem, s>>>(g)));
    return NNQS_OK;
}

// N per CTA: the whole N rounded up to 16 when it fits in 128 columns, else
// the widest multiple of 16 up to 128 that divides N (fewer N tiles restage
// the A tile fewer times), else 128
int nt_base(int64_t N) {
    if (N <= 128) return (int)((N + 15) / 16 * 16);
    for (int nt = 128; nt >= 16; nt -= 16)
        if (N % nt == 0) return nt;
    return 128;
}

// for few row tiles (the sampler's one-token steps) the N tiles are halved
// down to 16 columns until two CTAs per SM are launched: a CTA's epilogue
// then covers fewer columns and the launch finishes sooner
int nt_for(int64_t M, int64_t N) {
    int nt = nt_base(N);
    const int64_t mt = (M + tc::kTileM - 1) / tc::kTileM;
    while (nt > 16 && nt % 32 == 0 && mt * ((N + nt - 1) / nt) < 2 * 152) nt /= 2;
    if (nt % 16 != 0) nt = (nt + 15) / 16 * 16;
    return nt;
}

int tmem_cols_for(int Nt) {
    int cols = 32;
    while (cols < Nt) cols <<= 1;
    return cols;
}

// the warp-specialised kernel takes a non-transposed layer with K = 64 (one
// K chunk per tile) when the TMA epilogue is on, its boxes and the FP32 /
// operand rings fit in shared memory, and there are enough row tiles to keep
// every SM busy for a few tiles
int ws_smem_of(const tc::Args &g, bool split) {
    const int w_bytes = (split ? 2 : 1) * g.Nt * 128;
    return (w_bytes + 1023) / 1024 * 1024 + 2 * tc::kWsStage + 2 * (split ? 2 : 1) * tc::kABytes + 2 * g.p_wg_epi +
           tc::kWsFixed;
}

bool ws_eligible(tc::Args &g, bool split, int epi) {
    if (!g.use_tma || g.Nt % 32 != 0 || g.Nt > 128 || g.K != tc::kChunkK || g.Kpad != tc::kChunkK) return false;
    const int64_t m_tiles = (g.M + tc::kTileM - 1) / tc::kTileM;
    if (m_tiles < 4 * int64_t(num_sms())) return false;
    const bool two = epi == tc::EPI_GELU || epi == tc::EPI_RELU;
    g.p_wg_epi = two ? 2 * 16384 : (g.Nt / 32 + 1) / 2 * 16384;
    if (ws_smem_of(g, split) > tc::kWsSmemMax) return false;
    return make_box_map(&g.tmX, g.X, g.K, g.M, 1, g.ldx);
}

template <int EPI, bool SPLIT>
nnqs_status launch_ws(tc::Args g, cudaStream_t s) {
    static int attr = 0;
    const int smem = ws_smem_of(g, SPLIT);
    if (smem > attr) {
        NNQS_CUDA_TRY(
            cudaFuncSetAttribute(tc::k_tc_gemm_ws<EPI, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        attr = smem;
    }
    const int ntiles = (int)((g.N + g.Nt - 1) / g.Nt);
    const int64_t m_tiles = (g.M + tc::kTileM - 1) / tc::kTileM;
    int64_t grid = (int64_t)(num_sms() / ntiles) * ntiles;
    grid = std::min<int64_t>(grid, m_tiles * ntiles);
    g.p_ntiles = ntiles;
    g.tmem_cols = tmem_cols_for(2 * g.Nt);
    NNQS_LAUNCH("k_tc_gemm", s, (tc::k_tc_gemm_ws<EPI, SPLIT><<<(unsigned)grid, tc::kWsThreads, smem, s>>>(g)));
    return NNQS_OK;
}

}  // namespace

void tc_weights_take(const nnqs_model *M, Arena &a, TcWeights *w) {
    const int n_slots = 4 * M->L + 1;
    int64_t total = 0;
    TcWeights tmp;
    TcWeights &t = w ? *w : tmp;
    t.n_slots = n_slots;
    for (int sl = 0; sl < n_slots; ++sl) {
        if (sl / 4 == M->L && sl % 4 != 0) continue;
        int64_t N, K, src;
        slot_shapes(M, sl, N, K, src);
        t.off[sl] = total;
        t.rows[sl] = (int32_t)N;
        t.cols[sl] = (int32_t)K;
        t.pcols[sl] = (int32_t)kpad_of(K);
        t.src[sl] = src;
        total += N * kpad_of(K);
        t.toff[sl] = total;
        t.tpcols[sl] = (int32_t)kpad_of(N);
        total += K * kpad_of(N);
    }
    t.bf16 = a.take<__nv_bfloat16>(size_t(total));
    t.bf16_lo = a.take<__nv_bfloat16>(size_t(total));
    int64_t tiles = 0;
    for (int sl = 0; sl < 4 * M->L; ++sl) {
        t.tile_off[sl] = tiles;
        tiles += 2 * int64_t(t.rows[sl]) * t.pcols[sl];
    }
    t.tiles = a.take<__nv_bfloat16>(size_t(std::max<int64_t>(tiles, 1)));
    int64_t b8 = 0, s8 = 0;
    for (int sl = 0; sl < n_slots; ++sl) {
        if (sl / 4 == M->L && sl % 4 != 0) continue;
        t.off8[sl] = b8;
        t.soff8[sl] = s8;
        t.pcols8[sl] = (int32_t)((t.cols[sl] + 127) / 128 * 128);
        b8 += int64_t(t.rows[sl]) * t.pcols8[sl];
        s8 += t.rows[sl];
    }
    t.w8 = a.take<uint8_t>(size_t(std::max<int64_t>(b8, 16)));
    t.w8inv = a.take<float>(size_t(std::max<int64_t>(s8, 1)));
}

nnqs_status tc_weights_prepare(const nnqs_model *M, const float *params, TcWeights &w, cudaStream_t s) {
    ConvTab tab{};
    auto flush = [&]() -> nnqs_status {
        if (tab.n == 0) return NNQS_OK;
        dim3 grid(64, (unsigned)tab.n);
        NNQS_LAUNCH("k_to_bf16", s, k_to_bf16_all<<<grid, 256, 0, s>>>(params, tab));
        tab.n = 0;
        return NNQS_OK;
    };
    __nv_bfloat16 *hi = static_cast<__nv_bfloat16 *>(w.bf16), *lo = static_cast<__nv_bfloat16 *>(w.bf16_lo);
    __nv_bfloat16 *tl = static_cast<__nv_bfloat16 *>(w.tiles);
    for (int sl = 0; sl < w.n_slots; ++sl) {
        if (sl / 4 == M->L && sl % 4 != 0) continue;
        const int64_t N = w.rows[sl], K = w.cols[sl], Kp = w.pcols[sl];
        if (tab.n + 3 > kMaxConvJobs) NNQS_TRY(flush());
        tab.j[tab.n++] = ConvJob{w.src[sl], N, K, Kp, hi + w.off[sl], lo + w.off[sl], 0};
        tab.j[tab.n++] = ConvJob{w.src[sl], K, N, w.tpcols[sl], hi + w.toff[sl], nullptr, 1};
        if (sl < 4 * M->L)
            tab.j[tab.n++] = ConvJob{w.src[sl], N, K, Kp, tl + w.tile_off[sl], tl + w.tile_off[sl] + N * Kp, 2};
    }
    NNQS_TRY(flush());
    if (!w.fp8) return NNQS_OK;
    Fp8Tab t8{};
    for (int sl = 0; sl < w.n_slots; ++sl) {
        if (sl / 4 == M->L && sl % 4 != 0) continue;
        t8.j[t8.n++] = Fp8Job{w.src[sl], w.rows[sl], w.cols[sl], w.pcols8[sl], w.w8 + w.off8[sl], w.w8inv + w.soff8[sl]};
        if (t8.n == 64 || sl + 1 == w.n_slots) {
            NNQS_LAUNCH("k_to_bf16", s, k_to_fp8_all<<<dim3(16, (unsigned)t8.n), 256, 0, s>>>(params, t8));
            t8.n = 0;
        }
    }
    if (t8.n > 0) NNQS_LAUNCH("k_to_bf16", s, k_to_fp8_all<<<dim3(16, (unsigned)t8.n), 256, 0, s>>>(params, t8));
    return NNQS_OK;
}

nnqs_status tc_linear_dx(cudaStream_t s, const TcWeights &w, int slot, const float *dY, int64_t rows, float *dX,
                         int act, const float *Z, float *colpart, bool *colpart_done) {
    if (colpart_done) *colpart_done = false;
    if (rows == 0) return NNQS_OK;
    if (act != 0 && Z == nullptr) return set_error(NNQS_E_INVAL, "tensor-core input gradient: pre-activation missing");
    tc::Args g{};
    const int64_t out = w.rows[slot], in = w.cols[slot];
    g.X = dY;
    g.ldx = out;
    g.Wt = static_cast<const __nv_bfloat16 *>(w.bf16) + w.toff[slot];
    g.Kpad = w.tpcols[slot];
    g.Y = dX;
    g.ldy = in;
    g.M = rows;
    g.N = in;
    g.K = out;
    g.Nt = nt_for(g.M, g.N);
    g.vec_x = (out % 4 == 0) && (reinterpret_cast<uintptr_t>(dY) % 16 == 0);
    g.tmem_cols = tmem_cols_for(g.Nt);
    g.st = w.st;
    g.resid = Z;
    setup_tma(g, act == 1 ? tc::EPI_DGELU : act == 2 ? tc::EPI_DRELU : tc::EPI_STORE, 1);
    if (g.use_tma && g.Nt % 32 == 0 && colpart) {
        g.colpart = colpart;
        if (colpart_done) *colpart_done = true;
    }
    note_work("k_tc_gemm", 2.0 * double(rows) * double(in) * double(out),
              4.0 * double(rows) * out + 2.0 * double(in) * g.Kpad + (act ? 8.0 : 4.0) * double(rows) * in);
    const int64_t ntn = (g.N + g.Nt - 1) / g.Nt;
    if (act == 1) return launch<tc::EPI_DGELU>(g, ntn, s);
    if (act == 2) return launch<tc::EPI_DRELU>(g, ntn, s);
    return launch<tc::EPI_STORE>(g, ntn, s);
}

nnqs_status tc_linear_dw(cudaStream_t s, const float *dY, int64_t rows, int64_t out, const float *X, int64_t in,
                         float *dW, float *scratch, size_t scratch_elems, DevStatus *st) {
    if (rows == 0) return NNQS_OK;
    // dW = dY^T X ([out][in]) or its transpose X^T dY ([in][out]): the
    // orientation whose 128-row tiles and N tiles waste fewer padded rows
    auto padded = [](int64_t M, int64_t N) {
        const int64_t nt = nt_base(N);
        return ((M + tc::kTileM - 1) / tc::kTileM * tc::kTileM) * ((N + nt - 1) / nt * nt);
    };
    const bool swap = padded(in, out) < padded(out, in);
    tc::Args g{};
    g.X = swap ? X : dY;
    g.ldx = swap ? in : out;
    g.Xb = swap ? dY : X;
    g.ldb = swap ? out : in;
    g.M = swap ? in : out;
    g.N = swap ? out : in;
    g.K = rows;
    g.Nt = nt_base(g.N);
    g.vec_x = (out % 4 == 0) && (in % 4 == 0) && (reinterpret_cast<uintptr_t>(dY) % 16 == 0) &&
              (reinterpret_cast<uintptr_t>(X) % 16 == 0);
    g.tmem_cols = tmem_cols_for(g.Nt);
    g.st = st;
    const int64_t ntn = (g.N + g.Nt - 1) / g.Nt;
    const int64_t tiles = ((g.M + tc::kTileM - 1) / tc::kTileM) * ntn;
    // about four CTAs per SM over the row splits
    int64_t splits = std::max<int64_t>(1, (4 * 152 + tiles - 1) / tiles);
    splits = std::min<int64_t>(splits, (rows + tc::kChunkK - 1) / tc::kChunkK);
    splits = std::min<int64_t>(splits, (int64_t)(scratch_elems / size_t(out * in)));
    if (splits < 1) return set_error(NNQS_E_WORKSPACE, "tensor-core weight gradient: scratch too small");
    g.kchunk = ((rows + splits - 1) / splits + tc::kChunkK - 1) / tc::kChunkK * tc::kChunkK;
    splits = (rows + g.kchunk - 1) / g.kchunk;
    g.Y = scratch;
    g.ldy = g.N;
    setup_tma(g, tc::EPI_STORE, splits);
    note_work("k_tc_gemm", 2.0 * double(rows) * double(in) * double(out),
              4.0 * double(rows) * (out + in) + 4.0 * double(splits) * out * in);
    NNQS_TRY((launch<tc::EPI_STORE, true>(g, ntn, s, splits)));
    if ((out * in) % 4 == 0)
        NNQS_LAUNCH("k_tc_reduce", s,
                    k_tc_reduce4<<<(unsigned)((out * in + 127) / 128), 1024, 0, s>>>(scratch, splits, out, in,
                                                                                    swap ? 1 : 0, dW));
    else
        NNQS_LAUNCH("k_tc_reduce", s,
                    k_tc_reduce<<<grid_for(out * in, 256), 256, 0, s>>>(scratch, splits, out, in, swap ? 1 : 0, dW));
    return NNQS_OK;
}

template <>
nnqs_status tc_linear_fwd_ld<float>(cudaStream_t s, const TcWeights &w, int slot, int epi, const float *X,
                                    int64_t rows, int64_t in, const float *bias, float *Y, int64_t ldy, float *Y2,
                                    const float *resid) {
    if (rows == 0) return NNQS_OK;
    if (in != w.cols[slot]) return set_error(NNQS_E_INVAL, "tensor-core layer: input width mismatch");
    if ((epi == tc::EPI_GELU || epi == tc::EPI_RELU) && Y2 == nullptr)
        return set_error(NNQS_E_INVAL, "tensor-core layer: activation output missing");
    if (epi == tc::EPI_RESID && resid == nullptr)
        return set_error(NNQS_E_INVAL, "tensor-core layer: residual input missing");
    tc::Args g{};
    g.X = X;
    g.ldx = in;
    g.Wt = static_cast<const __nv_bfloat16 *>(w.bf16) + w.off[slot];
    g.Wt2 = static_cast<const __nv_bfloat16 *>(w.bf16_lo) + w.off[slot];
    g.Kpad = w.pcols[slot];
    g.bias = bias;
    g.resid = resid;
    g.Y = Y;
    g.Y2 = Y2;
    g.ldy = ldy;
    g.M = rows;
    g.N = w.rows[slot];
    g.K = in;
    g.Nt = nt_for(g.M, g.N);
    g.vec_x = (in % 4 == 0) && (reinterpret_cast<uintptr_t>(X) % 16 == 0);
    g.tmem_cols = tmem_cols_for(g.Nt);
    g.st = w.st;
    setup_tma(g, epi, 1);
    const int64_t ntn = (g.N + g.Nt - 1) / g.Nt;
    // algorithmic bytes: X in, the BF16 weights (and their low parts), Y out,
    // plus the activation output or the residual read
    const bool two = epi == tc::EPI_GELU || epi == tc::EPI_RELU || epi == tc::EPI_RESID;
    // flops: the method's product only (the split mode issues three BF16
    // products for it)
    note_work("k_tc_gemm", 2.0 * double(rows) * double(g.N) * double(in),
              4.0 * double(rows) * in + (w.split ? 4.0 : 2.0) * double(g.N) * g.Kpad +
                  (two ? 8.0 : 4.0) * double(rows) * g.N);
    if (w.fp8) {
        g.W8 = w.w8 + w.off8[slot];
        g.Kpad8 = w.pcols8[slot];
        g.wsinv = w.w8inv + w.soff8[slot];
        switch (epi) {
            case tc::EPI_STORE: return launch<tc::EPI_STORE, false, false, true>(g, ntn, s);
            case tc::EPI_GELU: return launch<tc::EPI_GELU, false, false, true>(g, ntn, s);
            case tc::EPI_RELU: return launch<tc::EPI_RELU, false, false, true>(g, ntn, s);
            case tc::EPI_RESID: return launch<tc::EPI_RESID, false, false, true>(g, ntn, s);
            default: return set_error(NNQS_E_INVAL, "tensor-core layer: bad epilogue");
        }
    }
    // the warp-specialised kernel only where it measured faster: the split
    // forward with a plain store (the qkv layer: 412 -> 320 us for the four
    // launches of a 40-qubit step); with two outputs or a residual its one
    // epilogue role per SM is slower than three interleaved CTAs
    if (w.split && epi == tc::EPI_STORE && ws_eligible(g, true, epi)) return launch_ws<tc::EPI_STORE, true>(g, s);
    if (w.split) {
        switch (epi) {
            case tc::EPI_STORE: return launch<tc::EPI_STORE, false, true>(g, ntn, s);
            case tc::EPI_GELU: return launch<tc::EPI_GELU, false, true>(g, ntn, s);
            case tc::EPI_RELU: return launch<tc::EPI_RELU, false, true>(g, ntn, s);
            case tc::EPI_RESID: return launch<tc::EPI_RESID, false, true>(g, ntn, s);
            default: return set_error(NNQS_E_INVAL, "tensor-core layer: bad epilogue");
        }
    }
    switch (epi) {
        case tc::EPI_STORE: return launch<tc::EPI_STORE>(g, ntn, s);
        case tc::EPI_GELU: return launch<tc::EPI_GELU>(g, ntn, s);
        case tc::EPI_RELU: return launch<tc::EPI_RELU>(g, ntn, s);
        case tc::EPI_RESID: return launch<tc::EPI_RESID>(g, ntn, s);
        default: return set_error(NNQS_E_INVAL, "tensor-core layer: bad epilogue");
    }
}

template <>
nnqs_status tc_linear_fwd_ld<double>(cudaStream_t, const TcWeights &, int, int, const double *, int64_t, int64_t,
                                     const double *, double *, int64_t, double *, const double *) {
    return set_error(NNQS_E_UNSUPPORTED, "the tensor-core path computes in BF16/FP32, not FP64");
}

template <class R>
nnqs_status tc_linear_fwd(cudaStream_t s, const TcWeights &w, int slot, int epi, const R *X, int64_t rows, int64_t in,
                          const R *bias, R *Y, R *Y2, const R *resid) {
    return tc_linear_fwd_ld<R>(s, w, slot, epi, X, rows, in, bias, Y, w.rows[slot], Y2, resid);
}
template nnqs_status tc_linear_fwd<float>(cudaStream_t, const TcWeights &, int, int, const float *, int64_t, int64_t,
                                          const float *, float *, float *, const float *);
template nnqs_status tc_linear_fwd<double>(cudaStream_t, const TcWeights &, int, int, const double *, int64_t, int64_t,
                                           const double *, double *, double *, const double *);

}  // namespace nnqs
