// Host side of the tcgen05 linear layers used by NNQS_MIXED and NNQS_BF16X3:
// BF16 copies of the weight matrices (K padded to 64 with zeros) and their
// low parts, and the launch of tc::k_tc_gemm.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "dev_common.cuh"
#include "tc_gemm.cuh"
#include "tc_gemm.h"

namespace nnqs {
namespace {

// every conversion of one tc_weights_prepare in one launch: job y is a
// padded copy (with its low part) or a transposed copy of one slot
struct ConvJob {
    int64_t src, rows, cols, pad, dst;  // dst [rows][pad] BF16; source W [N][K] FP32
    int trans;                          // 0: rows = N, cols = K; 1: rows = K, cols = N (dst = W^T)
};
constexpr int kMaxConvJobs = 40;
struct ConvTab {
    int n;
    ConvJob j[kMaxConvJobs];
};

__global__ void k_to_bf16_all(const float *__restrict__ params, ConvTab tab, __nv_bfloat16 *__restrict__ base,
                              __nv_bfloat16 *__restrict__ base_lo) {
    const ConvJob jb = tab.j[blockIdx.y];
    const int64_t total = jb.rows * jb.pad;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / jb.pad, c = i % jb.pad;
        float v = 0.f;
        if (c < jb.cols) v = jb.trans ? params[jb.src + c * jb.rows + r] : params[jb.src + r * jb.cols + c];
        const __nv_bfloat16 hi = __float2bfloat16_rn(v);
        base[jb.dst + i] = hi;
        if (!jb.trans) base_lo[jb.dst + i] = __float2bfloat16_rn(v - __bfloat162float(hi));
    }
}

// dW[i] += sum_z partial[z][i], splits in order
__global__ void k_tc_reduce(const float *__restrict__ partial, int64_t splits, int64_t n, float *__restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float acc = 0.f;
    for (int64_t z = 0; z < splits; ++z) acc += partial[z * n + i];
    out[i] += acc;
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

bool g_attr_set[2][2][tc::kNumEpi] = {};

template <int EPI, bool TRANS = false, bool SPLIT = false>
nnqs_status launch(const tc::Args &g, int64_t n_tiles_n, cudaStream_t s, int64_t splits = 1) {
    constexpr int smem = SPLIT ? tc::kSmemBytesSplit : tc::kSmemBytes;
    if (!g_attr_set[TRANS][SPLIT][EPI]) {
        NNQS_CUDA_TRY(cudaFuncSetAttribute(tc::k_tc_gemm<EPI, TRANS, SPLIT>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        g_attr_set[TRANS][SPLIT][EPI] = true;
    }
    dim3 grid((unsigned)n_tiles_n, (unsigned)((g.M + tc::kTileM - 1) / tc::kTileM), (unsigned)splits);
    NNQS_LAUNCH("k_tc_gemm", s, (tc::k_tc_gemm<EPI, TRANS, SPLIT><<<grid, tc::kThreads, smem, s>>>(g)));
    return NNQS_OK;
}

// N per CTA: the whole N when it fits in 64 columns, else 128-column tiles
// when N is a multiple of 128, else 64-column tiles (epilogue slabs are 64
// columns wide)
int nt_base(int64_t N) {
    if (N <= 64) return (int)((N + 15) / 16 * 16);
    return (N % 128 == 0) ? 128 : 64;
}

// for few row tiles (the sampler's one-token steps) the N tiles are halved
// down to 16 columns until two CTAs per SM are launched: a CTA's epilogue
// then covers fewer columns and the launch finishes sooner
int nt_for(int64_t M, int64_t N) {
    int nt = nt_base(N);
    const int64_t mt = (M + tc::kTileM - 1) / tc::kTileM;
    while (nt > 16 && nt % 32 == 0 && mt * ((N + nt - 1) / nt) < 2 * 152) nt /= 2;
    return nt;
}

int tmem_cols_for(int Nt) {
    int cols = 32;
    while (cols < Nt) cols <<= 1;
    return cols;
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
}

nnqs_status tc_weights_prepare(const nnqs_model *M, const float *params, TcWeights &w, cudaStream_t s) {
    ConvTab tab{};
    auto flush = [&]() -> nnqs_status {
        if (tab.n == 0) return NNQS_OK;
        dim3 grid(64, (unsigned)tab.n);
        NNQS_LAUNCH("k_to_bf16", s,
                    k_to_bf16_all<<<grid, 256, 0, s>>>(params, tab, static_cast<__nv_bfloat16 *>(w.bf16),
                                                       static_cast<__nv_bfloat16 *>(w.bf16_lo)));
        tab.n = 0;
        return NNQS_OK;
    };
    for (int sl = 0; sl < w.n_slots; ++sl) {
        if (sl / 4 == M->L && sl % 4 != 0) continue;
        const int64_t N = w.rows[sl], K = w.cols[sl];
        if (tab.n + 2 > kMaxConvJobs) NNQS_TRY(flush());
        // W [N][K] -> [N][Kpad] (+ low parts); W^T [K][Npad]
        tab.j[tab.n++] = ConvJob{w.src[sl], N, K, w.pcols[sl], w.off[sl], 0};
        tab.j[tab.n++] = ConvJob{w.src[sl], K, N, w.tpcols[sl], w.toff[sl], 1};
    }
    return flush();
}

nnqs_status tc_linear_dx(cudaStream_t s, const TcWeights &w, int slot, const float *dY, int64_t rows, float *dX,
                         int act, const float *Z) {
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
    tc::Args g{};
    g.X = dY;
    g.ldx = out;
    g.Xb = X;
    g.ldb = in;
    g.M = out;
    g.N = in;
    g.K = rows;
    g.Nt = nt_base(g.N);
    g.vec_x = (out % 4 == 0) && (in % 4 == 0) && (reinterpret_cast<uintptr_t>(dY) % 16 == 0) &&
              (reinterpret_cast<uintptr_t>(X) % 16 == 0);
    g.tmem_cols = tmem_cols_for(g.Nt);
    g.st = st;
    const int64_t ntn = (g.N + g.Nt - 1) / g.Nt;
    const int64_t tiles = ((g.M + tc::kTileM - 1) / tc::kTileM) * ntn;
    int64_t splits = std::max<int64_t>(1, (2 * 152 + tiles - 1) / tiles);
    splits = std::min<int64_t>(splits, (rows + tc::kChunkK - 1) / tc::kChunkK);
    splits = std::min<int64_t>(splits, (int64_t)(scratch_elems / size_t(out * in)));
    if (splits < 1) return set_error(NNQS_E_WORKSPACE, "tensor-core weight gradient: scratch too small");
    g.kchunk = ((rows + splits - 1) / splits + tc::kChunkK - 1) / tc::kChunkK * tc::kChunkK;
    splits = (rows + g.kchunk - 1) / g.kchunk;
    g.Y = scratch;
    g.ldy = in;
    note_work("k_tc_gemm", 2.0 * double(rows) * double(in) * double(out),
              4.0 * double(rows) * (out + in) + 4.0 * double(splits) * out * in);
    NNQS_TRY((launch<tc::EPI_STORE, true>(g, ntn, s, splits)));
    NNQS_LAUNCH("k_tc_reduce", s,
                k_tc_reduce<<<grid_for(out * in, 256), 256, 0, s>>>(scratch, splits, out * in, dW));
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
    const int64_t ntn = (g.N + g.Nt - 1) / g.Nt;
    // algorithmic bytes: X in, the BF16 weights (and their low parts), Y out,
    // plus the activation output or the residual read
    const bool two = epi == tc::EPI_GELU || epi == tc::EPI_RELU || epi == tc::EPI_RESID;
    note_work("k_tc_gemm", (w.split ? 6.0 : 2.0) * double(rows) * double(g.N) * double(in),
              4.0 * double(rows) * in + (w.split ? 4.0 : 2.0) * double(g.N) * g.Kpad +
                  (two ? 8.0 : 4.0) * double(rows) * g.N);
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
