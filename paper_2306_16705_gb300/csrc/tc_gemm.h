// Tensor-core (tcgen05) linear layers for NNQS_MIXED, NNQS_BF16X3 and NNQS_FP8:
// BF16 copies of the weight matrices (and their low parts), and
// Y = X W^T + epilogue with FP32 accumulation.
#pragma once
#include "model.h"

namespace nnqs {

struct TcWeights {
    int n_slots = 0;
    bool split = false;            // forward layers with split operands (NNQS_BF16X3)
    void *bf16 = nullptr;          // all weight matrices, BF16, padded
    void *bf16_lo = nullptr;       // low parts W - bf16(W) of the forward copies (same offsets)
    int64_t off[4 * 64 + 1] = {};  // element offset of each slot
    int32_t rows[4 * 64 + 1] = {}, cols[4 * 64 + 1] = {}, prows[4 * 64 + 1] = {}, pcols[4 * 64 + 1] = {};
    int64_t src[4 * 64 + 1] = {};  // offset of the FP32 source matrix in the parameter vector
    int64_t toff[4 * 64 + 1] = {};  // transposed copy W^T [cols][pad(rows)] for input gradients
    int32_t tpcols[4 * 64 + 1] = {};
    // per forward slot, the shared-memory image of every 64-column K block
    // (rows of 128 bytes, 16-byte granules XOR-swizzled by the row), high part
    // at tile_off, low part right after: one bulk copy puts a block in place
    void *tiles = nullptr;
    int64_t tile_off[4 * 64 + 1] = {};
    // NNQS_FP8: E4M3 copies of the forward matrices [N][pad128(K)], each row
    // n scaled by a power of two s_n (its largest entry lands in (224, 448]),
    // and 1 / s_n per row
    bool fp8 = false;
    uint8_t *w8 = nullptr;
    float *w8inv = nullptr;
    int64_t off8[4 * 64 + 1] = {}, soff8[4 * 64 + 1] = {};
    int32_t pcols8[4 * 64 + 1] = {};
    DevStatus *st = nullptr;       // where a timed-out wait is recorded
};

// slot of a weight: layer l, which = 0 qkv, 1 out-proj, 2 FFN-in, 3 FFN-out;
// (L, 0) = phase MLP hidden layer
inline int tc_slot(int layer, int which) { return layer * 4 + which; }

void tc_weights_take(const nnqs_model *M, Arena &a, TcWeights *w = nullptr);
nnqs_status tc_weights_prepare(const nnqs_model *M, const float *params, TcWeights &w, cudaStream_t s);

template <class R>
nnqs_status tc_linear_fwd(cudaStream_t s, const TcWeights &w, int slot, int epi, const R *X, int64_t rows,
                          int64_t in, const R *bias, R *Y, R *Y2, const R *resid);

// as tc_linear_fwd with an explicit output row stride ldy
template <class R>
nnqs_status tc_linear_fwd_ld(cudaStream_t s, const TcWeights &w, int slot, int epi, const R *X, int64_t rows,
                             int64_t in, const R *bias, R *Y, int64_t ldy, R *Y2, const R *resid);
template <>
nnqs_status tc_linear_fwd_ld<float>(cudaStream_t s, const TcWeights &w, int slot, int epi, const float *X,
                                    int64_t rows, int64_t in, const float *bias, float *Y, int64_t ldy, float *Y2,
                                    const float *resid);
template <>
nnqs_status tc_linear_fwd_ld<double>(cudaStream_t s, const TcWeights &w, int slot, int epi, const double *X,
                                     int64_t rows, int64_t in, const double *bias, double *Y, int64_t ldy,
                                     double *Y2, const double *resid);

// dX[rows][in] = dY[rows][out] W[out][in] on tensor cores (W^T copy of `slot`);
// act 1 / 2 multiplies by GELU'(Z) / ReLU'(Z) of the pre-activation Z[rows][in]
// colpart (optional): [ceil(rows/128)][in] column sums of dX per 128-row tile;
// *colpart_done says whether they were written (TMA epilogue only)
nnqs_status tc_linear_dx(cudaStream_t s, const TcWeights &w, int slot, const float *dY, int64_t rows, float *dX,
                         int act = 0, const float *Z = nullptr, float *colpart = nullptr,
                         bool *colpart_done = nullptr);
// dW[out][in] += dY[rows][out]^T X[rows][in] on tensor cores, split over rows;
// partials go to `scratch` (scratch_elems floats) and are added in order
nnqs_status tc_linear_dw(cudaStream_t s, const float *dY, int64_t rows, int64_t out, const float *X, int64_t in,
                         float *dW, float *scratch, size_t scratch_elems, DevStatus *st);

}  // namespace nnqs
