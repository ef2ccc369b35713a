// Fused reverse mode of the transformer amplitude's decoder layers (Sec. 3.1;
// the gradient of the energy, Sec. 2.1) on tcgen05 tensor cores: per 128-row
// tile, one layer's forward recomputed on chip from its saved input, the
// input gradient passed on in place, and the weight gradients accumulated in
// TMEM over all of a CTA's tiles (one partial per CTA, added in CTA order).
#pragma once
#include <stdint.h>

#include "internal.h"

namespace nnqs {

// floats of one CTA's partial gradients of a layer's FFN half:
// dW1 [256][64] | dW2 [64][256] | db1 [256] | dgamma2 [64] | dbeta2 [64] | dbo [64]
constexpr int kBwdFfnPart = 256 * 64 + 64 * 256 + 256 + 3 * 64;

// Where the saved rows live: row r of a contiguous [rows][64] array, or (anc
// set) the row of the tree node of token row r = i T + t, node
// anc[t * anc_stride + i], whose rows are node_stride floats apart (the
// sampler's kept activations)
struct BwdRowSource {
    const int32_t *anc;
    int64_t anc_stride, node_stride;
    int T;
};

struct BwdFfnArgs {
    const float *hmid;  // [rows][64] residual after the attention (the input of LN2); with src.anc, node 0's row
    float *dh;          // [rows][64] in: gradient of the layer output; out: gradient of hmid
    int64_t rows;
    BwdRowSource src;   // src.anc null: hmid is contiguous
    const float *ln2g, *ln2b, *b1;  // 16-byte aligned
    // BF16 shared-memory images of the forward: FFN-in W1 [256][64] (high
    // part, low part right after) and FFN-out W2 as four [64][64] K blocks
    const void *t1, *t2;
    float *part;        // [grid][kBwdFfnPart]
    DevStatus *st;
};

// d = 64, FFN width 256
bool bwd_ffn_supported(int d, int F);
// CTAs bwd_ffn_launch uses for `rows` rows (the partials it writes)
int bwd_ffn_grid(int64_t rows);
nnqs_status bwd_ffn_launch(const BwdFfnArgs &a, bool split, cudaStream_t s);
// adds the partials of `grid` CTAs (in CTA order) into the gradients: dw1
// [256][64], dw2 [64][256], db1 [256], dg2 / db2 (LN2 gain / shift) and dbo
// (out-projection bias, the column sums of the gradient of hmid), each [64]
nnqs_status bwd_ffn_reduce(const float *part, int grid, float *dw1, float *dw2, float *db1, float *dg2, float *db2,
                           float *dbo, cudaStream_t s);

// floats of one CTA's partial gradients of a layer's attention half:
// dWqkv [192][64] | dWo [64][64] | dbqkv [192] | dgamma1 [64] | dbeta1 [64] | dsum [64]
constexpr int kBwdAttnPart = 192 * 64 + 64 * 64 + 192 + 3 * 64;

struct BwdAttnArgs {
    const float *hin;   // [rows][64] the layer's input (LN1's input); with src.anc, node 0's row
    float *dh;          // [rows][64] in: gradient of hmid; out: gradient of the layer input
    int64_t n;          // samples; rows = n T
    int T, spt;         // tokens per sample, samples per 128-row tile (floor(128 / T))
    BwdRowSource src;   // src.anc null: hin is contiguous (src.T must equal T when set)
    const float *ln1g, *ln1b, *bqkv;  // 16-byte aligned
    // BF16 shared-memory images of the forward: qkv [192][64] (high part, low
    // part right after) and the out-projection [64][64] (high part)
    const void *tqkv, *to;
    float *part;        // [grid][kBwdAttnPart]
    DevStatus *st;
};

// d = 64, head dimension 8 or 16, T <= 64
bool bwd_attn_supported(int d, int dh, int T);
int bwd_attn_grid(int64_t n, int T);
nnqs_status bwd_attn_launch(const BwdAttnArgs &a, bool split, int dh, cudaStream_t s);
// adds the partials of `grid` CTAs (in CTA order) into dwqkv [192][64], dwo
// [64][64], dbqkv [192], dg1 / db1 (LN1 gain / shift) and, when not null,
// dsum (the column sums of the gradient of the layer input: the previous
// layer's FFN-out bias gradient), each [64]
nnqs_status bwd_attn_reduce(const float *part, int grid, float *dwqkv, float *dwo, float *dbqkv, float *dg1,
                            float *db1, float *dsum, cudaStream_t s);

}  // namespace nnqs
