// Fused forward of the transformer amplitude (Sec. 3.1, mask of Sec. 3.3) on
// tcgen05 tensor cores: log|psi| of whole samples with every decoder layer
// of a 128-row tile of token rows kept on chip.
#pragma once
#include <stdint.h>

#include "internal.h"

namespace nnqs {

constexpr int kFusedMaxLayers = 16;

struct FusedFwdArgs {
    const uint64_t *x;  // [n][W] samples
    int64_t n;
    int W, T, L, n_alpha, n_beta;
    int spt;            // samples per 128-row tile: floor(128 / T)
    int64_t n_tiles;
    // FP32 parameters (the caller's layout)
    const float *tok, *pos, *lnf_g, *lnf_b, *hw, *hb;
    const float *ln1g[kFusedMaxLayers], *ln1b[kFusedMaxLayers], *bqkv[kFusedMaxLayers], *bo[kFusedMaxLayers];
    const float *ln2g[kFusedMaxLayers], *ln2b[kFusedMaxLayers], *b1[kFusedMaxLayers], *b2[kFusedMaxLayers];
    // swizzled shared-memory images of the BF16 weights (high part; the low
    // part follows at + rows * K elements): qkv [192 x 64], out-projection
    // [64 x 64], FFN in [256 x 64], FFN out [64 x 256] as four K blocks
    const void *tqkv[kFusedMaxLayers], *to[kFusedMaxLayers], *t1[kFusedMaxLayers], *t2[kFusedMaxLayers];
    double2 *out;       // [n]: .x = log|psi| written (.y untouched)
    // keep mode (hbuf not null): activations for the reverse mode, in the
    // layout of the layer-by-layer forward (row = sample * T + t of this call,
    // rows = n T): hbuf [L+1][rows][64] (input of each layer, then the final
    // residual), hmid [L][rows][64], hf [rows][64], meanf / rstdf [rows],
    // pi [rows][4], tok_out [rows] (the token of each row); with `a` not null
    // also a / a2 / o [L][rows][64], qkv [L][rows][192], u / gu
    // [L][rows][256], mean1 / rstd1 / mean2 / rstd2 [L][rows] and
    // lse [L][n][H][T] (natural units).  The fused reverse mode needs only
    // the first group: it recomputes the rest on chip.
    float *hbuf, *a, *a2, *hmid, *o, *qkv, *u, *gu, *mean1, *rstd1, *mean2, *rstd2, *lse, *hf, *meanf, *rstdf, *pi;
    uint8_t *tok_out;
    int64_t rows;
    DevStatus *st;
    int64_t row_offset; // sample index of x[0] in the caller's numbering (status rows)
};

// d = 64, FFN width 256, head dimension 8 or 16, T <= 64, BF16 (split or not)
bool fused_fwd_supported(int d, int F, int dh, int T, int L);
// every parameter vector and weight image 16-byte aligned (vector loads, bulk copies)
bool fused_fwd_aligned(const FusedFwdArgs &a);
nnqs_status fused_fwd_launch(const FusedFwdArgs &a, bool split, int dh, cudaStream_t s);

}  // namespace nnqs
