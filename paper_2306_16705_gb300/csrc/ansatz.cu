// Ansatz of Sec. 3.1 (transformer amplitude + MLP phase) with the number
// mask of Sec. 3.3: forward log psi and its reverse mode, on CUDA cores,
// templated over the arithmetic type R (double for NNQS_FP64, float for
// NNQS_FP32 and for the non-GEMM parts of NNQS_MIXED).
//
// Layout: activations of a chunk of C samples are row-major [C*T][width]
// (one row per token).  The FP32 parameters are converted once per call to
// R in the workspace.  Samples are processed in chunks so that the saved
// activations of one chunk fit the workspace; weight gradients accumulate
// across chunks in R.
//
// Reductions over samples (weight and bias gradients) run with split-K /
// split-row partial buffers summed in a fixed order: results do not depend
// on scheduling.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <new>

#include "dev_common.cuh"
#include "model.h"
#include "tc_gemm.h"
#include "tc_gemm.cuh"
#include "bwd_fused.cuh"
#include "fwd_fused.cuh"

namespace nnqs {
namespace {

// ------------------------------------------------------------------ math
template <class R>
__device__ __forceinline__ R erf_(R x);
template <>
__device__ __forceinline__ double erf_<double>(double x) { return erf(x); }
template <>
__device__ __forceinline__ float erf_<float>(float x) { return erff(x); }
template <class R>
__device__ __forceinline__ R exp_(R x);
template <>
__device__ __forceinline__ double exp_<double>(double x) { return exp(x); }
template <>
__device__ __forceinline__ float exp_<float>(float x) { return expf(x); }
template <class R>
__device__ __forceinline__ R log_(R x);
template <>
__device__ __forceinline__ double log_<double>(double x) { return log(x); }
template <>
__device__ __forceinline__ float log_<float>(float x) { return logf(x); }

// Units of the attention softmax.  FP64: natural units and exp().  FP32:
// base-2 units -- the scores carry a factor log2 e, folded into the query
// scale -- and the special-function unit's 2^x (ex2.approx.ftz: relative
// error near 2^-22, results below 2^-126 flushed to zero, 2^-inf = 0), one
// instruction where expf takes several.  Every attention kernel (forward,
// cached decode, backward) forms its weights through these, so the cached
// sampler still reproduces the recomputed conditionals bit for bit.  The
// stored log-sum-exp stays in natural units.
template <class R>
struct Softmax;
template <>
struct Softmax<double> {
    static constexpr double kUnit = 1.0;
    __device__ static double pexp(double x) { return exp(x); }
    __device__ static double lse(double m, double l) { return m + log(l); }  // natural, from (max, sum)
    __device__ static double unit_lse(double L) { return L; }                // natural -> score units
};
template <>
struct Softmax<float> {
    static constexpr float kUnit = 1.44269504088896340736f;  // log2 e
    __device__ static float pexp(float x) {
        float y;
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y;
    }
    __device__ static float lse(float m, float l) { return (m + log2f(l)) * 0.69314718055994530942f; }
    __device__ static float unit_lse(float L) { return L * kUnit; }
};
// the query factor 1 / sqrt(DH), in score units
template <class R, int DH>
__device__ __forceinline__ R score_scale() {
    return R(1) / sqrt(R(DH)) * Softmax<R>::kUnit;
}

template <class R>
__device__ __forceinline__ R gelu_(R x) {
    return R(0.5) * x * (R(1) + erf_<R>(x * R(0.70710678118654752440)));
}
template <class R>
__device__ __forceinline__ R gelu_grad_(R x) {
    return R(0.5) * (R(1) + erf_<R>(x * R(0.70710678118654752440))) +
           x * exp_<R>(R(-0.5) * x * x) * R(0.39894228040143267794);
}

template <class R>
__device__ __forceinline__ R neg_inf() {
    return -R(INFINITY);
}

__device__ __forceinline__ int bit_of(const uint64_t *x, int j) { return (int)((x[j >> 6] >> (j & 63)) & 1ull); }

// token at position t of a bitstring: spatial orbital p = T-1-t,
// value y_alpha + 2 y_beta (Sec. 3.3, reverse order)
__device__ __forceinline__ int token_at(const uint64_t *x, int T, int t) {
    const int p = T - 1 - t;
    return bit_of(x, 2 * p) + 2 * bit_of(x, 2 * p + 1);
}

// ------------------------------------------------------------------ small kernels
template <class R>
__global__ void k_convert_params(const float *__restrict__ src, R *__restrict__ dst, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (R)src[i];
}

template <class R>
__global__ void k_fill(R *__restrict__ p, int64_t n, R v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

// h[(i*T+t)*d + c] = tok_emb[inp][c] + pos_emb[t][c]; tok[i*T+t] = token t
// (S = sequence length, <= T; prefixes of length S-1 use S = their length + 1)
template <class R>
__global__ void k_embed(const uint64_t *__restrict__ x, int W, int64_t n, int S, int T, int d,
                        const R *__restrict__ tok_emb, const R *__restrict__ pos_emb, R *__restrict__ h,
                        uint8_t *__restrict__ tok) {
    const int64_t total = n * S * d;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(idx % d);
        const int t = (int)((idx / d) % S);
        const int64_t i = idx / ((int64_t)S * d);
        const uint64_t *xi = x + i * W;
        const int inp = t == 0 ? 4 : token_at(xi, T, t - 1);
        h[idx] = tok_emb[inp * d + c] + pos_emb[t * d + c];
        if (c == 0) tok[i * S + t] = (uint8_t)token_at(xi, T, t);
    }
}

// the same with 16-byte stores (d % 4 == 0): thread = (row, 4 columns), the
// row's input token read once per thread
template <class R>
__global__ void k_embed_v(const uint64_t *__restrict__ x, int W, int64_t n, int S, int T, int d,
                          const R *__restrict__ tok_emb, const R *__restrict__ pos_emb, R *__restrict__ h,
                          uint8_t *__restrict__ tok) {
    const int d4 = d / 4;
    const int64_t total = n * S * d4;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = idx / d4;
        const int c = 4 * (int)(idx - row * d4);
        const int t = (int)(row % S);
        const uint64_t *xi = x + (row / S) * W;
        const int inp = t == 0 ? 4 : token_at(xi, T, t - 1);
        const R *te = tok_emb + inp * d + c, *pe = pos_emb + t * d + c;
        R *hr = h + row * d + c;
        if constexpr (sizeof(R) == 4) {
            const float4 a = *reinterpret_cast<const float4 *>(te), b = *reinterpret_cast<const float4 *>(pe);
            *reinterpret_cast<float4 *>(hr) = make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
        } else {
            hr[0] = te[0] + pe[0];
            hr[1] = te[1] + pe[1];
            hr[2] = te[2] + pe[2];
            hr[3] = te[3] + pe[3];
        }
        if (c == 0) tok[row] = (uint8_t)token_at(xi, T, t);
    }
}

// ------------------------------------------------------------------ LayerNorm
constexpr int kMaxDPerLane = 8;  // d <= 256

template <class R>
__global__ void k_ln_fwd(const R *__restrict__ x, const R *__restrict__ g, const R *__restrict__ b, R *__restrict__ y,
                         R *__restrict__ mean, R *__restrict__ rstd, int64_t rows, int d) {
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= rows) return;
    const R *xr = x + row * d;
    R v[kMaxDPerLane];
    R s = 0;
#pragma unroll
    for (int k = 0; k < kMaxDPerLane; ++k) {
        const int c = lane + 32 * k;
        v[k] = c < d ? xr[c] : R(0);
        s += v[k];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const R mu = s / R(d);
    R q = 0;
#pragma unroll
    for (int k = 0; k < kMaxDPerLane; ++k) {
        const int c = lane + 32 * k;
        const R z = c < d ? v[k] - mu : R(0);
        q += z * z;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    const R rs = R(1) / sqrt(q / R(d) + R(1e-5));
#pragma unroll
    for (int k = 0; k < kMaxDPerLane; ++k) {
        const int c = lane + 32 * k;
        if (c < d) y[row * d + c] = (v[k] - mu) * rs * g[c] + b[c];
    }
    if (lane == 0) {
        if (mean) mean[row] = mu;
        if (rstd) rstd[row] = rs;
    }
}

// dx of LayerNorm, added into acc: acc += rstd (dxh - mean(dxh) - xh mean(dxh xh)), dxh = dy g
template <class R>
__global__ void k_ln_bwd(const R *__restrict__ x, const R *__restrict__ mean, const R *__restrict__ rstd,
                         const R *__restrict__ g, const R *__restrict__ dy, R *__restrict__ acc, int64_t rows, int d) {
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= rows) return;
    const R mu = mean[row], rs = rstd[row];
    R xh[kMaxDPerLane], dxh[kMaxDPerLane];
    R s1 = 0, s2 = 0;
#pragma unroll
    for (int k = 0; k < kMaxDPerLane; ++k) {
        const int c = lane + 32 * k;
        if (c < d) {
            xh[k] = (x[row * d + c] - mu) * rs;
            dxh[k] = dy[row * d + c] * g[c];
        } else {
            xh[k] = dxh[k] = 0;
        }
        s1 += dxh[k];
        s2 += dxh[k] * xh[k];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    s1 /= R(d);
    s2 /= R(d);
#pragma unroll
    for (int k = 0; k < kMaxDPerLane; ++k) {
        const int c = lane + 32 * k;
        if (c < d) acc[row * d + c] += rs * (dxh[k] - s1 - xh[k] * s2);
    }
}

// FP32 rows with d = 4 LPR (LPR a power of two <= 32): LPR lanes per row, one
// float4 per lane, 32/LPR rows per warp and kLnRows such row groups per warp
// with every load issued before the first reduction (the one-row-per-warp
// kernels above leave most of a warp idle and have one load in flight)
constexpr int kLnRows = 4;

// per-lane pieces of the FP32 LayerNorm (one float4 of the row per lane);
// the fused decode layer applies the same pieces in the same tree order
__device__ __forceinline__ float ln_part_sum(float4 v) { return (v.x + v.y) + (v.z + v.w); }
__device__ __forceinline__ float ln_part_sq(float4 v, float mu) {
    const float zx = v.x - mu, zy = v.y - mu, zz = v.z - mu, zw = v.w - mu;
    return (zx * zx + zy * zy) + (zz * zz + zw * zw);
}
__device__ __forceinline__ float ln_rstd(float q, int d) { return 1.0f / sqrtf(q / float(d) + 1e-5f); }
__device__ __forceinline__ float4 ln_apply(float4 v, float mu, float rs, float4 gg, float4 bb) {
    const float zx = v.x - mu, zy = v.y - mu, zz = v.z - mu, zw = v.w - mu;
    return make_float4(zx * rs * gg.x + bb.x, zy * rs * gg.y + bb.y, zz * rs * gg.z + bb.z, zw * rs * gg.w + bb.w);
}

template <int LPR>
__global__ void __launch_bounds__(256) k_ln_fwd_v(const float *__restrict__ x, const float *__restrict__ g,
                                                  const float *__restrict__ b, float *__restrict__ y,
                                                  float *__restrict__ mean, float *__restrict__ rstd, int64_t rows) {
    constexpr int RPW = 32 / LPR, d = 4 * LPR;
    const int lane = threadIdx.x & 31, sub = lane / LPR, l = lane % LPR;
    const int64_t base = ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5) * (RPW * kLnRows);
    float4 v[kLnRows];
#pragma unroll
    for (int u = 0; u < kLnRows; ++u) {
        const int64_t row = base + u * RPW + sub;
        v[u] = row < rows ? __ldg(reinterpret_cast<const float4 *>(x + row * d) + l) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const float4 gg = __ldg(reinterpret_cast<const float4 *>(g) + l), bb = __ldg(reinterpret_cast<const float4 *>(b) + l);
#pragma unroll
    for (int u = 0; u < kLnRows; ++u) {
        const int64_t row = base + u * RPW + sub;
        float s = ln_part_sum(v[u]);
#pragma unroll
        for (int o = LPR / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const float mu = s / float(d);
        float q = ln_part_sq(v[u], mu);
#pragma unroll
        for (int o = LPR / 2; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
        const float rs = ln_rstd(q, d);
        if (row < rows) {
            reinterpret_cast<float4 *>(y + row * d)[l] = ln_apply(v[u], mu, rs, gg, bb);
            if (l == 0) {
                if (mean) mean[row] = mu;
                if (rstd) rstd[row] = rs;
            }
        }
    }
}

template <int LPR>
__global__ void __launch_bounds__(256) k_ln_bwd_v(const float *__restrict__ x, const float *__restrict__ mean,
                                                  const float *__restrict__ rstd, const float *__restrict__ g,
                                                  const float *__restrict__ dy, float *__restrict__ acc, int64_t rows) {
    constexpr int RPW = 32 / LPR, d = 4 * LPR;
    const int lane = threadIdx.x & 31, sub = lane / LPR, l = lane % LPR;
    const int64_t base = ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5) * (RPW * kLnRows);
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 xv[kLnRows], dv[kLnRows], av[kLnRows];
    float mu[kLnRows], rs[kLnRows];
#pragma unroll
    for (int u = 0; u < kLnRows; ++u) {
        const int64_t row = base + u * RPW + sub;
        const bool ok = row < rows;
        xv[u] = ok ? __ldg(reinterpret_cast<const float4 *>(x + row * d) + l) : z4;
        dv[u] = ok ? __ldg(reinterpret_cast<const float4 *>(dy + row * d) + l) : z4;
        av[u] = ok ? reinterpret_cast<const float4 *>(acc + row * d)[l] : z4;
        mu[u] = ok ? mean[row] : 0.f;
        rs[u] = ok ? rstd[row] : 0.f;
    }
    const float4 gg = __ldg(reinterpret_cast<const float4 *>(g) + l);
#pragma unroll
    for (int u = 0; u < kLnRows; ++u) {
        const int64_t row = base + u * RPW + sub;
        const float hx = (xv[u].x - mu[u]) * rs[u], hy = (xv[u].y - mu[u]) * rs[u];
        const float hz = (xv[u].z - mu[u]) * rs[u], hw = (xv[u].w - mu[u]) * rs[u];
        const float ex = dv[u].x * gg.x, ey = dv[u].y * gg.y, ez = dv[u].z * gg.z, ew = dv[u].w * gg.w;
        float s1 = (ex + ey) + (ez + ew);
        float s2 = (ex * hx + ey * hy) + (ez * hz + ew * hw);
#pragma unroll
        for (int o = LPR / 2; o > 0; o >>= 1) {
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        }
        s1 /= float(d);
        s2 /= float(d);
        if (row < rows) {
            const float r = rs[u];
            reinterpret_cast<float4 *>(acc + row * d)[l] =
                make_float4(av[u].x + r * (ex - s1 - hx * s2), av[u].y + r * (ey - s1 - hy * s2),
                            av[u].z + r * (ez - s1 - hz * s2), av[u].w + r * (ew - s1 - hw * s2));
        }
    }
}

inline bool al16(const void *p) { return reinterpret_cast<uintptr_t>(p) % 16 == 0; }

template <class R>
bool ln_vec_ok(int d) {
    return sizeof(R) == 4 && d % 4 == 0 && d >= 4 && d <= 128 && ((d / 4) & (d / 4 - 1)) == 0;
}

template <int LPR>
unsigned ln_blocks(int64_t rows) {
    const int64_t per_block = 8 * (32 / LPR) * kLnRows;  // 8 warps
    return (unsigned)((rows + per_block - 1) / per_block);
}

// y = LayerNorm(x) g + b over rows of d; mean/rstd per row if non-null
template <class R>
nnqs_status ln_fwd(cudaStream_t s, const R *x, const R *g, const R *b, R *y, R *mean, R *rstd, int64_t rows, int d) {
    if (rows == 0) return NNQS_OK;
    if constexpr (sizeof(R) == 4) {
        if (ln_vec_ok<R>(d) && al16(x) && al16(g) && al16(b) && al16(y)) {
            const float *xf = x, *gf = g, *bf = b;
#define NNQS_LNF(LPR) NNQS_LAUNCH("k_ln_fwd", s, (k_ln_fwd_v<LPR><<<ln_blocks<LPR>(rows), 256, 0, s>>>(xf, gf, bf, y, mean, rstd, rows)))
            switch (d / 4) {
                case 1: NNQS_LNF(1); break;
                case 2: NNQS_LNF(2); break;
                case 4: NNQS_LNF(4); break;
                case 8: NNQS_LNF(8); break;
                case 16: NNQS_LNF(16); break;
                default: NNQS_LNF(32); break;
            }
#undef NNQS_LNF
            return NNQS_OK;
        }
    }
    NNQS_LAUNCH("k_ln_fwd", s, k_ln_fwd<R><<<grid_for(rows * 32, 256), 256, 0, s>>>(x, g, b, y, mean, rstd, rows, d));
    return NNQS_OK;
}

// acc += dx of LayerNorm for the output gradient dy
template <class R>
nnqs_status ln_bwd(cudaStream_t s, const R *x, const R *mean, const R *rstd, const R *g, const R *dy, R *acc,
                   int64_t rows, int d) {
    if (rows == 0) return NNQS_OK;
    if constexpr (sizeof(R) == 4) {
        if (ln_vec_ok<R>(d) && al16(x) && al16(g) && al16(dy) && al16(acc)) {
#define NNQS_LNB(LPR) NNQS_LAUNCH("k_ln_bwd", s, (k_ln_bwd_v<LPR><<<ln_blocks<LPR>(rows), 256, 0, s>>>(x, mean, rstd, g, dy, acc, rows)))
            switch (d / 4) {
                case 1: NNQS_LNB(1); break;
                case 2: NNQS_LNB(2); break;
                case 4: NNQS_LNB(4); break;
                case 8: NNQS_LNB(8); break;
                case 16: NNQS_LNB(16); break;
                default: NNQS_LNB(32); break;
            }
#undef NNQS_LNB
            return NNQS_OK;
        }
    }
    NNQS_LAUNCH("k_ln_bwd", s, k_ln_bwd<R><<<grid_for(rows * 32, 256), 256, 0, s>>>(x, mean, rstd, g, dy, acc, rows, d));
    return NNQS_OK;
}

// ------------------------------------------------------------------ column reductions
// Bias and LayerNorm-parameter gradients are column sums over all rows of a
// [rows][cols] activation gradient.  k_colred: each block sums a contiguous
// range of rows (16-byte vector loads, eight rows in flight per thread), the
// row phases of a block are added in a fixed order into partial[blk][.], and
// the last block to finish (counter in global memory, reset by that block)
// adds the partial rows in a fixed order into out[.] (+=).  The result is
// independent of the scheduling order.  Modes:
//   0: out0[c] += sum_r A[r][c]                                  (bias)
//   1: out0[c] += sum_r A[r][c] xh(r, c), out1[c] += sum_r A[r][c]  (LayerNorm
//      gain and bias; xh = (X - mean) rstd)
constexpr int kColThreads = 256;
constexpr int kColUnroll = 8;

template <class R, int VW>
struct ColVec {
    R v[VW];
};

template <class R, int VW>
__device__ __forceinline__ ColVec<R, VW> ld_vec(const R *p) {
    ColVec<R, VW> r;
    if constexpr (VW * sizeof(R) == 16) {
        const uint4 u = __ldg(reinterpret_cast<const uint4 *>(p));
        memcpy(&r, &u, 16);
    } else {
#pragma unroll
        for (int e = 0; e < VW; ++e) r.v[e] = p[e];
    }
    return r;
}

// as ld_vec through L2 only (data written by other blocks of this launch)
template <class R, int VW>
__device__ __forceinline__ ColVec<R, VW> ld_vec_cg(const R *p) {
    ColVec<R, VW> r;
    if constexpr (VW * sizeof(R) == 16) {
        const uint4 u = __ldcg(reinterpret_cast<const uint4 *>(p));
        memcpy(&r, &u, 16);
    } else {
#pragma unroll
        for (int e = 0; e < VW; ++e) r.v[e] = __ldcg(p + e);
    }
    return r;
}

// out[c] += sum_b partial[b * ld + c] for c_lo <= c < c_hi (one block).  A lane takes
// VW consecutive columns, a warp a tile of 32 VW columns; the warps split the
// column tiles and, when there are fewer tiles than warps, the rows b (split
// q takes b = q, q + rs, ...), and the splits are added in order.  Eight rows
// are loaded before they are added.
template <class R, int VW>
__device__ void sum_partial_rows(const R *partial, int64_t nblk, int64_t ld, int c_lo, int c_hi, R *out, R *sh) {
    constexpr int NW = kColThreads / 32, TC = 32 * VW;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_ct = (c_hi - c_lo + TC - 1) / TC;
    const int rs = max(1, NW / n_ct);
    const int tpar = NW / rs;
    for (int t0 = 0; t0 < n_ct; t0 += tpar) {
        const int ti = warp / rs, q = warp % rs, tile = t0 + ti;
        const int c = c_lo + tile * TC + lane * VW;
        R acc[VW];
#pragma unroll
        for (int e = 0; e < VW; ++e) acc[e] = 0;
        if (ti < tpar && tile < n_ct && c < c_hi) {
            int64_t b = q;
            for (; b + 7 * rs < nblk; b += 8 * rs) {
                ColVec<R, VW> v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) v[u] = ld_vec_cg<R, VW>(partial + (b + u * rs) * ld + c);
#pragma unroll
                for (int u = 0; u < 8; ++u)
#pragma unroll
                    for (int e = 0; e < VW; ++e) acc[e] += v[u].v[e];
            }
            for (; b < nblk; b += rs) {
                const ColVec<R, VW> v = ld_vec_cg<R, VW>(partial + b * ld + c);
#pragma unroll
                for (int e = 0; e < VW; ++e) acc[e] += v.v[e];
            }
        }
#pragma unroll
        for (int e = 0; e < VW; ++e) sh[warp * TC + lane * VW + e] = acc[e];
        __syncthreads();
        for (int idx = threadIdx.x; idx < tpar * TC; idx += kColThreads) {
            const int t2 = idx / TC, cc = idx % TC;
            const int col = c_lo + (t0 + t2) * TC + cc;
            if (t0 + t2 < n_ct && col < c_hi) {
                R t = 0;
                for (int k = 0; k < rs; ++k) t += sh[(t2 * rs + k) * TC + cc];
                out[col] += t;
            }
        }
        __syncthreads();
    }
}

template <class R, int MODE, int VW>
__global__ void __launch_bounds__(kColThreads) k_colred(const R *__restrict__ A, const R *__restrict__ X,
                                                        const R *__restrict__ mean, const R *__restrict__ rstd,
                                                        int64_t rows, int cols, int64_t rows_per_block,
                                                        R *__restrict__ partial, unsigned *counter,
                                                        R *__restrict__ out0, R *__restrict__ out1,
                                                        int chunk_cv, int last_reduce) {
    __shared__ R sh[(MODE ? 2 : 1) * kColThreads * VW];
    __shared__ bool last;
    const int tid = threadIdx.x;
    const int64_t r0 = blockIdx.x * rows_per_block;
    const int64_t r1 = min(rows, r0 + rows_per_block);
    const int64_t pcols = (MODE ? 2 : 1) * (int64_t)cols;
    // vector columns of this block: chunk blockIdx.y of chunk_cv
    const int cv_all = cols / VW;
    const int cbeg = blockIdx.y * chunk_cv, cv = min(cv_all, cbeg + chunk_cv);
    const int ct = min(cv - cbeg, kColThreads);  // threads per row within a column tile
    const int phases = kColThreads / ct;         // rows in parallel
    const int p = tid / ct, j = tid % ct;
    for (int v0 = cbeg; v0 < cv; v0 += ct) {
        const int vc = v0 + j;
        const bool act = p < phases && vc < cv;
        R acc[VW], acc2[VW];
#pragma unroll
        for (int e = 0; e < VW; ++e) acc[e] = acc2[e] = 0;
        if (act) {
            int64_t r = r0 + p;
            for (; r + (kColUnroll - 1) * phases < r1; r += kColUnroll * phases) {
                ColVec<R, VW> va[kColUnroll], vx[kColUnroll];
#pragma unroll
                for (int u = 0; u < kColUnroll; ++u) {
                    va[u] = ld_vec<R, VW>(A + (r + u * phases) * cols + vc * VW);
                    if (MODE) vx[u] = ld_vec<R, VW>(X + (r + u * phases) * cols + vc * VW);
                }
#pragma unroll
                for (int u = 0; u < kColUnroll; ++u) {
                    R mu = 0, rs = 0;
                    if (MODE) {
                        mu = mean[r + u * phases];
                        rs = rstd[r + u * phases];
                    }
#pragma unroll
                    for (int e = 0; e < VW; ++e) {
                        if (MODE) acc2[e] += va[u].v[e] * ((vx[u].v[e] - mu) * rs);
                        acc[e] += va[u].v[e];
                    }
                }
            }
            for (; r < r1; r += phases) {
                const ColVec<R, VW> va = ld_vec<R, VW>(A + r * cols + vc * VW);
                ColVec<R, VW> vx;
                R mu = 0, rs = 0;
                if (MODE) {
                    vx = ld_vec<R, VW>(X + r * cols + vc * VW);
                    mu = mean[r];
                    rs = rstd[r];
                }
#pragma unroll
                for (int e = 0; e < VW; ++e) {
                    if (MODE) acc2[e] += va.v[e] * ((vx.v[e] - mu) * rs);
                    acc[e] += va.v[e];
                }
            }
        }
#pragma unroll
        for (int e = 0; e < VW; ++e) {
            sh[tid * VW + e] = acc[e];
            if (MODE) sh[(kColThreads + tid) * VW + e] = acc2[e];
        }
        __syncthreads();
        if (p == 0 && vc < cv) {
#pragma unroll
            for (int e = 0; e < VW; ++e) {
                R t = 0, t2 = 0;
                for (int q = 0; q < phases; ++q) {
                    t += sh[(q * ct + j) * VW + e];
                    if (MODE) t2 += sh[(kColThreads + q * ct + j) * VW + e];
                }
                const int64_t c = (int64_t)vc * VW + e;
                if (MODE) {
                    partial[blockIdx.x * pcols + c] = t2;         // gain part
                    partial[blockIdx.x * pcols + cols + c] = t;   // bias part
                } else {
                    partial[blockIdx.x * pcols + c] = t;
                }
            }
        }
        __syncthreads();
    }
    // last block: add the partial rows of all blocks, in block order (wide
    // rows leave this to k_sum_partials, spread over the columns)
    if (!last_reduce) return;
    __threadfence();
    __syncthreads();
    if (tid == 0) last = atomicAdd(counter, 1u) == gridDim.x * gridDim.y - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    sum_partial_rows<R, VW>(partial, gridDim.x, pcols, 0, cols, out0, sh);
    if (MODE) sum_partial_rows<R, VW>(partial + cols, gridDim.x, pcols, 0, cols, out1, sh);
    if (tid == 0) *counter = 0u;
}

// out[c] += sum_b partial[b][c] for c < cols, partial rows ld apart; block x
// takes columns [32 x, 32 x + 32)
template <class R>
__global__ void __launch_bounds__(kColThreads) k_sum_partials(const R *__restrict__ partial, int64_t nblk,
                                                              int64_t cols, R *__restrict__ out, int64_t ld = -1) {
    __shared__ R sh[kColThreads];
    const int64_t c0 = blockIdx.x * 32;
    sum_partial_rows<R, 1>(partial, nblk, ld < 0 ? cols : ld, (int)c0, (int)min(cols, c0 + 32), out, sh);
}

// ---- LayerNorm backward with its parameter gradients (FP32, d = 4 LPR)
// k_ln_bwd_v's arithmetic per row (acc += dx), and in the same pass the column
// sums the reverse mode needs next: out_g += sum dy xh (gain), out_b += sum dy
// (bias) and, if out_h is given, out_h += sum of the updated acc (the bias
// gradient of the layer whose output gradient acc now is).  Warps walk row
// groups grid-stride, a lane keeps the sums of its 4 columns, and the sums are
// combined in a fixed order: the rows of a warp, the warps of a block, then
// the last block adds the blocks' partial rows in block order.
template <int LPR>
__global__ void __launch_bounds__(256) k_ln_bwd_sums(const float *__restrict__ x, const float *__restrict__ mean,
                                                     const float *__restrict__ rstd, const float *__restrict__ g,
                                                     const float *__restrict__ dy, float *__restrict__ acc,
                                                     int64_t rows, float *__restrict__ partial, unsigned *counter,
                                                     float *__restrict__ out_g, float *__restrict__ out_b,
                                                     float *__restrict__ out_h, bool acc_zero) {
    constexpr int RPW = 32 / LPR, d = 4 * LPR, NW = 8;
    __shared__ float sh[NW * 3 * d > kColThreads * 4 ? NW * 3 * d : kColThreads * 4];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, sub = lane / LPR, l = lane % LPR, warp = threadIdx.x >> 5;
    const int64_t gw = blockIdx.x * (int64_t)NW + warp, GW = (int64_t)gridDim.x * NW;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 gg = __ldg(reinterpret_cast<const float4 *>(g) + l);
    float sg[4] = {0.f, 0.f, 0.f, 0.f}, sb[4] = {0.f, 0.f, 0.f, 0.f}, shh[4] = {0.f, 0.f, 0.f, 0.f};
    for (int64_t base = gw * (RPW * kLnRows); base < rows; base += GW * (RPW * kLnRows)) {
        float4 xv[kLnRows], dv[kLnRows], av[kLnRows];
        float mu[kLnRows], rs[kLnRows];
#pragma unroll
        for (int u = 0; u < kLnRows; ++u) {
            const int64_t row = base + u * RPW + sub;
            const bool ok = row < rows;
            xv[u] = ok ? __ldg(reinterpret_cast<const float4 *>(x + row * d) + l) : z4;
            dv[u] = ok ? __ldg(reinterpret_cast<const float4 *>(dy + row * d) + l) : z4;
            av[u] = ok && !acc_zero ? reinterpret_cast<const float4 *>(acc + row * d)[l] : z4;
            mu[u] = ok ? mean[row] : 0.f;
            rs[u] = ok ? rstd[row] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kLnRows; ++u) {
            const int64_t row = base + u * RPW + sub;
            const float hx = (xv[u].x - mu[u]) * rs[u], hy = (xv[u].y - mu[u]) * rs[u];
            const float hz = (xv[u].z - mu[u]) * rs[u], hw = (xv[u].w - mu[u]) * rs[u];
            const float ex = dv[u].x * gg.x, ey = dv[u].y * gg.y, ez = dv[u].z * gg.z, ew = dv[u].w * gg.w;
            float s1 = (ex + ey) + (ez + ew);
            float s2 = (ex * hx + ey * hy) + (ez * hz + ew * hw);
#pragma unroll
            for (int o = LPR / 2; o > 0; o >>= 1) {
                s1 += __shfl_xor_sync(0xffffffffu, s1, o);
                s2 += __shfl_xor_sync(0xffffffffu, s2, o);
            }
            s1 /= float(d);
            s2 /= float(d);
            if (row < rows) {
                const float r = rs[u];
                const float4 nv = make_float4(av[u].x + r * (ex - s1 - hx * s2), av[u].y + r * (ey - s1 - hy * s2),
                                              av[u].z + r * (ez - s1 - hz * s2), av[u].w + r * (ew - s1 - hw * s2));
                reinterpret_cast<float4 *>(acc + row * d)[l] = nv;
                sg[0] += dv[u].x * hx; sg[1] += dv[u].y * hy; sg[2] += dv[u].z * hz; sg[3] += dv[u].w * hw;
                sb[0] += dv[u].x; sb[1] += dv[u].y; sb[2] += dv[u].z; sb[3] += dv[u].w;
                shh[0] += nv.x; shh[1] += nv.y; shh[2] += nv.z; shh[3] += nv.w;
            }
        }
    }
    // rows of the warp (lanes with the same columns), in sub order
#pragma unroll
    for (int o = LPR; o < 32; o <<= 1)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            sg[e] += __shfl_xor_sync(0xffffffffu, sg[e], o);
            sb[e] += __shfl_xor_sync(0xffffffffu, sb[e], o);
            shh[e] += __shfl_xor_sync(0xffffffffu, shh[e], o);
        }
    if (sub == 0) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            sh[(warp * 3 + 0) * d + 4 * l + e] = sg[e];
            sh[(warp * 3 + 1) * d + 4 * l + e] = sb[e];
            sh[(warp * 3 + 2) * d + 4 * l + e] = shh[e];
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < 3 * d; c += blockDim.x) {
        const int k = c / d, cc = c % d;
        float t = 0.f;
        for (int w = 0; w < NW; ++w) t += sh[(w * 3 + k) * d + cc];
        partial[blockIdx.x * 3 * (int64_t)d + c] = t;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    sum_partial_rows<float, 4>(partial, gridDim.x, 3 * d, 0, d, out_g, sh);
    sum_partial_rows<float, 4>(partial + d, gridDim.x, 3 * d, 0, d, out_b, sh);
    if (out_h) sum_partial_rows<float, 4>(partial + 2 * d, gridDim.x, 3 * d, 0, d, out_h, sh);
    if (threadIdx.x == 0) *counter = 0u;
}

// ------------------------------------------------------------------ GEMM (CUDA cores)
// C[m][n] = sum_k A(m,k) B(n,k), A(m,k) = A[m*sAm + k*sAk], B(n,k) = B[n*sBn + k*sBk],
// then an epilogue.  Tile 64x64x16, 256 threads, 4x4 outputs per thread.
enum Epi { EPI_STORE = 0, EPI_GELU = 1, EPI_RELU = 2, EPI_RESID = 3, EPI_ACCUM = 4 };
constexpr int GM = 64, GN = 64, GK = 16;

template <class R>
struct GemmArgs {
    const R *A;
    int64_t sAm, sAk;
    const R *B;
    int64_t sBn, sBk;
    R *C;
    int64_t ldc;
    R *C2;           // EPI_GELU / EPI_RELU: activation output
    const R *bias;   // [N] or null
    const R *resid;  // EPI_RESID: C = resid + acc + bias
    int64_t M, N, K;
    int64_t kchunk;  // split-K chunk
    R *partial;      // split-K partials [splits][M][N] or null
};

template <class R, int EPI>
__device__ __forceinline__ void epilogue(const GemmArgs<R> &g, int64_t m, int64_t n, R acc) {
    const int64_t o = m * g.ldc + n;
    const R bv = g.bias ? g.bias[n] : R(0);
    if (EPI == EPI_STORE) {
        g.C[o] = acc + bv;
    } else if (EPI == EPI_GELU) {
        const R v = acc + bv;
        g.C[o] = v;
        g.C2[o] = gelu_<R>(v);
    } else if (EPI == EPI_RELU) {
        const R v = acc + bv;
        g.C[o] = v;
        g.C2[o] = v > R(0) ? v : R(0);
    } else if (EPI == EPI_RESID) {
        g.C[o] = g.resid[o] + acc + bv;
    } else {
        g.C[o] += acc;
    }
}

template <class R, int EPI>
__global__ void __launch_bounds__(256) k_gemm(GemmArgs<R> g) {
    __shared__ R As[GK][GM + 1];
    __shared__ R Bs[GK][GN + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t m0 = blockIdx.y * (int64_t)GM, n0 = blockIdx.x * (int64_t)GN;
    const int64_t k_begin = blockIdx.z * g.kchunk;
    const int64_t k_end = min(g.K, k_begin + g.kchunk);
    const bool a_kfast = g.sAk == 1, b_kfast = g.sBk == 1;
    R acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0;
    for (int64_t k0 = k_begin; k0 < k_end; k0 += GK) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int e = threadIdx.x + 256 * r;
            int mm, kk;
            if (a_kfast) {
                kk = e % GK;
                mm = e / GK;
            } else {
                mm = e % GM;
                kk = e / GM;
            }
            const int64_t m = m0 + mm, k = k0 + kk;
            As[kk][mm] = (m < g.M && k < k_end) ? g.A[m * g.sAm + k * g.sAk] : R(0);
            int nn, kb;
            if (b_kfast) {
                kb = e % GK;
                nn = e / GK;
            } else {
                nn = e % GN;
                kb = e / GN;
            }
            const int64_t n = n0 + nn, k2 = k0 + kb;
            Bs[kb][nn] = (n < g.N && k2 < k_end) ? g.B[n * g.sBn + k2 * g.sBk] : R(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            R a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
            if (m >= g.M || n >= g.N) continue;
            if (g.partial)
                g.partial[(blockIdx.z * g.M + m) * g.N + n] = acc[i][j];
            else
                epilogue<R, EPI>(g, m, n, acc[i][j]);
        }
}

template <class R, int EPI>
__global__ void k_gemm_reduce(GemmArgs<R> g, int64_t splits) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= g.M * g.N) return;
    const int64_t m = idx / g.N, n = idx % g.N;
    R s = 0;
    for (int64_t z = 0; z < splits; ++z) s += g.partial[z * g.M * g.N + idx];
    epilogue<R, EPI>(g, m, n, s);
}

int sm_count() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 152;
    }
    return sms;
}

// Scratch for split-K partials and column reductions (elements of R).
template <class R>
struct Scratch {
    R *buf;
    size_t elems;
    unsigned *ctr;  // column-reduction block counter, zero between launches
};

template <class R>
nnqs_status gemm(cudaStream_t s, int epi, const R *A, int64_t sAm, int64_t sAk, const R *B, int64_t sBn, int64_t sBk,
                 R *C, int64_t ldc, R *C2, const R *bias, const R *resid, int64_t M, int64_t N, int64_t K,
                 Scratch<R> scr) {
    if (M == 0 || N == 0) return NNQS_OK;
    GemmArgs<R> g{A, sAm, sAk, B, sBn, sBk, C, ldc, C2, bias, resid, M, N, K, K, nullptr};
    const int64_t tiles = ((M + GM - 1) / GM) * ((N + GN - 1) / GN);
    int64_t splits = 1;
    if (tiles < 2 * sm_count() && K > 4 * GK * 16) {
        splits = std::min<int64_t>((2 * sm_count() + tiles - 1) / tiles, (K + 255) / 256);
        splits = std::min<int64_t>(splits, (int64_t)(scr.elems / size_t(M * N)));
        splits = std::max<int64_t>(splits, 1);
    }
    if (splits > 1) {
        g.kchunk = (((K + splits - 1) / splits) + GK - 1) / GK * GK;
        splits = (K + g.kchunk - 1) / g.kchunk;
        g.partial = scr.buf;
    }
    dim3 grid((unsigned)((N + GN - 1) / GN), (unsigned)((M + GM - 1) / GM), (unsigned)splits);
    note_work("k_gemm", 2.0 * double(M) * double(N) * double(K),
              double(sizeof(R)) * (double(M) * K + double(N) * K + double(M) * N));
#define NNQS_GEMM_CASE(E)                                                                           \
    case E:                                                                                         \
        NNQS_LAUNCH("k_gemm", s, k_gemm<R, E><<<grid, 256, 0, s>>>(g));                             \
        if (splits > 1)                                                                             \
            NNQS_LAUNCH("k_gemm_reduce", s, k_gemm_reduce<R, E><<<grid_for(M * N, 256), 256, 0, s>>>(g, splits)); \
        break;
    switch (epi) {
        NNQS_GEMM_CASE(EPI_STORE)
        NNQS_GEMM_CASE(EPI_GELU)
        NNQS_GEMM_CASE(EPI_RELU)
        NNQS_GEMM_CASE(EPI_RESID)
        NNQS_GEMM_CASE(EPI_ACCUM)
        default: return set_error(NNQS_E_INVAL, "bad GEMM epilogue");
    }
#undef NNQS_GEMM_CASE
    return NNQS_OK;
}

// Y[rows][out] (epilogue) = X[rows][in] W[out][in]^T
template <class R>
nnqs_status linear_fwd(cudaStream_t s, int epi, const R *X, int64_t rows, int64_t in, const R *Wt, int64_t out,
                       const R *bias, R *Y, R *Y2, const R *resid, Scratch<R> scr) {
    return gemm<R>(s, epi, X, in, 1, Wt, in, 1, Y, out, Y2, bias, resid, rows, out, in, scr);
}
// dX[rows][in] (= or +=) dY[rows][out] W[out][in]
template <class R>
nnqs_status linear_dx(cudaStream_t s, int epi, const R *dY, int64_t rows, int64_t out, const R *Wt, int64_t in, R *dX,
                      Scratch<R> scr) {
    return gemm<R>(s, epi, dY, out, 1, Wt, 1, in, dX, in, nullptr, nullptr, nullptr, rows, in, out, scr);
}
// dW[out][in] += dY[rows][out]^T X[rows][in]
template <class R>
nnqs_status linear_dw(cudaStream_t s, const R *dY, int64_t rows, int64_t out, const R *X, int64_t in, R *dW,
                      Scratch<R> scr) {
    return gemm<R>(s, EPI_ACCUM, dY, 1, out, X, 1, in, dW, in, nullptr, nullptr, nullptr, out, in, rows, scr);
}

template <class R>
nnqs_status act_bwd(cudaStream_t s, int act, R *dX, const R *Z, int64_t n);

// backward GEMMs of the weights that have BF16 copies: tensor cores for
// NNQS_MIXED (tcw != null, FP32 activations), CUDA cores otherwise.
// act 1 / 2: dX is then multiplied by GELU'(Z) / ReLU'(Z) (in the tensor-core
// epilogue, or by a separate pass)
template <class R>
nnqs_status bw_dx(cudaStream_t s, const TcWeights *tcw, int slot, const R *dY, int64_t rows, int64_t out, const R *Wt,
                  int64_t in, R *dX, Scratch<R> scr, int act = 0, const R *Z = nullptr, R *colpart = nullptr,
                  bool *colpart_done = nullptr) {
    if (colpart_done) *colpart_done = false;
    NNQS_TRY(linear_dx<R>(s, EPI_STORE, dY, rows, out, Wt, in, dX, scr));
    return act_bwd<R>(s, act, dX, Z, rows * in);
}
template <>
nnqs_status bw_dx<float>(cudaStream_t s, const TcWeights *tcw, int slot, const float *dY, int64_t rows, int64_t out,
                         const float *Wt, int64_t in, float *dX, Scratch<float> scr, int act, const float *Z,
                         float *colpart, bool *colpart_done) {
    if (colpart_done) *colpart_done = false;
    if (tcw) return tc_linear_dx(s, *tcw, slot, dY, rows, dX, act, Z, colpart, colpart_done);
    NNQS_TRY(linear_dx<float>(s, EPI_STORE, dY, rows, out, Wt, in, dX, scr));
    return act_bwd<float>(s, act, dX, Z, rows * in);
}
template <class R>
nnqs_status bw_dw(cudaStream_t s, const TcWeights *tcw, const R *dY, int64_t rows, int64_t out, const R *X,
                  int64_t in, R *dW, Scratch<R> scr) {
    return linear_dw<R>(s, dY, rows, out, X, in, dW, scr);
}
template <>
nnqs_status bw_dw<float>(cudaStream_t s, const TcWeights *tcw, const float *dY, int64_t rows, int64_t out,
                         const float *X, int64_t in, float *dW, Scratch<float> scr) {
    if (tcw) return tc_linear_dw(s, dY, rows, out, X, in, dW, scr.buf, scr.elems, tcw->st);
    return linear_dw<float>(s, dY, rows, out, X, in, dW, scr);
}

// column sums of a [rows][cols] gradient into out0 (+=); mode 1 also the
// LayerNorm gain gradient: out0 += sum A xh, out1 += sum A
template <class R>
nnqs_status colsum(cudaStream_t s, int mode, const R *A, const R *X, const R *mean, const R *rstd, int64_t rows,
                   int cols, R *out0, R *out1, Scratch<R> scr) {
    if (rows == 0) return NNQS_OK;
    constexpr int V = int(16 / sizeof(R));
    const bool vec = cols % V == 0 && reinterpret_cast<uintptr_t>(A) % 16 == 0 &&
                     (mode == 0 || reinterpret_cast<uintptr_t>(X) % 16 == 0);
    const int64_t pc = (mode ? 2 : 1) * (int64_t)cols;
    // wide rows (more than 64 vector columns): 32-vector-column chunks over
    // blockIdx.y (8 rows in flight per block instead of one or two), the
    // partial rows then added column-parallel by k_sum_partials
    const int vw = vec ? V : 1;
    const int cv = cols / vw;
    const bool wide = cv > 64;
    const int chunk_cv = wide ? 32 : cv;
    const int64_t n_chunks = (cv + chunk_cv - 1) / chunk_cv;
    int64_t nblk = wide ? std::min<int64_t>((rows + 63) / 64, (8 * sm_count() + n_chunks - 1) / n_chunks)
                        : std::min<int64_t>((rows + 63) / 64, 2 * sm_count());
    nblk = std::min<int64_t>(nblk, (int64_t)(scr.elems / size_t(pc)));
    nblk = std::max<int64_t>(nblk, 1);
    const int64_t rpb = (rows + nblk - 1) / nblk;
    nblk = (rows + rpb - 1) / rpb;
    const dim3 g((unsigned)nblk, (unsigned)n_chunks);
    const int lr = wide ? 0 : 1;
    if (mode == 0 && vec)
        NNQS_LAUNCH("k_colred", s, (k_colred<R, 0, V><<<g, kColThreads, 0, s>>>(A, X, mean, rstd, rows, cols, rpb, scr.buf, scr.ctr, out0, out1, chunk_cv, lr)));
    else if (mode == 0)
        NNQS_LAUNCH("k_colred", s, (k_colred<R, 0, 1><<<g, kColThreads, 0, s>>>(A, X, mean, rstd, rows, cols, rpb, scr.buf, scr.ctr, out0, out1, chunk_cv, lr)));
    else if (vec)
        NNQS_LAUNCH("k_colred", s, (k_colred<R, 1, V><<<g, kColThreads, 0, s>>>(A, X, mean, rstd, rows, cols, rpb, scr.buf, scr.ctr, out0, out1, chunk_cv, lr)));
    else
        NNQS_LAUNCH("k_colred", s, (k_colred<R, 1, 1><<<g, kColThreads, 0, s>>>(A, X, mean, rstd, rows, cols, rpb, scr.buf, scr.ctr, out0, out1, chunk_cv, lr)));
    if (wide) {
        NNQS_LAUNCH("k_colred", s, (k_sum_partials<R><<<(unsigned)((cols + 31) / 32), kColThreads, 0, s>>>(scr.buf, nblk, cols, out0, pc)));
        if (mode)
            NNQS_LAUNCH("k_colred", s, (k_sum_partials<R><<<(unsigned)((cols + 31) / 32), kColThreads, 0, s>>>(scr.buf + cols, nblk, cols, out1, pc)));
    }
    return NNQS_OK;
}

// LayerNorm backward (acc += dx) with its gain and bias gradients (out_g,
// out_b) and, when out_h is given, the column sums of the updated acc: one
// pass for FP32 rows of d = 4 LPR, else the separate kernels
template <class R>
nnqs_status ln_bwd_sums(cudaStream_t s, const R *x, const R *mean, const R *rstd, const R *g, const R *dy, R *acc,
                        int64_t rows, int d, R *out_g, R *out_b, R *out_h, Scratch<R> scr, bool acc_zero = false) {
    if (rows == 0) return NNQS_OK;
    if constexpr (sizeof(R) == 4) {
        if (ln_vec_ok<R>(d) && al16(x) && al16(g) && al16(dy) && al16(acc) && d >= 4) {
            const int lpr = d / 4;
            const int64_t per_block = 8 * (32 / lpr) * kLnRows;
            int64_t nblk = std::min<int64_t>((rows + per_block - 1) / per_block, 2 * sm_count());
            nblk = std::max<int64_t>(1, std::min<int64_t>(nblk, (int64_t)(scr.elems / size_t(3 * d))));
#define NNQS_LNS(LPR) NNQS_LAUNCH("k_ln_bwd", s, (k_ln_bwd_sums<LPR><<<(unsigned)nblk, 256, 0, s>>>(x, mean, rstd, g, dy, acc, rows, scr.buf, scr.ctr, out_g, out_b, out_h, acc_zero)))
            switch (lpr) {
                case 1: NNQS_LNS(1); break;
                case 2: NNQS_LNS(2); break;
                case 4: NNQS_LNS(4); break;
                case 8: NNQS_LNS(8); break;
                case 16: NNQS_LNS(16); break;
                default: NNQS_LNS(32); break;
            }
#undef NNQS_LNS
            return NNQS_OK;
        }
    }
    if (acc_zero) NNQS_LAUNCH("k_fill", s, k_fill<R><<<grid_for(rows * d, 256), 256, 0, s>>>(acc, rows * d, R(0)));
    NNQS_TRY(ln_bwd<R>(s, x, mean, rstd, g, dy, acc, rows, d));
    NNQS_TRY(colsum<R>(s, 1, dy, x, mean, rstd, rows, d, out_g, out_b, scr));
    if (out_h) NNQS_TRY(colsum<R>(s, 0, acc, nullptr, nullptr, nullptr, rows, d, out_h, nullptr, scr));
    return NNQS_OK;
}

// ------------------------------------------------------------------ attention
// One thread per (sample, head, query): causal softmax(q k^T / sqrt(dh)) v
// with an online max/sum; also writes the log-sum-exp for the backward.
template <class R, int DH>
__global__ void k_attn_fwd(const R *__restrict__ qkv, R *__restrict__ o, R *__restrict__ lse, int64_t n, int T, int H,
                           int d) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n * H * T) return;
    const int q = (int)(idx % T);
    const int hh = (int)((idx / T) % H);
    const int64_t i = idx / ((int64_t)T * H);
    const R scale = score_scale<R, DH>();
    const R *base = qkv + i * T * 3 * d;
    R qv[DH], acc[DH];
#pragma unroll
    for (int c = 0; c < DH; ++c) {
        qv[c] = base[q * 3 * d + hh * DH + c] * scale;
        acc[c] = 0;
    }
    R m = neg_inf<R>(), l = 0;
    for (int j = 0; j <= q; ++j) {
        const R *kj = base + j * 3 * d + d + hh * DH;
        const R *vj = base + j * 3 * d + 2 * d + hh * DH;
        R sc = 0;
#pragma unroll
        for (int c = 0; c < DH; ++c) sc += qv[c] * kj[c];
        const R mn = sc > m ? sc : m;
        const R corr = Softmax<R>::pexp(m - mn);
        const R p = Softmax<R>::pexp(sc - mn);
        l = l * corr + p;
#pragma unroll
        for (int c = 0; c < DH; ++c) acc[c] = acc[c] * corr + p * vj[c];
        m = mn;
    }
    const R inv = R(1) / l;
#pragma unroll
    for (int c = 0; c < DH; ++c) o[(i * T + q) * d + hh * DH + c] = acc[c] * inv;
    lse[idx] = Softmax<R>::lse(m, l);
}

// dq for each query: dq = scale sum_j p_ij (dp_ij - D_i) k_j, dp_ij = do_i . v_j,
// D_i = do_i . o_i
template <class R, int DH>
__global__ void k_attn_bwd_q(const R *__restrict__ qkv, const R *__restrict__ o, const R *__restrict__ lse,
                             const R *__restrict__ dout, R *__restrict__ dqkv, R *__restrict__ Dbuf, int64_t n, int T,
                             int H, int d) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n * H * T) return;
    const int q = (int)(idx % T);
    const int hh = (int)((idx / T) % H);
    const int64_t i = idx / ((int64_t)T * H);
    const R scale = R(1) / sqrt(R(DH)), qs = score_scale<R, DH>();
    const R *base = qkv + i * T * 3 * d;
    R qv[DH], dov[DH], dq[DH];
    R D = 0;
#pragma unroll
    for (int c = 0; c < DH; ++c) {
        qv[c] = base[q * 3 * d + hh * DH + c] * qs;
        dov[c] = dout[(i * T + q) * d + hh * DH + c];
        D += dov[c] * o[(i * T + q) * d + hh * DH + c];
        dq[c] = 0;
    }
    Dbuf[idx] = D;
    const R L = Softmax<R>::unit_lse(lse[idx]);
    for (int j = 0; j <= q; ++j) {
        const R *kj = base + j * 3 * d + d + hh * DH;
        const R *vj = base + j * 3 * d + 2 * d + hh * DH;
        R sc = 0, dp = 0;
#pragma unroll
        for (int c = 0; c < DH; ++c) {
            sc += qv[c] * kj[c];
            dp += dov[c] * vj[c];
        }
        const R ds = Softmax<R>::pexp(sc - L) * (dp - D);
#pragma unroll
        for (int c = 0; c < DH; ++c) dq[c] += ds * kj[c];
    }
#pragma unroll
    for (int c = 0; c < DH; ++c) dqkv[(i * T + q) * 3 * d + hh * DH + c] = dq[c] * scale;
}

// dk, dv for each key j: dv = sum_{i>=j} p_ij do_i, dk = scale sum_{i>=j} p_ij (dp_ij - D_i) q_i
template <class R, int DH>
__global__ void k_attn_bwd_kv(const R *__restrict__ qkv, const R *__restrict__ lse, const R *__restrict__ dout,
                              const R *__restrict__ Dbuf, R *__restrict__ dqkv, int64_t n, int T, int H, int d) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n * H * T) return;
    const int j = (int)(idx % T);
    const int hh = (int)((idx / T) % H);
    const int64_t i = idx / ((int64_t)T * H);
    const R scale = R(1) / sqrt(R(DH)), qs = score_scale<R, DH>();
    const R *base = qkv + i * T * 3 * d;
    R kv[DH], vv[DH], dk[DH], dv[DH];
#pragma unroll
    for (int c = 0; c < DH; ++c) {
        kv[c] = base[j * 3 * d + d + hh * DH + c];
        vv[c] = base[j * 3 * d + 2 * d + hh * DH + c];
        dk[c] = dv[c] = 0;
    }
    const int64_t row0 = (i * H + hh) * T;
    for (int q = j; q < T; ++q) {
        const R *qq = base + q * 3 * d + hh * DH;
        const R *dq = dout + (i * T + q) * d + hh * DH;
        R sc = 0, dp = 0;
#pragma unroll
        for (int c = 0; c < DH; ++c) {
            sc += qq[c] * kv[c];
            dp += dq[c] * vv[c];
        }
        const R p = Softmax<R>::pexp(sc * qs - Softmax<R>::unit_lse(lse[row0 + q]));
        const R ds = p * (dp - Dbuf[row0 + q]);
#pragma unroll
        for (int c = 0; c < DH; ++c) {
            dv[c] += p * dq[c];
            dk[c] += ds * qq[c];
        }
    }
#pragma unroll
    for (int c = 0; c < DH; ++c) {
        dqkv[(i * T + j) * 3 * d + d + hh * DH + c] = dk[c] * scale;
        dqkv[(i * T + j) * 3 * d + 2 * d + hh * DH + c] = dv[c];
    }
}

// Shared-memory attention: one CTA per sample, the sample's q|k|v rows
// staged once (padded rows, conflict-free column reads), one thread per
// (head, position).  Used whenever a sample's rows fit in shared memory.
// Column c of a staged input row sits at shared column swz_col<R, NC>(c):
// the 16-byte pieces of a head (NC of them, NC a power of two <= 8) are
// XOR-rotated by the index of the 128-byte bank row they start in, so that
// the threads of a warp reading piece k of every head of one row (the
// attention loops: all lanes on the same key row) hit distinct banks.  With
// heads of 32 bytes (8 FP32) and no rotation, heads h and h + 4 share banks
// and every such read takes two wavefronts.  NC = 1: no rotation.
template <class R, int NC>
__device__ __forceinline__ int swz_col(int c) {
    constexpr int V = int(16 / sizeof(R));
    if constexpr (NC <= 1) {
        return c;
    } else {
        const int p = c / V;
        return (p ^ ((p >> 3) & (NC - 1))) * V + (c - p * V);
    }
}

// copies between a contiguous [T][w] block in global memory and shared rows
// of stride ld (padded against bank conflicts): 16-byte global accesses when
// w and the pointer allow, the (row, column) of a thread advanced by adds;
// columns placed by swz_col<R, NC>
template <class R, int NC = 1>
__device__ __forceinline__ void rows_to_smem(R *dst, int ld, const R *__restrict__ src, int T, int w) {
    constexpr int V = int(16 / sizeof(R));
    if (w % V == 0 && reinterpret_cast<uintptr_t>(src) % 16 == 0) {
        const int wv = w / V, nt = blockDim.x;
        const int sr = nt / wv, sc = nt % wv;
        int r = threadIdx.x / wv, c = threadIdx.x % wv;
        while (r < T) {
            const ColVec<R, V> v = ld_vec<R, V>(src + (int64_t)r * w + c * V);
            const int cs = swz_col<R, NC>(c * V);
#pragma unroll
            for (int e = 0; e < V; ++e) dst[r * ld + cs + e] = v.v[e];
            r += sr;
            c += sc;
            if (c >= wv) {
                c -= wv;
                ++r;
            }
        }
    } else {
        for (int e = threadIdx.x; e < T * w; e += blockDim.x) dst[(e / w) * ld + swz_col<R, NC>(e % w)] = src[e];
    }
}

template <class R>
__device__ __forceinline__ void smem_to_rows(R *__restrict__ dst, const R *src, int ld, int T, int w) {
    constexpr int V = int(16 / sizeof(R));
    if (w % V == 0 && reinterpret_cast<uintptr_t>(dst) % 16 == 0) {
        const int wv = w / V, nt = blockDim.x;
        const int sr = nt / wv, sc = nt % wv;
        int r = threadIdx.x / wv, c = threadIdx.x % wv;
        const bool vec = ld % V == 0;  // 16-byte shared rows
        while (r < T) {
            ColVec<R, V> v;
            if (vec) {
                const uint4 u = *reinterpret_cast<const uint4 *>(src + r * ld + c * V);
                memcpy(&v, &u, 16);
            } else {
#pragma unroll
                for (int e = 0; e < V; ++e) v.v[e] = src[r * ld + c * V + e];
            }
            *reinterpret_cast<ColVec<R, V> *>(dst + (int64_t)r * w + c * V) = v;
            r += sr;
            c += sc;
            if (c >= wv) {
                c -= wv;
                ++r;
            }
        }
    } else {
        for (int e = threadIdx.x; e < T * w; e += blockDim.x) dst[e] = src[(e / w) * ld + e % w];
    }
}

// rows_to_smem with every load of a thread issued before its shared stores
// (one memory round trip per block instead of one per 16-byte piece): up to
// MAXV 16-byte pieces per thread, for w a multiple of the vector width, a
// 16-byte aligned source and T * w / V <= MAXV * blockDim.x (the caller
// checks with fits())
template <class R, int MAXV>
struct RowBatch {
    static constexpr int V = int(16 / sizeof(R));
    ColVec<R, V> v[MAXV];
    __device__ static bool fits(const R *src, int T, int w) {
        return w % V == 0 && reinterpret_cast<uintptr_t>(src) % 16 == 0 && T * (w / V) <= MAXV * (int)blockDim.x;
    }
    __device__ __forceinline__ void load(const R *__restrict__ src, int T, int w) {
        const int total = T * (w / V);
#pragma unroll
        for (int k = 0; k < MAXV; ++k) {
            const int e = threadIdx.x + k * blockDim.x;
            if (e < total) v[k] = ld_vec<R, V>(src + (int64_t)e * V);
        }
    }
    // columns placed by swz_col<R, NC>
    template <int NC = 1>
    __device__ __forceinline__ void store(R *dst, int ld, int T, int w) const {
        const int wv = w / V, total = T * wv;
        const bool vec = ld % V == 0;  // 16-byte shared rows
#pragma unroll
        for (int k = 0; k < MAXV; ++k) {
            const int e = threadIdx.x + k * blockDim.x;
            if (e < total) {
                const int r = e / wv, c = swz_col<R, NC>((e - r * wv) * V);
                if (vec) {
                    uint4 u;
                    memcpy(&u, &v[k], 16);
                    *reinterpret_cast<uint4 *>(dst + r * ld + c) = u;
                } else {
#pragma unroll
                    for (int q = 0; q < V; ++q) dst[r * ld + c + q] = v[k].v[q];
                }
            }
        }
    }
};

// Head groups: a sample whose whole attention state does not fit one CTA's
// shared memory is split over gridDim.y CTAs, CTA g taking heads
// [g Hg, (g + 1) Hg) (columns [g dg, (g + 1) dg) of every d-wide segment).
// seg_rows_to_smem gathers a [T][nseg dfull] block's nseg segments, columns
// off .. off + dg - 1 of each, into staged rows [seg 0 | seg 1 | ...] of
// width nseg dg (columns placed by swz_col<R, NC>); smem_to_seg_rows writes
// staged rows back the same way (unrotated).  Both need 16-byte aligned
// rows and dg, dfull, off multiples of the vector width.
template <class R, int NC>
__device__ __forceinline__ void seg_rows_to_smem(R *dst, int ld, const R *__restrict__ src, int T, int nseg,
                                                 int dfull, int off, int dg) {
    constexpr int V = int(16 / sizeof(R));
    const int pv = dg / V, per_row = nseg * pv;
    for (int e = threadIdx.x; e < T * per_row; e += blockDim.x) {
        const int r = e / per_row, q = e - r * per_row, sg = q / pv, c = (q - sg * pv) * V;
        const ColVec<R, V> v = ld_vec<R, V>(src + ((int64_t)r * nseg + sg) * dfull + off + c);
        const int cs = swz_col<R, NC>(sg * dg + c);
#pragma unroll
        for (int k = 0; k < V; ++k) dst[r * ld + cs + k] = v.v[k];
    }
}

template <class R>
__device__ __forceinline__ void smem_to_seg_rows(R *__restrict__ dst, const R *src, int ld, int T, int nseg, int dfull,
                                                 int off, int dg) {
    constexpr int V = int(16 / sizeof(R));
    const int pv = dg / V, per_row = nseg * pv;
    for (int e = threadIdx.x; e < T * per_row; e += blockDim.x) {
        const int r = e / per_row, q = e - r * per_row, sg = q / pv, c = (q - sg * pv) * V;
        ColVec<R, V> v;
#pragma unroll
        for (int k = 0; k < V; ++k) v.v[k] = src[r * ld + sg * dg + c + k];
        *reinterpret_cast<ColVec<R, V> *>(dst + ((int64_t)r * nseg + sg) * dfull + off + c) = v;
    }
}

// 16-byte pieces per thread of a sample's q|k|v rows (3 d = 3 H DH columns,
// at least H T threads): 3 DH / V, capped
template <class R, int DH>
constexpr int qkv_pieces() {
    constexpr int n = (3 * DH * int(sizeof(R)) + 15) / 16;
    return n < 1 ? 1 : (n > 12 ? 12 : n);
}
template <class R, int DH>
constexpr int row_pieces() {
    constexpr int n = (DH * int(sizeof(R)) + 15) / 16;
    return n < 1 ? 1 : (n > 4 ? 4 : n);
}

// DH consecutive values of one head from shared memory: 16-byte reads when
// DH is a multiple of the vector width and the rows are unpadded (kVec),
// else scalar reads (padded rows)
template <class R, int DH>
struct HeadVec {
    static constexpr int V = int(16 / sizeof(R));
    static constexpr bool kVec = DH % V == 0;
    // pieces per head rotated in staged input rows (swz_col); 1 = none
    static constexpr int kNC = (kVec && DH / V <= 8) ? DH / V : 1;
    // head values at column col (a multiple of DH) of a staged input row
    // (placed by swz_col<R, kNC>): piece k from column swz_col(col + k V)
    __device__ __forceinline__ static void read_in(const R *row, int col, R (&out)[DH]) {
        if constexpr (kVec && kNC > 1) {
            const int p0 = col / V, sx = (p0 >> 3) & (kNC - 1);
#pragma unroll
            for (int k = 0; k < kNC; ++k) {
                const uint4 u = *reinterpret_cast<const uint4 *>(row + (p0 + (k ^ sx)) * V);
                R tmp[V];
                memcpy(tmp, &u, 16);
#pragma unroll
                for (int e = 0; e < V; ++e) out[k * V + e] = tmp[e];
            }
        } else {
            read(row + col, out);
        }
    }
    __device__ __forceinline__ static void read(const R *p, R (&out)[DH]) {
        if constexpr (kVec) {
#pragma unroll
            for (int c = 0; c < DH; c += V) {
                const uint4 u = *reinterpret_cast<const uint4 *>(p + c);
                R tmp[V];
                memcpy(tmp, &u, 16);
#pragma unroll
                for (int e = 0; e < V; ++e) out[c + e] = tmp[e];
            }
        } else {
#pragma unroll
            for (int c = 0; c < DH; ++c) out[c] = p[c];
        }
    }
    __device__ __forceinline__ static void write(R *p, const R (&in)[DH]) {
        if constexpr (kVec) {
#pragma unroll
            for (int c = 0; c < DH; c += V) {
                uint4 u;
                memcpy(&u, in + c, 16);
                *reinterpret_cast<uint4 *>(p + c) = u;
            }
        } else {
#pragma unroll
            for (int c = 0; c < DH; ++c) p[c] = in[c];
        }
    }
    // row stride in shared memory for w columns, padded so that consecutive
    // rows start 4 banks apart: 16 bytes (rows stay 16-byte aligned) for
    // vector reads, one element for scalar ones
    __host__ __device__ static constexpr int ld(int w) { return kVec ? w + V : w + 1; }
};

template <class R, int DH>
__global__ void k_attn_fwd_smem(const R *__restrict__ qkv, R *__restrict__ o, R *__restrict__ lse, int T, int H,
                                int d) {
    using HV = HeadVec<R, DH>;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    R *sq = reinterpret_cast<R *>(sm_raw);  // [T][ldq]
    const int ldq = HV::ld(3 * d), ldo = HV::ld(d);
    R *so = sq + T * ldq;                    // [T][ldo]
    const int64_t i = blockIdx.x;
    const int tid = threadIdx.x;
    const R *src = qkv + i * T * 3 * d;
    {
        RowBatch<R, qkv_pieces<R, DH>()> b;
        if (b.fits(src, T, 3 * d)) {
            b.load(src, T, 3 * d);
            b.template store<HV::kNC>(sq, ldq, T, 3 * d);
        } else {
            rows_to_smem<R, HV::kNC>(sq, ldq, src, T, 3 * d);
        }
    }
    __syncthreads();
    if (tid < H * T) {
        const int hh = tid % H, q = tid / H;  // heads fastest: a warp holds a few positions (even loop trips)
        const R scale = score_scale<R, DH>();
        R qv[DH], acc[DH];
        HV::read_in(sq + q * ldq, hh * DH, qv);
#pragma unroll
        for (int c = 0; c < DH; ++c) {
            qv[c] = qv[c] * scale;
            acc[c] = 0;
        }
        R m = neg_inf<R>(), l = 0;
#pragma unroll 2
        for (int j = 0; j <= q; ++j) {
            R kj[DH], vj[DH];
            HV::read_in(sq + j * ldq, d + hh * DH, kj);
            HV::read_in(sq + j * ldq, 2 * d + hh * DH, vj);
            R sc = 0;
#pragma unroll
            for (int c = 0; c < DH; ++c) sc += qv[c] * kj[c];
            const R mn = sc > m ? sc : m;
            const R corr = Softmax<R>::pexp(m - mn);
            const R p = Softmax<R>::pexp(sc - mn);
            l = l * corr + p;
#pragma unroll
            for (int c = 0; c < DH; ++c) acc[c] = acc[c] * corr + p * vj[c];
            m = mn;
        }
        const R inv = R(1) / l;
#pragma unroll
        for (int c = 0; c < DH; ++c) acc[c] = acc[c] * inv;
        HV::write(so + q * ldo + hh * DH, acc);
        lse[(i * H + hh) * T + q] = Softmax<R>::lse(m, l);
    }
    __syncthreads();
    R *dst = o + i * T * d;
    smem_to_rows<R>(dst, so, ldo, T, d);
}

// colsum (optional): [n][3d] column sums of the sample's dq|dk|dv over its
// T positions (added in position order), for the qkv bias gradient
// With head groups (gridDim.y > 1): H and d are the group's heads and width,
// Hfull and dfull the model's; blockIdx.y is the group.
template <class R, int DH>
__global__ void k_attn_bwd_smem(const R *__restrict__ qkv, const R *__restrict__ o, const R *__restrict__ lse,
                                const R *__restrict__ dout, R *__restrict__ dqkv, int T, int H, int d,
                                R *__restrict__ colsum, int Hfull, int dfull) {
    using HV = HeadVec<R, DH>;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int ldq = HV::ld(3 * d), ldo = HV::ld(d);
    R *sq = reinterpret_cast<R *>(sm_raw);  // q|k|v [T][ldq]
    R *sg = sq + T * ldq;                    // dq|dk|dv [T][ldq]
    R *sdo = sg + T * ldq;                   // dout [T][ldo]
    R *so = sdo + T * ldo;                   // o [T][ldo]
    R *slse = so + T * ldo;                  // [H][T]
    R *sD = slse + H * T;                    // [H][T]
    const int64_t i = blockIdx.x;
    const int tid = threadIdx.x, nt = blockDim.x;
    const bool grouped = gridDim.y > 1;
    const int goff = blockIdx.y * d;  // first column of this group within a segment
    if (grouped) {
        seg_rows_to_smem<R, HV::kNC>(sq, ldq, qkv + i * T * 3 * dfull, T, 3, dfull, goff, d);
        seg_rows_to_smem<R, HV::kNC>(sdo, ldo, dout + i * T * dfull, T, 1, dfull, goff, d);
        seg_rows_to_smem<R, HV::kNC>(so, ldo, o + i * T * dfull, T, 1, dfull, goff, d);
        const R *lg = lse + (i * Hfull + blockIdx.y * H) * T;
        for (int e = tid; e < H * T; e += nt) slse[e] = Softmax<R>::unit_lse(lg[e]);
    } else {
        // all three blocks' loads in flight together
        const R *s1 = qkv + i * T * 3 * d, *s2 = dout + i * T * d, *s3 = o + i * T * d;
        RowBatch<R, qkv_pieces<R, DH>()> b1;
        RowBatch<R, row_pieces<R, DH>()> b2, b3;
        const bool f = b1.fits(s1, T, 3 * d) && b2.fits(s2, T, d) && b3.fits(s3, T, d);
        R l0 = tid < H * T ? Softmax<R>::unit_lse(lse[i * H * T + tid]) : R(0);
        if (f) {
            b1.load(s1, T, 3 * d);
            b2.load(s2, T, d);
            b3.load(s3, T, d);
            b1.template store<HV::kNC>(sq, ldq, T, 3 * d);
            b2.template store<HV::kNC>(sdo, ldo, T, d);
            b3.template store<HV::kNC>(so, ldo, T, d);
        } else {
            rows_to_smem<R, HV::kNC>(sq, ldq, s1, T, 3 * d);
            rows_to_smem<R, HV::kNC>(sdo, ldo, s2, T, d);
            rows_to_smem<R, HV::kNC>(so, ldo, s3, T, d);
        }
        if (tid < H * T) slse[tid] = l0;
        for (int e = tid + nt; e < H * T; e += nt) slse[e] = Softmax<R>::unit_lse(lse[i * H * T + e]);
    }
    __syncthreads();
    const R scale = R(1) / sqrt(R(DH)), qs = score_scale<R, DH>();  // slse in score units
    const bool act = tid < H * T;
    const int hh = act ? tid % H : 0, pos = act ? tid / H : 0;  // heads fastest
    // D_q = do_q . o_q for every (head, position) first, so that the two
    // loops below (whose lengths q + 1 and T - j add up to T + 1 per thread)
    // run without a barrier between them
    R D = 0;
    if (act) {
        R dov[DH], ov[DH];
        HV::read_in(sdo + pos * ldo, hh * DH, dov);
        HV::read_in(so + pos * ldo, hh * DH, ov);
#pragma unroll
        for (int c = 0; c < DH; ++c) D += dov[c] * ov[c];
        sD[hh * T + pos] = D;
    }
    __syncthreads();
    if (act) {
        // dq_q = scale sum_{j<=q} p_qj (dp_qj - D_q) k_j
        const int q = pos;
        R qv[DH], dov[DH], dq[DH];
        HV::read_in(sq + q * ldq, hh * DH, qv);
        HV::read_in(sdo + q * ldo, hh * DH, dov);
#pragma unroll
        for (int c = 0; c < DH; ++c) {
            qv[c] = qv[c] * qs;
            dq[c] = 0;
        }
        const R L = slse[hh * T + q];
#pragma unroll 2
        for (int j = 0; j <= q; ++j) {
            R kj[DH], vj[DH];
            HV::read_in(sq + j * ldq, d + hh * DH, kj);
            HV::read_in(sq + j * ldq, 2 * d + hh * DH, vj);
            R sc = 0, dp = 0;
#pragma unroll
            for (int c = 0; c < DH; ++c) {
                sc += qv[c] * kj[c];
                dp += dov[c] * vj[c];
            }
            const R ds = Softmax<R>::pexp(sc - L) * (dp - D);
#pragma unroll
            for (int c = 0; c < DH; ++c) dq[c] += ds * kj[c];
        }
#pragma unroll
        for (int c = 0; c < DH; ++c) dq[c] = dq[c] * scale;
        HV::write(sg + q * ldq + hh * DH, dq);
    }
    if (act) {
        // dv_j = sum_{q>=j} p_qj do_q,  dk_j = scale sum_{q>=j} p_qj (dp_qj - D_q) q_q
        const int j = pos;
        R kv[DH], vv[DH], dk[DH], dv[DH];
        HV::read_in(sq + j * ldq, d + hh * DH, kv);
        HV::read_in(sq + j * ldq, 2 * d + hh * DH, vv);
#pragma unroll
        for (int c = 0; c < DH; ++c) dk[c] = dv[c] = 0;
#pragma unroll 2
        for (int q = j; q < T; ++q) {
            R qq[DH], dq[DH];
            HV::read_in(sq + q * ldq, hh * DH, qq);
            HV::read_in(sdo + q * ldo, hh * DH, dq);
            R sc = 0, dp = 0;
#pragma unroll
            for (int c = 0; c < DH; ++c) {
                sc += qq[c] * kv[c];
                dp += dq[c] * vv[c];
            }
            const R p = Softmax<R>::pexp(sc * qs - slse[hh * T + q]);
            const R ds = p * (dp - sD[hh * T + q]);
#pragma unroll
            for (int c = 0; c < DH; ++c) {
                dv[c] += p * dq[c];
                dk[c] += ds * qq[c];
            }
        }
#pragma unroll
        for (int c = 0; c < DH; ++c) dk[c] = dk[c] * scale;
        HV::write(sg + j * ldq + d + hh * DH, dk);
        HV::write(sg + j * ldq + 2 * d + hh * DH, dv);
    }
    __syncthreads();
    if (grouped)
        smem_to_seg_rows<R>(dqkv + i * T * 3 * dfull, sg, ldq, T, 3, dfull, goff, d);
    else
        smem_to_rows<R>(dqkv + i * T * 3 * d, sg, ldq, T, 3 * d);
    if (colsum) {
        for (int c = tid; c < 3 * d; c += nt) {
            R acc = 0;
            for (int t = 0; t < T; ++t) acc += sg[t * ldq + c];
            const int seg = c / d;
            colsum[i * 3 * dfull + seg * dfull + goff + (c - seg * d)] = acc;
        }
    }
}

// ------------------------------------------------------------------ head + masked log-softmax
constexpr int kMaxHeadD = 256;

// head weights [4][d] into shared memory (the whole block calls this)
template <class R>
__device__ void stage_head(const R *__restrict__ hw, int d, R *shw) {
    for (int k = threadIdx.x; k < 4 * d; k += blockDim.x) shw[k] = hw[k];
    __syncthreads();
}

// z[v] = hb[v] + sum_c hr[c] hw[v][c], c ascending; the row in 16-byte loads
// when it is aligned (the sampler's conditionals and the forward's pi~ use
// this same sum)
template <class R>
__device__ __forceinline__ void head_logits(const R *__restrict__ hr, const R *shw, const R *__restrict__ hb, int d,
                                            R (&z)[4]) {
    constexpr int V = int(16 / sizeof(R));
#pragma unroll
    for (int v = 0; v < 4; ++v) z[v] = hb[v];
    if (d % V == 0 && reinterpret_cast<uintptr_t>(hr) % 16 == 0) {
        for (int c = 0; c < d; c += 2 * V) {
            const ColVec<R, V> h0 = ld_vec<R, V>(hr + c);
            const bool two = c + V < d;
            const ColVec<R, V> h1 = two ? ld_vec<R, V>(hr + c + V) : h0;
#pragma unroll
            for (int e = 0; e < V; ++e)
#pragma unroll
                for (int v = 0; v < 4; ++v) z[v] += h0.v[e] * shw[v * d + c + e];
            if (two) {
#pragma unroll
                for (int e = 0; e < V; ++e)
#pragma unroll
                    for (int v = 0; v < 4; ++v) z[v] += h1.v[e] * shw[v * d + c + V + e];
            }
        }
    } else {
        for (int c = 0; c < d; ++c) {
            const R hv = hr[c];
#pragma unroll
            for (int v = 0; v < 4; ++v) z[v] += hv * shw[v * d + c];
        }
    }
}

// One warp per sample, lanes over positions.  pi~ of the 4 children at each
// position is stored for the backward; log|psi| = 1/2 sum_t log pi~(x_t).
template <class R>
__global__ void k_head(const uint64_t *__restrict__ x, int W, const R *__restrict__ hf, const R *__restrict__ hw,
                       const R *__restrict__ hb, const uint8_t *__restrict__ tok, int64_t n, int T, int d,
                       int n_alpha, int n_beta, R *__restrict__ pi, double2 *__restrict__ out, DevStatus *st,
                       int64_t row_offset) {
    __shared__ R shw[4 * kMaxHeadD];
    stage_head<R>(hw, d, shw);
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    const uint64_t *xi = x + i * W;
    R sum = 0;
    bool bad = false;
    for (int t = lane; t < T; t += 32) {
        // electrons already placed on orbitals p' > p = T-1-t (tokens < t)
        int ca = 0, cb = 0;
        for (int p2 = T - t; p2 < T; ++p2) {
            ca += bit_of(xi, 2 * p2);
            cb += bit_of(xi, 2 * p2 + 1);
        }
        const int rem = T - 1 - t;
        R z[4];
        head_logits<R>(hf + (i * T + t) * d, shw, hb, d, z);
        bool ok[4];
        R zmax = neg_inf<R>();
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int a = ca + (v & 1), b = cb + (v >> 1);
            ok[v] = a <= n_alpha && b <= n_beta && a + rem >= n_alpha && b + rem >= n_beta;
            if (ok[v] && z[v] > zmax) zmax = z[v];
        }
        R se = 0;
#pragma unroll
        for (int v = 0; v < 4; ++v)
            if (ok[v]) se += exp_<R>(z[v] - zmax);
        const R lse = zmax + log_<R>(se);
        const int tk = tok[i * T + t];
#pragma unroll
        for (int v = 0; v < 4; ++v) pi[(i * T + t) * 4 + v] = ok[v] ? exp_<R>(z[v] - lse) : R(0);
        if (ok[tk])
            sum += z[tk] - lse;
        else
            bad = true;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
    bad = __any_sync(0xffffffffu, bad);
    if (lane == 0) {
        const double la = bad ? -(double)INFINITY : 0.5 * (double)sum;
        out[i].x = la;
        if (bad) record_status(st, NNQS_E_SECTOR, row_offset + i);
    }
}

// ---- key/value-cached decoding for the sampler --------------------------
// Every node of the prefix tree owns one row of q|k|v per layer in a pool
// [node][L][3d]; a node at depth t attends over the rows of its ancestors
// at depths 0..t (found through parent pointers) and itself, in depth order,
// which is the order the full forward visits keys.
template <class R>
__global__ void k_embed_decode(const uint64_t *__restrict__ x, int W, int64_t n, int t, int T, int d,
                               const R *__restrict__ tok_emb, const R *__restrict__ pos_emb, R *__restrict__ h) {
    const int64_t total = n * d;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(idx % d);
        const int64_t i = idx / d;
        const int inp = t == 0 ? 4 : token_at(x + i * W, T, t - 1);
        h[idx] = tok_emb[inp * d + c] + pos_emb[t * d + c];
    }
}

constexpr int kMaxDepth = 64;

// One (prefix, head) of the cached attention: the prefix's node at depth t
// attends over the nodes anc[0..t-1] of its ancestors and itself, in depth
// order, with the online softmax of the full forward (same arithmetic, so the
// cached sampler reproduces the recomputed conditionals bit for bit).
template <class R, int DH>
__device__ __forceinline__ void attn_decode_row(const R *__restrict__ pool, const int32_t *__restrict__ anc_row,
                                                int64_t anc_stride, int64_t self, int t, int L, int l, int d, int hh,
                                                R (&o)[DH]) {
    const int64_t row = 3 * (int64_t)d;
    const R scale = score_scale<R, DH>();
    R qv[DH], acc[DH];
    const R *qp = pool + (self * L + l) * row + hh * DH;
#pragma unroll
    for (int c = 0; c < DH; ++c) {
        qv[c] = qp[c] * scale;
        acc[c] = 0;
    }
    R m = neg_inf<R>(), lsum = 0;
    for (int j = 0; j <= t; ++j) {
        const int64_t node = j < t ? (int64_t)anc_row[j * anc_stride] : self;
        const R *base = pool + (node * L + l) * row;
        const R *kj = base + d + hh * DH;
        const R *vj = base + 2 * d + hh * DH;
        R sc = 0;
#pragma unroll
        for (int c = 0; c < DH; ++c) sc += qv[c] * kj[c];
        const R mn = sc > m ? sc : m;
        const R corr = Softmax<R>::pexp(m - mn);
        const R p = Softmax<R>::pexp(sc - mn);
        lsum = lsum * corr + p;
#pragma unroll
        for (int c = 0; c < DH; ++c) acc[c] = acc[c] * corr + p * vj[c];
        m = mn;
    }
    const R inv = R(1) / lsum;
#pragma unroll
    for (int c = 0; c < DH; ++c) o[c] = acc[c] * inv;
}

// anc: depth-major ancestor table of the current level (anc[j * anc_stride +
// i] is the node of prefix i at depth j < t); prefix i is node g0 + i
template <class R, int DH>
__global__ void k_attn_decode(const R *__restrict__ pool, const int32_t *__restrict__ anc, int64_t anc_stride,
                              int64_t g0, int64_t n, int t, int L, int l, int H, int d, R *__restrict__ o) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n * H) return;
    const int hh = (int)(idx % H);
    const int64_t i = idx / H;
    R ov[DH];
    attn_decode_row<R, DH>(pool, anc + i, anc_stride, g0 + i, t, L, l, d, hh, ov);
#pragma unroll
    for (int c = 0; c < DH; ++c) o[i * d + hh * DH + c] = ov[c];
}

// pi~(v | prefix) at position t from the head logits zr: the number mask
// (children from which the remaining orbitals can still reach n_alpha,
// n_beta) and a softmax over the allowed children in FP64 -> out[4]; false
// when no child is allowed
template <class R>
__device__ __forceinline__ bool cond_from_logits(const uint64_t *xi, int T, int t, int n_alpha, int n_beta,
                                                 const R (&zr)[4], double *out) {
    int ca = 0, cb = 0;
    for (int p2 = T - t; p2 < T; ++p2) {
        ca += bit_of(xi, 2 * p2);
        cb += bit_of(xi, 2 * p2 + 1);
    }
    const int rem = T - 1 - t;
    // the softmax runs in the logits' precision and is widened at the end:
    // FP32 logits give FP32 conditionals (the binomial chain only needs them
    // to ~1e-7 relative), FP64 logits FP64 ones
    R z[4], zmax = neg_inf<R>();
    bool ok[4], any = false;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        z[v] = zr[v];
        const int aa = ca + (v & 1), bb = cb + (v >> 1);
        ok[v] = aa <= n_alpha && bb <= n_beta && aa + rem >= n_alpha && bb + rem >= n_beta;
        if (ok[v]) {
            any = true;
            zmax = z[v] > zmax ? z[v] : zmax;
        }
    }
    R e[4], se = R(0);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        e[v] = ok[v] ? exp_<R>(z[v] - zmax) : R(0);
        se += e[v];
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) out[v] = ok[v] ? (double)(e[v] / se) : 0.0;
    return any;
}

// ---- fused key/value-cached decode layer on tensor cores (d = 64, F = 256)
// One launch per layer and sampler step instead of seven: a CTA of 256
// threads takes 128 prefixes (one new token each) through LayerNorm -> qkv
// (rows written to the cache pool) -> attention over the cached ancestors ->
// out-projection + residual -> LayerNorm -> FFN in four 64-column chunks
// (W1 chunk, GELU, W2 chunk accumulated) -> residual, keeping the residual
// rows in shared memory, the A operands as BF16 (split hi/lo) swizzled tiles,
// the weights brought in by bulk copies of their pre-swizzled images, and the
// accumulators in TMEM.  Every step does the arithmetic of the
// unfused path in the same order (same LayerNorm tree, same MMA order per
// K step, same epilogue sums, the same attention loop), so the cached
// sampler still reproduces the recomputed conditionals bit for bit.
namespace dec {
constexpr int kThreads = 512, kRows = 128, kD = 64, kQKV = 192, kF = 256;
// columns of a 64-column TMEM chunk per thread in the epilogues: warp w reads
// lanes 32 (w % 4) .. + 31 (its TMEM lane quarter), columns kCW (w / 4) .. + kCW - 1
constexpr int kCW = 64 * 4 / (kThreads / 32);
constexpr int kOffA = 0;         // A operand hi [128][64] BF16 (16 KB); lo at +16 KB
constexpr int kOffG = 32768;     // Wo hi / lo (+8 KB); in the FFN [0, 128 KB) holds its [128][256] GELU operand
constexpr int kOffB = 65536;     // Wqkv hi / lo (+24 KB); after the qkv MMA: W1 hi, W1 lo, W2 hi, W2 lo
constexpr int kQkvLo = 24576;
constexpr int kW1Hi = 0, kW1Lo = 32768, kW2Hi = 65536, kW2Lo = 98304;  // 4 chunks of 8 KB each
constexpr int kOffH = kOffB + 131072;  // residual rows [128][65] FP32
constexpr int kHS = 65;
constexpr int kOffBar = kOffH + kRows * kHS * 4;
constexpr int kSmem = kOffBar + 64 + 1024;  // 230,976 bytes
// TMEM columns: q|k|v, then the attention's out-projection; the FFN-in
// product U (256 columns, one N = 256 product over the finished q|k|v and out-
// projection columns, chunk c at 64 c) and the FFN-out accumulator after them
constexpr uint32_t kColQKV = 0, kColO = 192, kColU = 0, kColY = 256, kTmemCols = 512;
__device__ __forceinline__ constexpr uint32_t col_u(int c) { return kColU + 64u * uint32_t(c); }
}  // namespace dec

constexpr int kDecMaxLayers = 16;

struct DecodeArgs {
    int64_t n;
    int rpc;  // prefixes per CTA (<= 128; rows past it in the 128-row tile are idle)
    float *pool;  // [node][L][192] q|k|v (the fused step writes k|v only: its q stays on chip)
    int L, Tm, t;
    int64_t g0;
    const int32_t *anc;  // depth-major ancestor nodes: anc[j * anc_stride + i], depths j < t
    int64_t anc_stride;
    // per layer: LayerNorm, bias vectors and the swizzled shared-memory images
    // of the weights (high part, then the low part): qkv [192 rows],
    // out-projection [64], FFN in [256], FFN out [64 rows, 4 K blocks]
    const float *ln1g[kDecMaxLayers], *ln1b[kDecMaxLayers], *ln2g[kDecMaxLayers], *ln2b[kDecMaxLayers];
    const float *bqkv[kDecMaxLayers], *bo[kDecMaxLayers], *b1[kDecMaxLayers], *b2[kDecMaxLayers];
    const __nv_bfloat16 *tqkv[kDecMaxLayers], *to[kDecMaxLayers], *t1[kDecMaxLayers], *t2[kDecMaxLayers];
    DevStatus *st;
    // the rows enter as the embeddings of the prefixes' last tokens
    // (tok_emb[input] + pos_emb[t]); after the last layer: final LayerNorm,
    // head and the masked conditionals pi~(. | prefix) -> cond[n][4]
    const uint64_t *x;  // [n][W] prefixes
    int W, n_alpha, n_beta;
    const float *tok_emb, *pos_emb, *lnf_g, *lnf_b, *hw, *hb;
    double *cond;
    // device-side counts (the sampler's steps without a host round trip):
    // when n_dev is set, n = *n_dev and g0 = *g0_dev, and the prefixes per CTA
    // are ceil(n / n_sms) (at most 128) computed on the device; the grid is
    // sized for the capacity and CTAs past n return at once
    const int64_t *n_dev, *g0_dev;
    int n_sms;
    // optional (both null or both set): per tree node the residual row at
    // each layer's input and after its attention, act[node][L][2][64], and the
    // final residual fin[node][64] (what the reverse mode of the energy
    // gradient reads, nnqs_energy_grad_sampled)
    float *act, *fin;
};

// one bulk asynchronous copy global -> shared, completing `bytes` on mbar
__device__ __forceinline__ void bulk_g2s(uint8_t *dst, const void *src, uint32_t bytes, uint32_t mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     tc::smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(mbar)
                 : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(mbar),
                 "r"(bytes)
                 : "memory");
}

// one 8-column granule of an A tile row: BF16 high part, and the low part
__device__ __forceinline__ void dec_store_granule(uint8_t *hi, uint8_t *lo, int r, int c, const float (&v)[8], bool split) {
    const int off = r * 128 + ((c ^ (r & 7)) << 4);
    *reinterpret_cast<uint4 *>(hi + off) = tc::pack8(v);
    if (split) {
        float x[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) x[e] = v[e] - __bfloat162float(__float2bfloat16_rn(v[e]));
        *reinterpret_cast<uint4 *>(lo + off) = tc::pack8(x);
    }
}

// LayerNorm of residual row r (shared, stride 65) into the A tile, the lane sums
// of the 16-lane FP32 kernel combined in its tree order, over 4 lanes per row
// (lanes 4 r' .. 4 r' + 3 of a warp, lq = lane & 3): lane lq holds the float4 pieces lq, lq + 4, lq + 8, lq + 12, so
// the first two levels of the 16-piece tree (pieces k + 8, then k + 4) are its
// own and the last two (k + 2, k + 1) are shuffles with lanes lq ^ 2 and lq ^ 1.
// Every addition pairs the same two values as one lane walking the tree (IEEE
// addition commutes), so the results are the same bits; each lane writes its
// four pieces as half granules.
__device__ __forceinline__ void dec_layernorm_row4(const float *sH, int r, int lq, const float *__restrict__ g,
                                                   const float *__restrict__ b, uint8_t *aHi, uint8_t *aLo,
                                                   bool split) {
    float4 v[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int k = lq + 4 * m;
        v[m] = make_float4(sH[r * dec::kHS + 4 * k], sH[r * dec::kHS + 4 * k + 1], sH[r * dec::kHS + 4 * k + 2],
                           sH[r * dec::kHS + 4 * k + 3]);
    }
    float s = (ln_part_sum(v[0]) + ln_part_sum(v[2])) + (ln_part_sum(v[1]) + ln_part_sum(v[3]));
    s = s + __shfl_xor_sync(0xffffffffu, s, 2);
    s = s + __shfl_xor_sync(0xffffffffu, s, 1);
    const float mu = s / float(dec::kD);
    float q = (ln_part_sq(v[0], mu) + ln_part_sq(v[2], mu)) + (ln_part_sq(v[1], mu) + ln_part_sq(v[3], mu));
    q = q + __shfl_xor_sync(0xffffffffu, q, 2);
    q = q + __shfl_xor_sync(0xffffffffu, q, 1);
    const float rs = ln_rstd(q, dec::kD);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int k = lq + 4 * m, c = k >> 1;
        const float4 y = ln_apply(v[m], mu, rs, __ldg(reinterpret_cast<const float4 *>(g) + k),
                                  __ldg(reinterpret_cast<const float4 *>(b) + k));
        const int off = r * 128 + ((c ^ (r & 7)) << 4) + 8 * (k & 1);
        const __nv_bfloat162 h0 = __floats2bfloat162_rn(y.x, y.y), h1 = __floats2bfloat162_rn(y.z, y.w);
        *reinterpret_cast<uint2 *>(aHi + off) =
            make_uint2(*reinterpret_cast<const uint32_t *>(&h0), *reinterpret_cast<const uint32_t *>(&h1));
        if (split) {
            const __nv_bfloat162 l0 = __floats2bfloat162_rn(y.x - __low2float(h0), y.y - __high2float(h0));
            const __nv_bfloat162 l1 = __floats2bfloat162_rn(y.z - __low2float(h1), y.w - __high2float(h1));
            *reinterpret_cast<uint2 *>(aLo + off) =
                make_uint2(*reinterpret_cast<const uint32_t *>(&l0), *reinterpret_cast<const uint32_t *>(&l1));
        }
    }
}

// the same LayerNorm by one lane per row, FP32 output values (the final LayerNorm)
__device__ __forceinline__ void dec_layernorm_row_f32(const float *sH, int r, const float *__restrict__ g,
                                                      const float *__restrict__ b, float (&y)[dec::kD]) {
    float4 v[16];
#pragma unroll
    for (int k = 0; k < 16; ++k)
        v[k] = make_float4(sH[r * dec::kHS + 4 * k], sH[r * dec::kHS + 4 * k + 1], sH[r * dec::kHS + 4 * k + 2],
                           sH[r * dec::kHS + 4 * k + 3]);
    float a[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) a[k] = ln_part_sum(v[k]);
#pragma unroll
    for (int o = 8; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < o; ++k) a[k] = a[k] + a[k + o];
    const float mu = a[0] / float(dec::kD);
#pragma unroll
    for (int k = 0; k < 16; ++k) a[k] = ln_part_sq(v[k], mu);
#pragma unroll
    for (int o = 8; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < o; ++k) a[k] = a[k] + a[k + o];
    const float rs = ln_rstd(a[0], dec::kD);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const float4 o = ln_apply(v[k], mu, rs, __ldg(reinterpret_cast<const float4 *>(g) + k),
                                  __ldg(reinterpret_cast<const float4 *>(b) + k));
        y[4 * k] = o.x;
        y[4 * k + 1] = o.y;
        y[4 * k + 2] = o.z;
        y[4 * k + 3] = o.w;
    }
}

// Head hh of NR prefixes (rows r0, r0 + 1, ...): the per-head arithmetic of
// attn_decode_row for each row, with the ancestor loop outside so that the
// keys and values of the NR rows are loaded together.  Threads hh = 0..H-1
// of a row group sit in consecutive lanes, so a warp's load covers whole
// 256-byte key (or value) segments of a few rows.
// The rows' q come from qslab (the CTA's tile, [128][64] FP32 with 16-byte
// granules XOR-swizzled by the row; tile row = row - safe).  Rows at or past
// n (the tail of the last CTA) read row `safe` (a valid row) instead and give
// zeros.
template <int DH, int NR>
__device__ __forceinline__ void dec_attention_rows(const float *__restrict__ pool, const float *qslab,
                                                   const int32_t *__restrict__ anc, int64_t anc_stride, int64_t g0,
                                                   int64_t r0, int64_t safe, int64_t n, int t, int L, int l, int hh,
                                                   float (&o)[NR][DH]) {
    constexpr int d = dec::kD;
    const int64_t row = 3 * (int64_t)d;
    const float scale = score_scale<float, DH>();
    float qv[NR][DH], acc[NR][DH], m[NR], lsum[NR];
    bool ok[NR];
    int64_t rr[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        ok[k] = r0 + k < n;
        rr[k] = ok[k] ? r0 + k : safe;
        const int tr = (int)(rr[k] - safe);  // tile row (safe = the CTA's first row)
#pragma unroll
        for (int e = 0; e < DH / 4; ++e) {
            const int gi = hh * (DH / 4) + e;
            const float4 q4 = *reinterpret_cast<const float4 *>(qslab + tr * 64 + 4 * (gi ^ (tr & 15)));
            qv[k][4 * e] = q4.x * scale;
            qv[k][4 * e + 1] = q4.y * scale;
            qv[k][4 * e + 2] = q4.z * scale;
            qv[k][4 * e + 3] = q4.w * scale;
        }
#pragma unroll
        for (int c = 0; c < DH; ++c) acc[k][c] = 0.f;
        m[k] = neg_inf<float>();
        lsum[k] = 0.f;
    }
    __syncthreads();  // every q is read before the outputs go to the same tile
    // keys and values of step j + 1 load while step j is computed (the last
    // prefetch rereads the row's own node); node ids are read one step further
    // ahead
    auto load_kv = [&](const int64_t (&nd)[NR], float (&kk)[NR][DH], float (&vv)[NR][DH]) {
#pragma unroll
        for (int k = 0; k < NR; ++k) {
            const float *base = pool + (nd[k] * L + l) * row;
#pragma unroll
            for (int e = 0; e < DH; e += 4) {
                const float4 k4 = *reinterpret_cast<const float4 *>(base + d + hh * DH + e);
                const float4 v4 = *reinterpret_cast<const float4 *>(base + 2 * d + hh * DH + e);
                kk[k][e] = k4.x; kk[k][e + 1] = k4.y; kk[k][e + 2] = k4.z; kk[k][e + 3] = k4.w;
                vv[k][e] = v4.x; vv[k][e + 1] = v4.y; vv[k][e + 2] = v4.z; vv[k][e + 3] = v4.w;
            }
        }
    };
    auto node_at = [&](int j, int k) -> int64_t { return j < t ? (int64_t)anc[j * anc_stride + rr[k]] : g0 + rr[k]; };
    float kk[NR][DH], vv[NR][DH];
    int64_t node[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) node[k] = node_at(0, k);
    load_kv(node, kk, vv);
#pragma unroll
    for (int k = 0; k < NR; ++k) node[k] = node_at(1, k);
    for (int j = 0; j <= t; ++j) {
        float kn[NR][DH], vn[NR][DH];
        load_kv(node, kn, vn);
#pragma unroll
        for (int k = 0; k < NR; ++k) node[k] = node_at(j + 2, k);
#pragma unroll
        for (int k = 0; k < NR; ++k) {
            float sc = 0;
#pragma unroll
            for (int c = 0; c < DH; ++c) sc += qv[k][c] * kk[k][c];
            const float mn = sc > m[k] ? sc : m[k];
            const float corr = Softmax<float>::pexp(m[k] - mn);
            const float p = Softmax<float>::pexp(sc - mn);
            lsum[k] = lsum[k] * corr + p;
#pragma unroll
            for (int c = 0; c < DH; ++c) acc[k][c] = acc[k][c] * corr + p * vv[k][c];
            m[k] = mn;
        }
#pragma unroll
        for (int k = 0; k < NR; ++k)
#pragma unroll
            for (int c = 0; c < DH; ++c) {
                kk[k][c] = kn[k][c];
                vv[k][c] = vn[k][c];
            }
    }
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        const float inv = 1.0f / lsum[k];
#pragma unroll
        for (int c = 0; c < DH; ++c) o[k][c] = ok[k] ? acc[k][c] * inv : 0.f;
    }
}

// 4 K steps of one 128 x N tile: (lo, hi), (hi, lo), (hi, hi) per step with
// split operands, as the unfused kernel issues them
__device__ __forceinline__ void dec_mma(uint32_t tmem, uint32_t aHi, uint32_t aLo, uint32_t bHi, uint32_t bLo, int N,
                                        bool split, bool acc0) {
    const uint32_t idesc = tc::idesc_bf16(dec::kRows, N);
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

// the CTA's residual rows (shared, stride 65) to rows of a per-node pool:
// thread (row tid / 4, quarter tid % 4) copies 16 floats of a valid row
__device__ __forceinline__ void dec_store_rows(const float *sH, float *dst, int64_t node0, int64_t rows,
                                               int64_t node_stride) {
    const int r = threadIdx.x >> 2, q = threadIdx.x & 3;
    if (r >= rows) return;
    float *o = dst + (node0 + r) * node_stride + 16 * q;
#pragma unroll
    for (int k = 0; k < 4; ++k)
        reinterpret_cast<float4 *>(o)[k] =
            make_float4(sH[r * dec::kHS + 16 * q + 4 * k], sH[r * dec::kHS + 16 * q + 4 * k + 1],
                        sH[r * dec::kHS + 16 * q + 4 * k + 2], sH[r * dec::kHS + 16 * q + 4 * k + 3]);
}

template <bool SPLIT, int DH>
__global__ void __launch_bounds__(dec::kThreads, 1) k_decode_step(const __grid_constant__ DecodeArgs g) {
    using namespace dec;
    constexpr int H = kD / DH, NR = kRows * H / kThreads;  // rows per thread in the attention
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = tc::smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *sb = smem_raw + (base - raw);
    uint8_t *aHi = sb + kOffA, *aLo = sb + kOffA + 16384;
    uint8_t *gHi = sb + kOffG;
    uint8_t *bB = sb + kOffB;
    float *sH = reinterpret_cast<float *>(sb + kOffH);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sb + kOffBar);
    uint64_t *wbar = reinterpret_cast<uint64_t *>(sb + kOffBar + 8);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sb + kOffBar + 16);
    const uint32_t uA = base + kOffA, uA2 = base + kOffA + 16384, uG = base + kOffG;
    const uint32_t uB = base + kOffB;
    const uint32_t wb = tc::smem_u32(wbar);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int64_t n = g.n, g0 = g.g0;
    int rpc = g.rpc;
    if (g.n_dev) {
        n = *g.n_dev;
        g0 = *g.g0_dev;
        const int64_t per = (n + g.n_sms - 1) / g.n_sms;
        rpc = per < 1 ? 1 : (per > kRows ? kRows : (int)per);
    }
    const int64_t m0 = blockIdx.x * (int64_t)rpc;
    if (m0 >= n) return;  // (device-side counts only: a CTA with no rows)
    const int64_t n_cta = min(n, m0 + rpc);  // rows of this CTA are m0 .. n_cta - 1
    // weight copies: phase 2 l brings layer l's Wqkv, phase 2 l + 1 its Wo,
    // W1 and W2 (one barrier, waited in issue order)
    auto issue_wqkv = [&](int l) {
        constexpr uint32_t q = kQKV * 128;
        mbar_expect_tx(wb, SPLIT ? 2 * q : q);
        bulk_g2s(bB, g.tqkv[l], q, wb);
        if (SPLIT) bulk_g2s(bB + kQkvLo, g.tqkv[l] + kQKV * kD, q, wb);
    };
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(tslot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        tc::mbar_init(tc::smem_u32(mbar), 1);
        tc::mbar_init(wb, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        issue_wqkv(0);
    }
    int wissued = 1, wdone = 0;  // weight-barrier phases issued / seen complete
    // residual rows: the embeddings, as k_embed_decode forms them; all of a
    // thread's loads are issued before its shared stores
    {
        constexpr int kIt = kRows * (kD / 4) / kThreads;
        float4 v[kIt];
#pragma unroll
        for (int i = 0; i < kIt; ++i) {
            const int it = tid + kThreads * i;
            const int r = it >> 4, c4 = it & 15;
            v[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (m0 + r < n_cta) {
                const int inp = g.t == 0 ? 4 : token_at(g.x + (m0 + r) * g.W, g.Tm, g.t - 1);
                const float4 te = __ldg(reinterpret_cast<const float4 *>(g.tok_emb + inp * kD) + c4);
                const float4 pe = __ldg(reinterpret_cast<const float4 *>(g.pos_emb + g.t * kD) + c4);
                v[i] = make_float4(te.x + pe.x, te.y + pe.y, te.z + pe.z, te.w + pe.w);
            }
        }
#pragma unroll
        for (int i = 0; i < kIt; ++i) {
            const int it = tid + kThreads * i;
            const int r = it >> 4, c4 = it & 15;
            sH[r * kHS + 4 * c4] = v[i].x;
            sH[r * kHS + 4 * c4 + 1] = v[i].y;
            sH[r * kHS + 4 * c4 + 2] = v[i].z;
            sH[r * kHS + 4 * c4 + 3] = v[i].w;
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const uint32_t mb = tc::smem_u32(mbar);
    uint32_t phase = 0;
    bool ok = true;
    auto sync_async = [&]() {
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
    };
    auto wait_mma = [&]() {
        ok = __syncthreads_and(tc::mbar_wait(mb, phase) ? 1 : 0) != 0;
        phase ^= 1u;
        tc::fence_after_sync();
    };
    auto wait_weights = [&]() {
        ok = __syncthreads_and(tc::mbar_wait(wb, uint32_t(wdone & 1)) ? 1 : 0) != 0;
        if (ok) ++wdone;
    };
    const int q4 = warp & 3, cq = warp >> 2, row = 32 * q4 + lane;
    const uint32_t tl = tmem + (uint32_t(32 * q4) << 16);
    // warps whose rows all lie past the CTA's share skip the per-row work
    // (the products keep rows apart, and those rows are never stored): the
    // TMEM-lane quadrant of 32 rows, the LayerNorms' 8 rows per warp
    const int rows_live = (int)(n_cta - m0);
    const bool q_live = 32 * q4 < rows_live, ln_live = 8 * warp < rows_live;

    const int64_t act_stride = 2 * (int64_t)g.L * kD;  // floats per node of g.act
    for (int l = 0; l < g.L && ok; ++l) {
        if (g.act) dec_store_rows(sH, g.act + 2 * l * kD, g0 + m0, n_cta - m0, act_stride);
        // ---- LayerNorm 1 -> qkv
        if (ln_live) dec_layernorm_row4(sH, tid >> 2, tid & 3, g.ln1g[l], g.ln1b[l], aHi, aLo, SPLIT);
        wait_weights();  // Wqkv of layer l
        sync_async();
        if (!ok) break;
        if (tid == 0) {
            dec_mma(tmem + kColQKV, uA, uA2, uB, uB + kQkvLo, kQKV, SPLIT, false);
            tc::mma_commit(mb);
        }
        wait_mma();
        if (!ok) break;
        // Wo into the (idle) FFN-out tile, the FFN weights over Wqkv: copies in
        // flight during the epilogue and the attention
        ++wissued;
        if (tid == 0) {
            constexpr uint32_t bo = kD * 128, bf = kF * 128;  // 8 KB, 32 KB
            mbar_expect_tx(wb, SPLIT ? 2 * (bo + 2 * bf) : bo + 2 * bf);
            bulk_g2s(gHi, g.to[l], bo, wb);
            bulk_g2s(bB + kW1Hi, g.t1[l], bf, wb);
            bulk_g2s(bB + kW2Hi, g.t2[l], bf, wb);
            if (SPLIT) {
                bulk_g2s(gHi + 8192, g.to[l] + kD * kD, bo, wb);
                bulk_g2s(bB + kW1Lo, g.t1[l] + kF * kD, bf, wb);
                bulk_g2s(bB + kW2Lo, g.t2[l] + kD * kF, bf, wb);
            }
        }
        // k|v + bias into the pool rows of the new nodes, 64 columns at a time
        // through the (free) A tile: TMEM -> shared (thread = row, 16-byte
        // granules XOR-swizzled by the row) -> global (16 threads per row, each
        // row a contiguous 256-byte segment); q + bias last, left in the tile
        // for this step's attention (only the rows' own attention reads it)
        float *slab = reinterpret_cast<float *>(aHi);
        {
            const float *bq = g.bqkv[l];
            for (int cc = 1; cc <= kQKV / 64; ++cc) {
                const int c = cc % (kQKV / 64);  // 1 (k), 2 (v), then 0 (q)
#pragma unroll
                for (int b = 0; b < (q_live ? kCW / 16 : 0); ++b) {
                    const int cl = kCW * cq + 16 * b;  // column within the chunk
                    uint32_t r16[16];
                    tc::tmem_ld16(tl + kColQKV + 64 * c + cl, r16);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int gi = (cl >> 2) + q;
                        const int col = 64 * c + 4 * gi;
                        *reinterpret_cast<float4 *>(slab + row * 64 + 4 * (gi ^ (row & 15))) =
                            make_float4(__uint_as_float(r16[4 * q]) + bq[col], __uint_as_float(r16[4 * q + 1]) + bq[col + 1],
                                        __uint_as_float(r16[4 * q + 2]) + bq[col + 2],
                                        __uint_as_float(r16[4 * q + 3]) + bq[col + 3]);
                    }
                }
                __syncthreads();
                if (c == 0) break;
#pragma unroll
                for (int i = 0; i < kRows * 16 / kThreads; ++i) {
                    const int it = tid + kThreads * i;
                    const int r = it >> 4, gi = it & 15;
                    if (m0 + r < n_cta) {
                        float *prow = g.pool + ((g0 + m0 + r) * g.L + l) * (int64_t)kQKV + 64 * c;
                        *reinterpret_cast<float4 *>(prow + 4 * gi) =
                            *reinterpret_cast<const float4 *>(slab + r * 64 + 4 * (gi ^ (r & 15)));
                    }
                }
                __syncthreads();
            }
        }
        // ---- attention (thread: head tid % H of the NR rows of group tid / H) -> A tile
        {
            const int hh = tid % H;
            const int r0 = (tid / H) * NR;
            float o[NR][DH];
            dec_attention_rows<DH, NR>(g.pool, slab, g.anc, g.anc_stride, g0, m0 + r0, m0, n_cta, g.t, g.L, l, hh, o);
#pragma unroll
            for (int k = 0; k < NR; ++k)
#pragma unroll
                for (int gi = 0; gi < DH / 8; ++gi) {
                    float x[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) x[e] = o[k][8 * gi + e];
                    dec_store_granule(aHi, aLo, r0 + k, hh * (DH / 8) + gi, x, SPLIT);
                }
        }
        wait_weights();  // Wo, W1, W2 of layer l
        sync_async();
        if (!ok) break;
        if (tid == 0) {
            dec_mma(tmem + kColO, uA, uA2, uG, uG + 8192, kD, SPLIT, false);
            tc::mma_commit(mb);
        }
        wait_mma();
        if (!ok) break;
        {
            // h += attn Wo^T + bo (kCW columns per thread)
            const float *bo = g.bo[l];
#pragma unroll
            for (int b = 0; b < (q_live ? kCW / 16 : 0); ++b) {
                const int c0 = kCW * cq + 16 * b;
                uint32_t r16[16];
                tc::tmem_ld16(tl + kColO + c0, r16);
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const float v = __uint_as_float(r16[j]) + bo[c0 + j];
                    sH[row * kHS + c0 + j] = sH[row * kHS + c0 + j] + v;
                }
            }
        }
        __syncthreads();
        if (g.act) dec_store_rows(sH, g.act + (2 * l + 1) * kD, g0 + m0, n_cta - m0, act_stride);
        // ---- LayerNorm 2 -> FFN: U = LN2 W1^T as one N = 256 product (the
        // four 64-row chunks of the W1 image are consecutive), then GELU and
        // the FFN-out product (below)
        if (ln_live) dec_layernorm_row4(sH, tid >> 2, tid & 3, g.ln2g[l], g.ln2b[l], aHi, aLo, SPLIT);
        sync_async();
        if (tid == 0) {
            dec_mma(tmem + kColU, uA, uA2, uB + kW1Hi, uB + kW1Lo, kF, SPLIT, false);
            tc::mma_commit(mb);
        }
        wait_mma();
        if (!ok) break;
        // GELU of every chunk U_c into shared memory first: the A and G tiles
        // and the FFN-in weights' region (all read by finished products) hold
        // the whole [128][256] operand, chunk c at 16 KB c (high part) and
        // 64 KB + 16 KB c (low part); then the 4 x 4 K steps of the FFN-out
        // product in the order of the chunked walk, Y = sum_c G_c W2_c^T
        const float *b1 = g.b1[l];
#pragma unroll 1
        for (int c = 0; c < (q_live ? kF / kD : 0); ++c) {
            float x[kCW];
#pragma unroll
            for (int b = 0; b < kCW / 16; ++b) {
                const int c0 = kCW * cq + 16 * b;
                uint32_t r16[16];
                tc::tmem_ld16(tl + col_u(c) + c0, r16);
#pragma unroll
                for (int e = 0; e < 16; ++e) x[16 * b + e] = tc::gelu_f(__uint_as_float(r16[e]) + b1[kD * c + c0 + e]);
            }
#pragma unroll
            for (int b = 0; b < kCW / 16; ++b)
#pragma unroll
                for (int gi = 0; gi < 2; ++gi) {
                    float xg[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) xg[e] = x[16 * b + 8 * gi + e];
                    dec_store_granule(sb + 16384 * c, sb + 65536 + 16384 * c, row, ((kCW * cq + 16 * b) >> 3) + gi,
                                      xg, SPLIT);
                }
        }
        sync_async();
        if (tid == 0) {
#pragma unroll
            for (int c = 0; c < kF / kD; ++c)
                dec_mma(tmem + kColY, base + 16384u * c, base + 65536u + 16384u * c, uB + kW2Hi + 8192 * c,
                        uB + kW2Lo + 8192 * c, kD, SPLIT, c > 0);
            tc::mma_commit(mb);
        }
        wait_mma();
        if (!ok) break;
        // the FFN-out product has read the operand: the next layer's Wqkv
        // comes in over its low part
        if (l + 1 < g.L) {
            ++wissued;
            if (tid == 0) issue_wqkv(l + 1);
        }
        {
            // h += FFN + b2, in the shared rows
            const float *b2 = g.b2[l];
#pragma unroll
            for (int b = 0; b < (q_live ? kCW / 16 : 0); ++b) {
                const int c0 = kCW * cq + 16 * b;
                uint32_t r16[16];
                tc::tmem_ld16(tl + kColY + c0, r16);
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const float y = __uint_as_float(r16[j]) + b2[c0 + j];
                    sH[row * kHS + c0 + j] = sH[row * kHS + c0 + j] + y;
                }
            }
        }
        __syncthreads();
    }
    if (ok && g.fin) dec_store_rows(sH, g.fin, g0 + m0, n_cta - m0, kD);
    // ---- final LayerNorm (k_ln_fwd_v's sums), head logits (head_logits'
    // sum) and the masked conditionals of the next token
    if (ok && tid < kRows && m0 + tid < n_cta) {
        float hf[kD];
        dec_layernorm_row_f32(sH, tid, g.lnf_g, g.lnf_b, hf);
        float zr[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) zr[v] = g.hb[v];
#pragma unroll
        for (int c = 0; c < kD; ++c)
#pragma unroll
            for (int v = 0; v < 4; ++v) zr[v] += hf[c] * __ldg(g.hw + v * kD + c);
        if (!cond_from_logits<float>(g.x + (m0 + tid) * g.W, g.Tm, g.t, g.n_alpha, g.n_beta, zr,
                                     g.cond + (m0 + tid) * 4))
            record_status(g.st, NNQS_E_SECTOR, m0 + tid);
    }
    if (!ok && tid == 0) {
        if (atomicCAS(&g.st->code, 0, (int)NNQS_E_TIMEOUT) == 0) g.st->index = -11;
        // let weight copies still in flight land (bounded) before the CTA ends
        for (int p = wdone; p < wissued; ++p) tc::mbar_wait(wb, (uint32_t)(p & 1));
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(dec::kTmemCols)
                     : "memory");
    }
}

// pi~(v | prefix) at position S-1 for each prefix (sampling): cond[i][4], FP64
// (rows of hf have stride S; the row used is i*S + S-1; t = the position)
template <class R>
__global__ void k_cond_last(const uint64_t *__restrict__ x, int W, const R *__restrict__ hf, const R *__restrict__ hw,
                            const R *__restrict__ hb, int64_t n, int S, int t, int T, int d, int n_alpha, int n_beta,
                            double *__restrict__ cond, DevStatus *st) {
    __shared__ R shw[4 * kMaxHeadD];
    stage_head<R>(hw, d, shw);
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    R zr[4];
    head_logits<R>(hf + (i * S + S - 1) * d, shw, hb, d, zr);
    if (!cond_from_logits<R>(x + i * W, T, t, n_alpha, n_beta, zr, cond + i * 4)) record_status(st, NNQS_E_SECTOR, i);
}

// dz[(i*T+t)*4+v] = 1/2 dla_i ([v = x_t] - pi_v) on allowed children
template <class R>
__global__ void k_head_bwd(const R *__restrict__ pi, const uint8_t *__restrict__ tok, const double2 *__restrict__ seed,
                           int64_t n, int T, R *__restrict__ dz) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n * T * 4) return;
    const int v = (int)(idx & 3);
    const int64_t row = idx >> 2;
    const int64_t i = row / T;
    const R p = pi[idx];
    const R g = R(0.5) * (R)seed[i].x;
    dz[idx] = p > R(0) || (int)tok[row] == v ? g * (((int)tok[row] == v ? R(1) : R(0)) - p) : R(0);
}

// Head reverse mode in one pass (d = VW * cv): per row r = i*T + t,
//   dz[v] = 1/2 seed_i ([v = x_t] - pi_v) on allowed children (as k_head_bwd),
//   dh[r][c] = sum_v dz[v] hw[v][c]                       (input gradient),
// and the column sums head_w[v][c] += sum_r dz[v] hf[r][c], head_b[v] +=
// sum_r dz[v], combined in a fixed order like k_colred (row phases of a
// block, then the last block adds the blocks in block order).
template <class R, int VW>
__global__ void __launch_bounds__(kColThreads) k_head_bwd_fused(const R *__restrict__ pi, const uint8_t *__restrict__ tok,
                                                                const double2 *__restrict__ seed,
                                                                const R *__restrict__ hf, const R *__restrict__ hw,
                                                                int64_t rows, int T, int d, int64_t rows_per_block,
                                                                R *__restrict__ dh, R *__restrict__ partial,
                                                                unsigned *counter, R *__restrict__ out_w,
                                                                R *__restrict__ out_b) {
    __shared__ R sh[5 * kColThreads * VW];
    __shared__ bool last;
    const int tid = threadIdx.x;
    const int64_t r0 = blockIdx.x * rows_per_block, r1 = min(rows, r0 + rows_per_block);
    const int cv = d / VW, ct = min(cv, kColThreads), phases = kColThreads / ct;
    const int p = tid / ct, j = tid % ct;
    const int64_t pw = 4 * (int64_t)d + 4;  // partial row: head_w [4][d], head_b [4]
    for (int v0 = 0; v0 < cv; v0 += ct) {
        const int vc = v0 + j;
        const bool act = p < phases && vc < cv;
        R aw[4][VW], ab[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            ab[v] = 0;
#pragma unroll
            for (int e = 0; e < VW; ++e) aw[v][e] = 0;
        }
        if (act) {
            R w[4][VW];
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const ColVec<R, VW> wv = ld_vec<R, VW>(hw + v * d + vc * VW);
#pragma unroll
                for (int e = 0; e < VW; ++e) w[v][e] = wv.v[e];
            }
            for (int64_t r = r0 + p; r < r1; r += phases) {
                const int64_t i = r / T;
                const int tk = tok[r];
                const R gsc = R(0.5) * (R)seed[i].x;
                R dz[4];
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const R pv = pi[r * 4 + v];
                    dz[v] = pv > R(0) || tk == v ? gsc * ((tk == v ? R(1) : R(0)) - pv) : R(0);
                }
                const ColVec<R, VW> hv = ld_vec<R, VW>(hf + r * d + vc * VW);
                ColVec<R, VW> o;
#pragma unroll
                for (int e = 0; e < VW; ++e) {
                    R a = 0;
#pragma unroll
                    for (int v = 0; v < 4; ++v) a += dz[v] * w[v][e];
                    o.v[e] = a;
                }
                *reinterpret_cast<ColVec<R, VW> *>(dh + r * d + vc * VW) = o;
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    ab[v] += dz[v];
#pragma unroll
                    for (int e = 0; e < VW; ++e) aw[v][e] += dz[v] * hv.v[e];
                }
            }
        }
#pragma unroll
        for (int v = 0; v < 4; ++v)
#pragma unroll
            for (int e = 0; e < VW; ++e) sh[(v * kColThreads + tid) * VW + e] = aw[v][e];
        __syncthreads();
        if (p == 0 && vc < cv) {
            for (int v = 0; v < 4; ++v)
#pragma unroll
                for (int e = 0; e < VW; ++e) {
                    R t = 0;
                    for (int q = 0; q < phases; ++q) t += sh[(v * kColThreads + q * ct + j) * VW + e];
                    partial[blockIdx.x * pw + v * d + vc * VW + e] = t;
                }
        }
        __syncthreads();
        // head_b from the threads of vector column 0 (each row counted once)
        if (v0 == 0) {
#pragma unroll
            for (int v = 0; v < 4; ++v) sh[v * kColThreads + tid] = (act && vc == 0) ? ab[v] : R(0);
            __syncthreads();
            if (tid < 4) {
                R t = 0;
                for (int q = 0; q < phases; ++q) t += sh[tid * kColThreads + q * ct];
                partial[blockIdx.x * pw + 4 * d + tid] = t;
            }
            __syncthreads();
        }
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) last = atomicAdd(counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    sum_partial_rows<R, 1>(partial, gridDim.x, pw, 0, 4 * d, out_w, sh);
    sum_partial_rows<R, 1>(partial + 4 * d, gridDim.x, pw, 0, 4, out_b, sh);
    if (tid == 0) *counter = 0u;
}

// ------------------------------------------------------------------ phase MLP
// z1[i][u] = b1[u] + sum over occupied qubits j of W1[u][j]; r1 = relu(z1)
// blocked form: thread u of a block keeps weight column u and walks 32
// samples (bits staged in shared memory); same sum order as k_phase_in
constexpr int kPhaseRows = 32;
// w1t[j][u] = w1[u][j]: the phase layer's input weights with the hidden unit
// fastest, so a warp reads 32 consecutive units of one input
template <class R>
__global__ void k_phase_w1t(const R *__restrict__ w1, int P, int N, R *__restrict__ w1t) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= (int64_t)P * N) return;
    const int u = (int)(idx / N), j = (int)(idx % N);
    w1t[(int64_t)j * P + u] = w1[idx];
}

// kPhaseRows samples per block, thread = hidden unit u: z1 = b1 + the sum of
// w1[u][j] over the occupied qubits j of the sample, in ascending j (the sum
// k_phase_in forms); the samples' bits sit in registers, and a warp reads 32
// consecutive units of input j from the transposed weights
// samples per block: 32 (FP32), 16 (FP64), so that a thread's sums and bits
// fit in the registers of a 512-thread block
template <class R>
constexpr int phase_rows() { return sizeof(R) == 8 ? 16 : kPhaseRows; }

template <class R>
__global__ void __launch_bounds__(512) k_phase_in_blk(const uint64_t *__restrict__ x, int W, int N,
                                                      const R *__restrict__ w1t, const R *__restrict__ b1, int64_t n,
                                                      int P, R *__restrict__ z1, R *__restrict__ r1) {
    constexpr int NR = phase_rows<R>();
    __shared__ uint64_t xs[NR * 2];
    const int u = threadIdx.x;
    const int64_t i0 = blockIdx.x * (int64_t)NR;
    const int ns = (int)min((int64_t)NR, n - i0);
    for (int k = threadIdx.x; k < NR * W; k += blockDim.x) xs[k] = k < ns * W ? x[i0 * W + k] : 0ull;
    __syncthreads();
    if (u >= P) return;
    R a[NR];
    const R bu = b1[u];
#pragma unroll
    for (int k = 0; k < NR; ++k) a[k] = bu;
    for (int w = 0; w < W; ++w) {
        uint64_t xr[NR];
#pragma unroll
        for (int k = 0; k < NR; ++k) xr[k] = xs[k * W + w];
        const int jend = min(64, N - 64 * w);
        for (int j = 0; j < jend; ++j) {
            const R wj = w1t[(int64_t)(64 * w + j) * P + u];
#pragma unroll
            for (int k = 0; k < NR; ++k)
                if ((xr[k] >> j) & 1ull) a[k] += wj;
        }
    }
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        if (k >= ns) break;
        const int64_t o = (i0 + k) * P + u;
        z1[o] = a[k];
        r1[o] = a[k] > R(0) ? a[k] : R(0);
    }
}

template <class R>
__global__ void k_phase_in(const uint64_t *__restrict__ x, int W, int N, const R *__restrict__ w1,
                           const R *__restrict__ b1, int64_t n, int P, R *__restrict__ z1, R *__restrict__ r1) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n * P) return;
    const int u = (int)(idx % P);
    const int64_t i = idx / P;
    const uint64_t *xi = x + i * W;
    R a = b1[u];
    for (int j = 0; j < N; ++j)
        if (bit_of(xi, j)) a += w1[(int64_t)u * N + j];
    z1[idx] = a;
    r1[idx] = a > R(0) ? a : R(0);
}

// phase_i = b3 + sum_u r2[i][u] w3[u]  (one warp per sample)
template <class R>
__global__ void k_phase_out(const R *__restrict__ r2, const R *__restrict__ w3, const R *__restrict__ b3, int64_t n,
                            int P, double2 *__restrict__ out) {
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    R s = 0;
    for (int u = lane; u < P; u += 32) s += r2[i * P + u] * w3[u];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) out[i].y = (double)(s + b3[0]);
}

// seeds: dla, dph of the chunk as R columns
template <class R>
__global__ void k_seed_cols(const double2 *__restrict__ seed, int64_t n, R *__restrict__ dph) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) dph[i] = (R)seed[i].y;
}

// dz2 = dph_i w3[u] [z2 > 0]
// Phase output layer backward in one pass over z2 (rows [r0, r0 + rpb) of a
// block, thread = hidden unit): dz2 = dph w3 [z2 > 0] and the block's partial sums of dW3 = sum dph relu(z2),
// db2 = sum dz2 and db3 = sum dph: partial[b] = [dW3 (P) | db2 (P) | db3]
template <class R>
__global__ void k_phase_out_bwd(const R *__restrict__ dph, const R *__restrict__ w3, const R *__restrict__ z2,
                                int64_t n, int P, int64_t rpb, R *__restrict__ dz2, R *__restrict__ partial) {
    const int64_t r0 = blockIdx.x * rpb, r1 = min(n, r0 + rpb);
    const int64_t pw = 2 * (int64_t)P + 1;
    for (int u = threadIdx.x; u < P; u += blockDim.x) {
        const R wu = w3[u];
        R aw = 0, ab = 0;
#pragma unroll 4
        for (int64_t i = r0; i < r1; ++i) {
            const R g = dph[i], z = z2[i * P + u];
            const R dz = z > R(0) ? g * wu : R(0);
            dz2[i * P + u] = dz;
            aw += g * (z > R(0) ? z : R(0));
            ab += dz;
        }
        partial[blockIdx.x * pw + u] = aw;
        partial[blockIdx.x * pw + P + u] = ab;
    }
    if (threadIdx.x == 0) {
        R s3 = 0;
        for (int64_t i = r0; i < r1; ++i) s3 += dph[i];
        partial[blockIdx.x * pw + 2 * P] = s3;
    }
}

// Phase input layer weight and bias gradients from dz1 and the occupation
// bits (the 0/1 inputs): dW1[u][64 word + j] = sum_i dz1[i][u] bit_j(x_i[word]),
// db1[u] = sum_i dz1[i][u] (word 0); per block partial[b][u][65].
// grid = (row blocks, P / 64); thread = (unit u of a 64-unit slice, 16 inputs)
template <class R>
__global__ void __launch_bounds__(256) k_phase_in_bwd(const R *__restrict__ dz1, const uint64_t *__restrict__ x, int W,
                                                      int64_t n, int P, int64_t rpb, int word,
                                                      R *__restrict__ partial) {
    const int64_t r0 = blockIdx.x * rpb, r1 = min(n, r0 + rpb);
    const int jg = threadIdx.x >> 6, u = blockIdx.y * 64 + (threadIdx.x & 63);
    if (u >= P) return;
    R acc[16], ab = 0;
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[j] = 0;
#pragma unroll 4
    for (int64_t i = r0; i < r1; ++i) {
        const R v = dz1[i * P + u];
        const uint64_t m = x[i * W + word] >> (16 * jg);
#pragma unroll
        for (int j = 0; j < 16; ++j)
            if ((m >> j) & 1ull) acc[j] += v;
        ab += v;
    }
    R *pp = partial + (blockIdx.x * (int64_t)P + u) * 65;
#pragma unroll
    for (int j = 0; j < 16; ++j) pp[16 * jg + j] = acc[j];
    if (jg == 0) pp[64] = ab;
}

// out_w[u][64 word + j] += sum_b partial[b][u][j] (j < nj), out_b[u] += sum_b
// partial[b][u][64] (out_b may be null), blocks in order
template <class R>
__global__ void k_phase_in_bwd_sum(const R *__restrict__ partial, int64_t nblk, int P, int N, int word, int nj,
                                   R *__restrict__ out_w, R *__restrict__ out_b) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= (int64_t)P * 65) return;
    const int u = (int)(idx / 65), j = (int)(idx % 65);
    if (j < 64 && j >= nj) return;
    if (j == 64 && !out_b) return;
    R t = 0;
    for (int64_t b = 0; b < nblk; ++b) t += partial[b * (int64_t)P * 65 + idx];
    if (j == 64)
        out_b[u] += t;
    else
        out_w[(int64_t)u * N + 64 * word + j] += t;
}

// a[idx] *= [z > 0]  or  a[idx] *= gelu'(z)
template <class R, bool GELU>
__global__ void k_act_bwd(R *__restrict__ a, const R *__restrict__ z, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (GELU)
            a[i] *= gelu_grad_<R>(z[i]);
        else
            a[i] = z[i] > R(0) ? a[i] : R(0);
    }
}

// dX *= GELU'(Z) (act 1) or ReLU'(Z) (act 2)
template <class R>
nnqs_status act_bwd(cudaStream_t s, int act, R *dX, const R *Z, int64_t n) {
    if (act == 1) NNQS_LAUNCH("k_act_bwd", s, (k_act_bwd<R, true><<<grid_for(n, 256), 256, 0, s>>>(dX, Z, n)));
    if (act == 2) NNQS_LAUNCH("k_act_bwd", s, (k_act_bwd<R, false><<<grid_for(n, 256), 256, 0, s>>>(dX, Z, n)));
    return NNQS_OK;
}

// token-embedding gradient: out[v][c] += sum over rows whose input token is v
// of dh[row][c] (the input of position t is token t-1, the start id 4 at
// t = 0).  Laid out like k_colred: 16-byte loads, row phases added in order,
// partial[blk][5 d], the last block adds the blocks in order.
template <class R, int VW>
__global__ void __launch_bounds__(kColThreads) k_tok_grad(const R *__restrict__ dh, const uint8_t *__restrict__ tok,
                                                          int64_t rows, int T, int d, int64_t rows_per_block,
                                                          R *__restrict__ partial, unsigned *counter,
                                                          R *__restrict__ out) {
    __shared__ R sh[5 * kColThreads * VW];
    __shared__ bool last;
    const int tid = threadIdx.x;
    const int64_t r0 = blockIdx.x * rows_per_block, r1 = min(rows, r0 + rows_per_block);
    const int cv = d / VW, ct = min(cv, kColThreads), phases = kColThreads / ct;
    const int p = tid / ct, j = tid % ct;
    for (int v0 = 0; v0 < cv; v0 += ct) {
        const int vc = v0 + j;
        const bool act = p < phases && vc < cv;
        R acc[5][VW];
#pragma unroll
        for (int k = 0; k < 5; ++k)
#pragma unroll
            for (int e = 0; e < VW; ++e) acc[k][e] = 0;
        if (act) {
            int64_t r = r0 + p;
            for (; r + 3 * phases < r1; r += 4 * phases) {
                ColVec<R, VW> va[4];
                int inp[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int64_t rr = r + u * phases;
                    va[u] = ld_vec<R, VW>(dh + rr * d + vc * VW);
                    inp[u] = (rr % T == 0) ? 4 : (int)tok[rr - 1];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int k = 0; k < 5; ++k)
#pragma unroll
                        for (int e = 0; e < VW; ++e) acc[k][e] += inp[u] == k ? va[u].v[e] : R(0);
            }
            for (; r < r1; r += phases) {
                const ColVec<R, VW> va = ld_vec<R, VW>(dh + r * d + vc * VW);
                const int inp = (r % T == 0) ? 4 : (int)tok[r - 1];
#pragma unroll
                for (int k = 0; k < 5; ++k)
#pragma unroll
                    for (int e = 0; e < VW; ++e) acc[k][e] += inp == k ? va.v[e] : R(0);
            }
        }
#pragma unroll
        for (int k = 0; k < 5; ++k)
#pragma unroll
            for (int e = 0; e < VW; ++e) sh[(k * kColThreads + tid) * VW + e] = acc[k][e];
        __syncthreads();
        if (p == 0 && vc < cv) {
            for (int k = 0; k < 5; ++k)
#pragma unroll
                for (int e = 0; e < VW; ++e) {
                    R t = 0;
                    for (int q = 0; q < phases; ++q) t += sh[(k * kColThreads + q * ct + j) * VW + e];
                    partial[blockIdx.x * 5 * (int64_t)d + k * d + vc * VW + e] = t;
                }
        }
        __syncthreads();
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) last = atomicAdd(counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    sum_partial_rows<R, VW>(partial, gridDim.x, 5 * d, 0, 5 * d, out, sh);
    if (tid == 0) *counter = 0u;
}

// ------------------------------------------------------------------ orchestration
template <class R>
struct Views {  // parameter views (type R) in the converted copy
    const R *tok, *pos, *lnf_g, *lnf_b, *hw, *hb, *w1p, *b1p, *w2p, *b2p, *w3p, *b3p;
    struct L {
        const R *ln1g, *ln1b, *wqkv, *bqkv, *wo, *bo, *ln2g, *ln2b, *w1, *b1, *w2, *b2;
    };
    std::vector<L> layer;
};

template <class R>
Views<R> make_views(const nnqs_model *M, const R *p) {
    const ParamLayout &Lo = M->lay;
    Views<R> v;
    v.tok = p + Lo.tok_emb;
    v.pos = p + Lo.pos_emb;
    v.lnf_g = p + Lo.lnf_g;
    v.lnf_b = p + Lo.lnf_b;
    v.hw = p + Lo.head_w;
    v.hb = p + Lo.head_b;
    v.w1p = p + Lo.ph_w1;
    v.b1p = p + Lo.ph_b1;
    v.w2p = p + Lo.ph_w2;
    v.b2p = p + Lo.ph_b2;
    v.w3p = p + Lo.ph_w3;
    v.b3p = p + Lo.ph_b3;
    for (auto &l : Lo.layer)
        v.layer.push_back({p + l.ln1_g, p + l.ln1_b, p + l.wqkv, p + l.bqkv, p + l.wo, p + l.bo, p + l.ln2_g,
                           p + l.ln2_b, p + l.w1, p + l.b1, p + l.w2, p + l.b2});
    return v;
}

// Per-chunk activation buffers.  With `keep` every layer's tensors are
// kept for the backward; otherwise one set is reused.
template <class R>
struct Acts {
    int64_t C = 0;
    bool keep = false;
    uint8_t *tok = nullptr;
    R *hbuf = nullptr;   // keep: [L+1][C*T*d] residual stream before each layer / final
    R *hmid = nullptr;   // keep: [L][C*T*d]
    R *a = nullptr, *a2 = nullptr, *qkv = nullptr, *o = nullptr, *u = nullptr, *gu = nullptr;
    R *mean1 = nullptr, *rstd1 = nullptr, *mean2 = nullptr, *rstd2 = nullptr, *lse = nullptr;
    R *hf = nullptr, *meanf = nullptr, *rstdf = nullptr, *pi = nullptr;
    R *z1 = nullptr, *r1 = nullptr, *z2 = nullptr, *r2 = nullptr;
    R *w1t = nullptr;  // [N][P] phase input weights, unit fastest
    Scratch<R> scr{nullptr, 0, nullptr};
};

template <class R>
// lite: the fused reverse mode's keep set (the layers' inputs and mid
// residuals, the head's activations); the per-layer activations stay null
void take_acts(const nnqs_model *M, int64_t C, bool keep, Arena &a, Acts<R> &A, bool lite = false) {
    const int64_t T = M->T, d = M->d, L = M->L, F = M->F, P = M->P, rows = C * T, H = M->H;
    const int64_t Lk = keep ? L : 1;
    A.C = C;
    A.keep = keep;
    A.tok = a.take<uint8_t>(rows);
    A.hbuf = a.take<R>((keep ? (L + 1) : 2) * rows * d);
    A.hmid = a.take<R>(Lk * rows * d);
    if (!lite) {
        A.a = a.take<R>(Lk * rows * d);
        A.a2 = a.take<R>(Lk * rows * d);
        A.qkv = a.take<R>(Lk * rows * 3 * d);
        A.o = a.take<R>(Lk * rows * d);
        A.u = a.take<R>(Lk * rows * F);
        A.gu = a.take<R>(Lk * rows * F);
        A.mean1 = a.take<R>(Lk * rows);
        A.rstd1 = a.take<R>(Lk * rows);
        A.mean2 = a.take<R>(Lk * rows);
        A.rstd2 = a.take<R>(Lk * rows);
        A.lse = a.take<R>(Lk * C * H * T);
    }
    A.hf = a.take<R>(rows * d);
    A.meanf = a.take<R>(rows);
    A.rstdf = a.take<R>(rows);
    A.pi = a.take<R>(rows * 4);
    A.z1 = a.take<R>(C * P);
    A.r1 = a.take<R>(C * P);
    A.z2 = a.take<R>(C * P);
    A.r2 = a.take<R>(C * P);
    A.w1t = a.take<R>((int64_t)M->N * P);
    // split-K / column-reduction partials: enough for the largest weight
    const int64_t wmax = std::max<int64_t>({3 * d * d, F * d, P * P, P * (int64_t)M->N});
    // split-K partials of weight gradients: ~600 splits of a layer matrix
    A.scr.elems = size_t(std::max<int64_t>({8 * wmax, 4 * 152 * std::max<int64_t>(F, P) * 5, 640 * F * d}));
    A.scr.buf = a.take<R>(A.scr.elems);
    A.scr.ctr = a.take<unsigned>(64);
}

constexpr size_t kAttnSmemMax = 200 * 1024;

template <class R>
size_t attn_fwd_smem_bytes(int T, int d) { return sizeof(R) * size_t(T) * (4 * d + 8); }
template <class R>
size_t attn_bwd_smem_bytes(int T, int H, int d) { return sizeof(R) * (size_t(T) * (8 * d + 16) + 2 * size_t(H) * T); }

template <class K>
nnqs_status allow_smem(K kernel, size_t bytes) {
    if (bytes > 48 * 1024) NNQS_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    return NNQS_OK;
}

template <int DH_, class R>
nnqs_status launch_attn_fwd(cudaStream_t s, const R *qkv, R *o, R *lse, int64_t n, int T, int H, int d) {
    const size_t sm = attn_fwd_smem_bytes<R>(T, d);
    if (H * T <= 1024 && sm <= kAttnSmemMax && n > 0) {
        NNQS_TRY(allow_smem(k_attn_fwd_smem<R, DH_>, sm));
        const int threads = (H * T + 31) / 32 * 32;
        NNQS_LAUNCH("k_attn_fwd", s, k_attn_fwd_smem<R, DH_><<<(unsigned)n, threads, sm, s>>>(qkv, o, lse, T, H, d));
        return NNQS_OK;
    }
    NNQS_LAUNCH("k_attn_fwd", s, k_attn_fwd<R, DH_><<<grid_for(n * H * T, 128), 128, 0, s>>>(qkv, o, lse, n, T, H, d));
    return NNQS_OK;
}

template <class R>
nnqs_status attn_fwd(cudaStream_t s, int dh, const R *qkv, R *o, R *lse, int64_t n, int T, int H, int d) {
    switch (dh) {
        case 1: return launch_attn_fwd<1>(s, qkv, o, lse, n, T, H, d);
        case 2: return launch_attn_fwd<2>(s, qkv, o, lse, n, T, H, d);
        case 4: return launch_attn_fwd<4>(s, qkv, o, lse, n, T, H, d);
        case 8: return launch_attn_fwd<8>(s, qkv, o, lse, n, T, H, d);
        case 16: return launch_attn_fwd<16>(s, qkv, o, lse, n, T, H, d);
        case 32: return launch_attn_fwd<32>(s, qkv, o, lse, n, T, H, d);
        case 64: return launch_attn_fwd<64>(s, qkv, o, lse, n, T, H, d);
        default: return set_error(NNQS_E_UNSUPPORTED, "head dimension must be a power of two <= 64");
    }
}

template <int DH_, class R>
nnqs_status launch_attn_bwd(cudaStream_t s, const R *qkv, const R *o, const R *lse, const R *dout, R *dqkv, R *Dbuf,
                            int64_t n, int T, int H, int d, R *colsum, bool *sums) {
    *sums = false;
    // the fewest head groups whose per-CTA state fits shared memory (the
    // group width a multiple of the 16-byte vector, rows 16-byte aligned)
    constexpr int V = int(16 / sizeof(R));
    for (int G = 1; G <= H && n > 0; G *= 2) {
        if (H % G != 0) break;
        const int Hg = H / G, dg = d / G;
        if (G > 1 && (dg % V != 0 || reinterpret_cast<uintptr_t>(qkv) % 16 || reinterpret_cast<uintptr_t>(o) % 16 ||
                      reinterpret_cast<uintptr_t>(dout) % 16 || reinterpret_cast<uintptr_t>(dqkv) % 16))
            break;
        const size_t sm = attn_bwd_smem_bytes<R>(T, Hg, dg);
        if (Hg * T > 1024 || sm > kAttnSmemMax) continue;
        NNQS_TRY(allow_smem(k_attn_bwd_smem<R, DH_>, sm));
        const int threads = (Hg * T + 31) / 32 * 32;
        NNQS_LAUNCH("k_attn_bwd", s,
                    k_attn_bwd_smem<R, DH_><<<dim3((unsigned)n, (unsigned)G), threads, sm, s>>>(
                        qkv, o, lse, dout, dqkv, T, Hg, dg, colsum, H, d));
        *sums = colsum != nullptr;
        return NNQS_OK;
    }
    NNQS_LAUNCH("k_attn_bwd_q", s, k_attn_bwd_q<R, DH_><<<grid_for(n * H * T, 128), 128, 0, s>>>(qkv, o, lse, dout, dqkv, Dbuf, n, T, H, d));
    NNQS_LAUNCH("k_attn_bwd_kv", s, k_attn_bwd_kv<R, DH_><<<grid_for(n * H * T, 128), 128, 0, s>>>(qkv, lse, dout, Dbuf, dqkv, n, T, H, d));
    return NNQS_OK;
}

template <class R>
nnqs_status attn_bwd(cudaStream_t s, int dh, const R *qkv, const R *o, const R *lse, const R *dout, R *dqkv, R *Dbuf,
                     int64_t n, int T, int H, int d, R *colsum = nullptr, bool *sums = nullptr) {
    bool dummy = false;
    if (!sums) sums = &dummy;
    switch (dh) {
        case 1: return launch_attn_bwd<1>(s, qkv, o, lse, dout, dqkv, Dbuf, n, T, H, d, colsum, sums);
        case 2: return launch_attn_bwd<2>(s, qkv, o, lse, dout, dqkv, Dbuf, n, T, H, d, colsum, sums);
        case 4: return launch_attn_bwd<4>(s, qkv, o, lse, dout, dqkv, Dbuf, n, T, H, d, colsum, sums);
        case 8: return launch_attn_bwd<8>(s, qkv, o, lse, dout, dqkv, Dbuf, n, T, H, d, colsum, sums);
        case 16: return launch_attn_bwd<16>(s, qkv, o, lse, dout, dqkv, Dbuf, n, T, H, d, colsum, sums);
        case 32: return launch_attn_bwd<32>(s, qkv, o, lse, dout, dqkv, Dbuf, n, T, H, d, colsum, sums);
        case 64: return launch_attn_bwd<64>(s, qkv, o, lse, dout, dqkv, Dbuf, n, T, H, d, colsum, sums);
        default: return set_error(NNQS_E_UNSUPPORTED, "head dimension must be a power of two <= 64");
    }
}

template <class R>
nnqs_status phase_mlp(const nnqs_model *M, const Views<R> &V, const uint64_t *x, int64_t C, Acts<R> &A, double2 *out,
                      const TcWeights *tcw, cudaStream_t s);

// Forward of one chunk of C samples (x: [C][W]), writing out[C] (log|psi|, phase).
// cond != null: sampling mode -- x are prefixes of S-1 tokens, the output is
// pi~(. | prefix) at position S-1 (no phase, no log psi).
template <class R>
nnqs_status forward_chunk(const nnqs_model *M, const Views<R> &V, const uint64_t *x, int64_t C, Acts<R> &A,
                          double2 *out, DevStatus *st, int64_t row_offset, const TcWeights *tcw, cudaStream_t s,
                          int S = 0, double *cond = nullptr) {
    const int Tm = M->T, d = M->d, L = M->L, F = M->F, H = M->H, W = M->W;
    const int T = S > 0 ? S : Tm;  // sequence length of this pass
    const int64_t rows = C * T;
    if (d % 4 == 0)
        NNQS_LAUNCH("k_embed", s, k_embed_v<R><<<grid_for(rows * d / 4, 256), 256, 0, s>>>(x, W, C, T, Tm, d, V.tok, V.pos, A.hbuf, A.tok));
    else
        NNQS_LAUNCH("k_embed", s, k_embed<R><<<grid_for(rows * d, 256), 256, 0, s>>>(x, W, C, T, Tm, d, V.tok, V.pos, A.hbuf, A.tok));
    for (int l = 0; l < L; ++l) {
        const auto &Lw = V.layer[l];
        const int64_t k = A.keep ? l : 0;
        R *hin = A.keep ? A.hbuf + l * rows * d : A.hbuf;
        R *hout = A.keep ? A.hbuf + (l + 1) * rows * d : A.hbuf;
        R *hmid = A.hmid + k * rows * d;
        R *a = A.a + k * rows * d, *a2 = A.a2 + k * rows * d, *qkv = A.qkv + k * rows * 3 * d, *o = A.o + k * rows * d;
        R *u = A.u + k * rows * F, *gu = A.gu + k * rows * F;
        NNQS_TRY(ln_fwd<R>(s, hin, Lw.ln1g, Lw.ln1b, a, A.mean1 + k * rows,
                                                             A.rstd1 + k * rows, rows, d));
        if (tcw) {
            NNQS_TRY(tc_linear_fwd<R>(s, *tcw, tc_slot(l, 0), EPI_STORE, a, rows, d, Lw.bqkv, qkv, nullptr, nullptr));
        } else {
            NNQS_TRY(linear_fwd<R>(s, EPI_STORE, a, rows, d, Lw.wqkv, 3 * d, Lw.bqkv, qkv, nullptr, nullptr, A.scr));
        }
        NNQS_TRY(attn_fwd<R>(s, M->dh, qkv, o, A.lse + k * C * H * T, C, T, H, d));
        if (tcw) {
            NNQS_TRY(tc_linear_fwd<R>(s, *tcw, tc_slot(l, 1), EPI_RESID, o, rows, d, Lw.bo, hmid, nullptr, hin));
        } else {
            NNQS_TRY(linear_fwd<R>(s, EPI_RESID, o, rows, d, Lw.wo, d, Lw.bo, hmid, nullptr, hin, A.scr));
        }
        NNQS_TRY(ln_fwd<R>(s, hmid, Lw.ln2g, Lw.ln2b, a2, A.mean2 + k * rows,
                                                             A.rstd2 + k * rows, rows, d));
        if (tcw) {
            NNQS_TRY(tc_linear_fwd<R>(s, *tcw, tc_slot(l, 2), EPI_GELU, a2, rows, d, Lw.b1, u, gu, nullptr));
            NNQS_TRY(tc_linear_fwd<R>(s, *tcw, tc_slot(l, 3), EPI_RESID, gu, rows, F, Lw.b2, hout, nullptr, hmid));
        } else {
            NNQS_TRY(linear_fwd<R>(s, EPI_GELU, a2, rows, d, Lw.w1, F, Lw.b1, u, gu, nullptr, A.scr));
            NNQS_TRY(linear_fwd<R>(s, EPI_RESID, gu, rows, F, Lw.w2, d, Lw.b2, hout, nullptr, hmid, A.scr));
        }
    }
    const R *hlast = A.keep ? A.hbuf + (int64_t)L * rows * d : A.hbuf;
    NNQS_TRY(ln_fwd<R>(s, hlast, V.lnf_g, V.lnf_b, A.hf, A.meanf, A.rstdf, rows, d));
    if (cond) {
        NNQS_LAUNCH("k_cond_last", s, k_cond_last<R><<<grid_for(C, 128), 128, 0, s>>>(x, W, A.hf, V.hw, V.hb, C, T, T - 1, Tm, d, M->cfg.n_alpha, M->cfg.n_beta, cond, st));
        return NNQS_OK;
    }
    NNQS_LAUNCH("k_head", s, k_head<R><<<grid_for(C * 32, 256), 256, 0, s>>>(x, W, A.hf, V.hw, V.hb, A.tok, C, T, d, M->cfg.n_alpha,
                                                    M->cfg.n_beta, A.pi, out, st, row_offset));
    return phase_mlp<R>(M, V, x, C, A, out, tcw, s);
}

// phase MLP N -> P -> P -> 1 (ReLU) of C samples into out[i].y
template <class R>
nnqs_status phase_mlp(const nnqs_model *M, const Views<R> &V, const uint64_t *x, int64_t C, Acts<R> &A, double2 *out,
                      const TcWeights *tcw, cudaStream_t s) {
    const int P = M->P, W = M->W, N = M->N, L = M->L;
    if (P <= 512 && W <= 2 && N <= P)
    {
        constexpr int NR = phase_rows<R>();
        NNQS_LAUNCH("k_phase_in", s, k_phase_w1t<R><<<grid_for((int64_t)P * N, 256), 256, 0, s>>>(V.w1p, P, N, A.w1t));
        NNQS_LAUNCH("k_phase_in", s, k_phase_in_blk<R><<<(unsigned)((C + NR - 1) / NR), (P + 31) / 32 * 32, 0, s>>>(x, W, N, A.w1t, V.b1p, C, P, A.z1, A.r1));
    }
    else
        NNQS_LAUNCH("k_phase_in", s, k_phase_in<R><<<grid_for(C * P, 256), 256, 0, s>>>(x, W, N, V.w1p, V.b1p, C, P, A.z1, A.r1));
    if (tcw) {
        NNQS_TRY(tc_linear_fwd<R>(s, *tcw, tc_slot(L, 0), EPI_RELU, A.r1, C, P, V.b2p, A.z2, A.r2, nullptr));
    } else {
        NNQS_TRY(linear_fwd<R>(s, EPI_RELU, A.r1, C, P, V.w2p, P, V.b2p, A.z2, A.r2, nullptr, A.scr));
    }
    NNQS_LAUNCH("k_phase_out", s, k_phase_out<R><<<grid_for(C * 32, 256), 256, 0, s>>>(A.r2, V.w3p, V.b3p, C, P, out));
    return NNQS_OK;
}

// Gradient buffers for the backward of one chunk.
template <class R>
struct Grads {
    R *dh, *dtmp, *dqkv, *du, *Dbuf, *dz, *dph, *dz1, *dz2;
    R *qkvsum;    // [C][3d] per-sample column sums of dqkv (qkv bias gradient)
    R *ucolpart;  // [ceil(C T / 128)][F] column sums of du per 128-row tile (FFN-in bias gradient)
    double2 *lp;  // forward output of the recomputation (not used further)
    float *part;  // fused reverse mode: per-CTA partial gradients of one layer
};

template <class R>
void take_grads(const nnqs_model *M, int64_t C, Arena &a, Grads<R> &G, bool lite = false) {
    const int64_t T = M->T, d = M->d, F = M->F, P = M->P, rows = C * T, H = M->H;
    G.dh = a.take<R>(rows * d);
    G.dtmp = a.take<R>(rows * std::max<int64_t>(d, 4));
    if (!lite) {
        G.dqkv = a.take<R>(rows * 3 * d);
        G.du = a.take<R>(rows * F);
        G.Dbuf = a.take<R>(C * H * T);
    }
    G.dz = a.take<R>(rows * 4);
    G.dph = a.take<R>(C);
    G.dz1 = a.take<R>(C * P);
    G.dz2 = a.take<R>(C * P);
    G.lp = a.take<double2>(C);
    if (!lite) {
        G.qkvsum = a.take<R>(C * 3 * d);
        G.ucolpart = a.take<R>((rows + 127) / 128 * F);
    }
    G.part = bwd_ffn_supported(M->d, M->F) ? a.take<float>(size_t(num_sms()) * kBwdFfnPart) : nullptr;
}

// Whether the reverse mode of the decoder layers runs fused (bwd_fused.cu),
// from NNQS_FUSED_BACKWARD in the environment (read once): 0 = the
// layer-by-layer reverse mode (for comparisons), else fused where it applies
// (BF16 / split BF16 forward operands, d = 64, FFN width 256).
bool fused_bwd_enabled() {
    static const bool on = [] {
        const char *e = std::getenv("NNQS_FUSED_BACKWARD");
        return !(e && e[0] == '0');
    }();
    return on;
}

// the decoder layers' reverse mode runs fused for this model and weights
bool fused_bwd_applies(const nnqs_model *M, const TcWeights *tcw) {
    return tcw && !tcw->fp8 && fused_bwd_enabled() && bwd_ffn_supported(M->d, M->F) &&
           bwd_attn_supported(M->d, M->dh, M->T);
}

int fused_fwd_level();

// The reverse mode of precision mode tcm (tc_mode) keeps only the lite set:
// the fused forward and the fused reverse mode both apply.  The workspace
// sizes and both reverse-mode entry points decide it here.
bool reverse_lite(const nnqs_model *M, int tcm) {
    return (tcm == 1 || tcm == 2) && fused_bwd_enabled() && bwd_ffn_supported(M->d, M->F) &&
           bwd_attn_supported(M->d, M->dh, M->T) && fused_fwd_level() >= 1 &&
           fused_fwd_supported(M->d, M->F, M->dh, M->T, M->L);
}

template <class R>
nnqs_status backward_chunk(const nnqs_model *M, const Views<R> &V, const uint64_t *x, int64_t C, Acts<R> &A,
                           Grads<R> &G, const double2 *seed, R *gacc, const TcWeights *tcw, cudaStream_t s,
                           const SampleKept *kept = nullptr) {
    const int T = M->T, d = M->d, L = M->L, F = M->F, P = M->P, H = M->H, N = M->N;
    const int64_t rows = C * T;
    const ParamLayout &Lo = M->lay;
    Scratch<R> scr = A.scr;
    (void)x;
    // ---- phase MLP
    NNQS_LAUNCH("k_seed_cols", s, k_seed_cols<R><<<grid_for(C, 256), 256, 0, s>>>(seed, C, G.dph));
    // dz2, dW3 = sum_i dph_i r2[i][:], db3 = sum_i dph_i and db2 = sum_i dz2 in
    // one pass over z2 (r2 = relu(z2)), the partial rows added in block order
    {
        const int64_t pw = 2 * P + 1;
        int64_t nblk = std::min<int64_t>((C + 15) / 16, 4 * sm_count());
        nblk = std::max<int64_t>(1, std::min<int64_t>(nblk, (int64_t)(scr.elems / size_t(pw))));
        const int64_t rpb = (C + nblk - 1) / nblk;
        nblk = (C + rpb - 1) / rpb;
        NNQS_LAUNCH("k_phase_dz2", s, k_phase_out_bwd<R><<<(unsigned)nblk, 256, 0, s>>>(G.dph, V.w3p, A.z2, C, P, rpb, G.dz2, scr.buf));
        NNQS_LAUNCH("k_phase_dz2", s, (k_sum_partials<R><<<(unsigned)((P + 31) / 32), kColThreads, 0, s>>>(scr.buf, nblk, P, gacc + Lo.ph_w3, pw)));
        NNQS_LAUNCH("k_phase_dz2", s, (k_sum_partials<R><<<(unsigned)((P + 31) / 32), kColThreads, 0, s>>>(scr.buf + P, nblk, P, gacc + Lo.ph_b2, pw)));
        NNQS_LAUNCH("k_phase_dz2", s, (k_sum_partials<R><<<1, kColThreads, 0, s>>>(scr.buf + 2 * P, nblk, 1, gacc + Lo.ph_b3, pw)));
    }
    NNQS_TRY(bw_dw<R>(s, tcw, G.dz2, C, P, A.r1, P, gacc + Lo.ph_w2, scr));
    NNQS_TRY(bw_dx<R>(s, tcw, tc_slot(L, 0), G.dz2, C, P, V.w2p, P, G.dz1, scr, 2, A.z1));
    // dW1 and db1 from dz1 and the occupation bits, 64 inputs per pass
    {
        const int W = M->W;
        const int64_t ns = (P + 63) / 64;  // 64-unit slices
        int64_t nblk = std::min<int64_t>((C + 31) / 32, (8 * sm_count() + ns - 1) / ns);
        nblk = std::max<int64_t>(1, std::min<int64_t>(nblk, (int64_t)(scr.elems / size_t(P * 65))));
        const int64_t rpb = (C + nblk - 1) / nblk;
        nblk = (C + rpb - 1) / rpb;
        for (int word = 0; word < W && 64 * word < N; ++word) {
            const int nj = std::min(64, (int)N - 64 * word);
            NNQS_LAUNCH("k_phase_in_bwd", s, k_phase_in_bwd<R><<<dim3((unsigned)nblk, (unsigned)ns), 256, 0, s>>>(G.dz1, x, W, C, P, rpb, word, scr.buf));
            NNQS_LAUNCH("k_phase_in_bwd", s, k_phase_in_bwd_sum<R><<<grid_for((int64_t)P * 65, 256), 256, 0, s>>>(scr.buf, nblk, P, N, word, nj, gacc + Lo.ph_w1, word == 0 ? gacc + Lo.ph_b1 : nullptr));
        }
    }
    // ---- head
    {
        constexpr int VH = int(16 / sizeof(R));
        int64_t nblk = std::min<int64_t>((rows + 63) / 64, 2 * sm_count());
        nblk = std::max<int64_t>(1, std::min<int64_t>(nblk, (int64_t)(scr.elems / size_t(4 * d + 4))));
        const int64_t rpb = (rows + nblk - 1) / nblk;
        nblk = (rows + rpb - 1) / rpb;
        if (d % VH == 0 && al16(A.hf) && al16(V.hw) && al16(G.dtmp))
            NNQS_LAUNCH("k_head_bwd", s, (k_head_bwd_fused<R, VH><<<(unsigned)nblk, kColThreads, 0, s>>>(A.pi, A.tok, seed, A.hf, V.hw, rows, T, d, rpb, G.dtmp, scr.buf, scr.ctr, gacc + Lo.head_w, gacc + Lo.head_b)));
        else
            NNQS_LAUNCH("k_head_bwd", s, (k_head_bwd_fused<R, 1><<<(unsigned)nblk, kColThreads, 0, s>>>(A.pi, A.tok, seed, A.hf, V.hw, rows, T, d, rpb, G.dtmp, scr.buf, scr.ctr, gacc + Lo.head_w, gacc + Lo.head_b)));
    }
    // final LayerNorm
    const R *hlast = A.hbuf + (int64_t)L * rows * d;
    // dh = the final LayerNorm's input gradient (written, not added); the
    // column sums of the new dh are the last layer's FFN-out bias gradient
    NNQS_TRY(ln_bwd_sums<R>(s, hlast, A.meanf, A.rstdf, V.lnf_g, G.dtmp, G.dh, rows, d, gacc + Lo.lnf_g,
                            gacc + Lo.lnf_b, gacc + Lo.layer[L - 1].b2, scr, true));
    const bool fused_ffn = sizeof(R) == 4 && G.part && fused_bwd_applies(M, tcw);
    const bool fused_attn = fused_ffn;
    // with the sampler's tree, the fused halves read each token row's layer
    // input and mid residual from its tree node (act[node][L][2][d])
    if (kept && !fused_ffn) return set_error(NNQS_E_UNSUPPORTED, "rows from the sampler's tree need the fused reverse mode");
    BwdRowSource src{};
    if (kept) src = BwdRowSource{kept->anc, kept->stride, 2 * (int64_t)L * d, T};
    for (int l = L - 1; l >= 0; --l) {
        const auto &Lw = V.layer[l];
        const auto &Lg = Lo.layer[l];
        const R *hin = A.hbuf + (int64_t)l * rows * d;
        const R *hmid = A.hmid + (int64_t)l * rows * d;
        const R *a = A.a + (int64_t)l * rows * d, *a2 = A.a2 + (int64_t)l * rows * d;
        const R *qkv = A.qkv + (int64_t)l * rows * 3 * d, *o = A.o + (int64_t)l * rows * d;
        const R *u = A.u + (int64_t)l * rows * F, *gu = A.gu + (int64_t)l * rows * F;
        // FFN: hout = hmid + gelu(a2 W1^T + b1) W2^T + b2
        // (b2's gradient came with the LayerNorm backward that produced dh)
        bool ffn_done = false;
        if constexpr (sizeof(R) == 4) {
            if (fused_ffn) {
                const __nv_bfloat16 *tiles = static_cast<const __nv_bfloat16 *>(tcw->tiles);
                BwdFfnArgs fa{};
                fa.hmid = kept ? reinterpret_cast<const float *>(kept->act) + (2 * l + 1) * (int64_t)d
                               : reinterpret_cast<const float *>(hmid);
                fa.src = src;
                fa.dh = G.dh;
                fa.rows = rows;
                fa.ln2g = Lw.ln2g;
                fa.ln2b = Lw.ln2b;
                fa.b1 = Lw.b1;
                fa.t1 = tiles + tcw->tile_off[tc_slot(l, 2)];
                fa.t2 = tiles + tcw->tile_off[tc_slot(l, 3)];
                fa.part = G.part;
                fa.st = tcw->st;
                NNQS_TRY(bwd_ffn_launch(fa, tcw->split, s));
                NNQS_TRY(bwd_ffn_reduce(G.part, bwd_ffn_grid(rows), gacc + Lg.w1, gacc + Lg.w2, gacc + Lg.b1,
                                        gacc + Lg.ln2_g, gacc + Lg.ln2_b, gacc + Lg.bo, s));
                ffn_done = true;
            }
        }
        if (!ffn_done) {
            NNQS_TRY(bw_dw<R>(s, tcw, G.dh, rows, d, gu, F, gacc + Lg.w2, scr));
            bool ucols = false;  // column sums of du per 128-row tile, from the input-gradient epilogue
            NNQS_TRY(bw_dx<R>(s, tcw, tc_slot(l, 3), G.dh, rows, d, Lw.w2, F, G.du, scr, 1, u, G.ucolpart, &ucols));
            NNQS_TRY(bw_dw<R>(s, tcw, G.du, rows, F, a2, d, gacc + Lg.w1, scr));
            if (ucols)
                NNQS_TRY(colsum<R>(s, 0, G.ucolpart, nullptr, nullptr, nullptr, (rows + 127) / 128, F, gacc + Lg.b1,
                                   nullptr, scr));
            else
                NNQS_TRY(colsum<R>(s, 0, G.du, nullptr, nullptr, nullptr, rows, F, gacc + Lg.b1, nullptr, scr));
            NNQS_TRY(bw_dx<R>(s, tcw, tc_slot(l, 2), G.du, rows, F, Lw.w1, d, G.dtmp, scr));
            NNQS_TRY(ln_bwd_sums<R>(s, hmid, A.mean2 + l * rows, A.rstd2 + l * rows, Lw.ln2g, G.dtmp, G.dh, rows, d,
                                    gacc + Lg.ln2_g, gacc + Lg.ln2_b, gacc + Lg.bo, scr));
        }
        // attention: hmid = hin + attn(a) Wo^T + bo
        if constexpr (sizeof(R) == 4) {
            if (fused_attn) {
                const __nv_bfloat16 *tiles = static_cast<const __nv_bfloat16 *>(tcw->tiles);
                BwdAttnArgs aa{};
                aa.hin = kept ? reinterpret_cast<const float *>(kept->act) + 2 * l * (int64_t)d
                              : reinterpret_cast<const float *>(hin);
                aa.src = src;
                aa.dh = G.dh;
                aa.n = C;
                aa.T = T;
                aa.spt = 128 / T;
                aa.ln1g = Lw.ln1g;
                aa.ln1b = Lw.ln1b;
                aa.bqkv = Lw.bqkv;
                aa.tqkv = tiles + tcw->tile_off[tc_slot(l, 0)];
                aa.to = tiles + tcw->tile_off[tc_slot(l, 1)];
                aa.part = G.part;
                aa.st = tcw->st;
                NNQS_TRY(bwd_attn_launch(aa, tcw->split, M->dh, s));
                NNQS_TRY(bwd_attn_reduce(G.part, bwd_attn_grid(C, T), gacc + Lg.wqkv, gacc + Lg.wo, gacc + Lg.bqkv,
                                         gacc + Lg.ln1_g, gacc + Lg.ln1_b, l > 0 ? gacc + Lo.layer[l - 1].b2 : nullptr,
                                         s));
                continue;
            }
        }
        NNQS_TRY(bw_dw<R>(s, tcw, G.dh, rows, d, o, d, gacc + Lg.wo, scr));
        NNQS_TRY(bw_dx<R>(s, tcw, tc_slot(l, 1), G.dh, rows, d, Lw.wo, d, G.dtmp, scr));
        bool qsums = false;
        NNQS_TRY(attn_bwd<R>(s, M->dh, qkv, o, A.lse + (int64_t)l * C * H * T, G.dtmp, G.dqkv, G.Dbuf, C, T, H, d,
                             G.qkvsum, &qsums));
        NNQS_TRY(bw_dw<R>(s, tcw, G.dqkv, rows, 3 * d, a, d, gacc + Lg.wqkv, scr));
        // qkv bias: per-sample sums from the attention kernel, else the rows
        if (qsums)
            NNQS_TRY(colsum<R>(s, 0, G.qkvsum, nullptr, nullptr, nullptr, C, 3 * d, gacc + Lg.bqkv, nullptr, scr));
        else
            NNQS_TRY(colsum<R>(s, 0, G.dqkv, nullptr, nullptr, nullptr, rows, 3 * d, gacc + Lg.bqkv, nullptr, scr));
        NNQS_TRY(bw_dx<R>(s, tcw, tc_slot(l, 0), G.dqkv, rows, 3 * d, Lw.wqkv, d, G.dtmp, scr));
        NNQS_TRY(ln_bwd_sums<R>(s, hin, A.mean1 + l * rows, A.rstd1 + l * rows, Lw.ln1g, G.dtmp, G.dh, rows, d,
                                gacc + Lg.ln1_g, gacc + Lg.ln1_b, l > 0 ? gacc + Lo.layer[l - 1].b2 : nullptr, scr));
    }
    // embeddings: pos[t][c] += sum_i dh[i][t][c]; tok[v][c] += sum over inputs v
    NNQS_TRY(colsum<R>(s, 0, G.dh, nullptr, nullptr, nullptr, C, T * d, gacc + Lo.pos_emb, nullptr, scr));
    {
        int64_t nblk = std::min<int64_t>((rows + 63) / 64, 2 * sm_count());
        nblk = std::max<int64_t>(1, std::min<int64_t>(nblk, (int64_t)(scr.elems / size_t(5 * d))));
        const int64_t rpb = (rows + nblk - 1) / nblk;
        nblk = (rows + rpb - 1) / rpb;
        constexpr int V = int(16 / sizeof(R));
        if (d % V == 0 && reinterpret_cast<uintptr_t>(G.dh) % 16 == 0)
            NNQS_LAUNCH("k_tok_grad", s, (k_tok_grad<R, V><<<(unsigned)nblk, kColThreads, 0, s>>>(G.dh, A.tok, rows, T, d, rpb, scr.buf, scr.ctr, gacc + Lo.tok_emb)));
        else
            NNQS_LAUNCH("k_tok_grad", s, (k_tok_grad<R, 1><<<(unsigned)nblk, kColThreads, 0, s>>>(G.dh, A.tok, rows, T, d, rpb, scr.buf, scr.ctr, gacc + Lo.tok_emb)));
    }
    return NNQS_OK;
}

template <class R>
__global__ void k_grad_out(const R *__restrict__ g, int64_t n, double *__restrict__ g64, float *__restrict__ g32) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (g64) g64[i] = (double)g[i];
        if (g32) g32[i] = (float)g[i];
    }
}

// samples per chunk: keep the saved activations within ~6 GB
int64_t chunk_for(const nnqs_model *M, int64_t n, size_t rbytes, bool backward) {
    const int64_t per = (int64_t)rbytes * M->T * M->d * (backward ? (16 * M->L + 12) : 12) +
                        (int64_t)rbytes * 5 * M->P;
    const int64_t budget = backward ? (int64_t(16) << 30) : (int64_t(3) << 30);
    int64_t c = std::max<int64_t>(256, budget / std::max<int64_t>(per, 1));
    c = std::min<int64_t>(c, 32768);
    return std::max<int64_t>(1, std::min(c, n));
}

template <class R>
size_t workspace_impl(const nnqs_model *M, int64_t n, bool backward, int tcm) {
    Arena a(nullptr);
    a.take<char>(kStatusBytes);
    a.take<R>(M->lay.total);  // converted parameters
    if (backward) a.take<R>(M->lay.total);  // gradient accumulator
    if (tcm) tc_weights_take(M, a);
    const int64_t C = chunk_for(M, std::max<int64_t>(n, 1), sizeof(R), backward);
    const bool lite = backward && sizeof(R) == 4 && reverse_lite(M, tcm);
    Acts<R> A;
    take_acts<R>(M, C, backward, a, A, lite);
    if (backward) {
        Grads<R> G;
        take_grads<R>(M, C, a, G, lite);
    }
    return a.used + 1024;
}

// Which forwards run fused (fwd_fused.cu), from NNQS_FUSED_FORWARD in the
// environment (read once): 0 = none (the layer-by-layer forward everywhere,
// for comparisons), 1 = log psi only (nnqs_logpsi, exact mode; the default),
// 2 = also the reverse mode's forward, with its activations written out.
int fused_fwd_level() {
    static const int level = [] {
        const char *e = std::getenv("NNQS_FUSED_FORWARD");
        if (!e || !e[0]) return 1;
        return e[0] == '0' ? 0 : e[0] == '2' ? 2 : 1;
    }();
    return level;
}
bool fused_fwd_enabled() { return fused_fwd_level() >= 1; }

// arguments of the fused forward for C samples x (FP32 parameters V, BF16
// weight images of tcw)
FusedFwdArgs fused_args(const nnqs_model *M, const Views<float> &V, const TcWeights &tcw, const uint64_t *x,
                        int64_t C, double2 *out, DevStatus *st, int64_t row_offset) {
    FusedFwdArgs a{};
    a.x = x;
    a.n = C;
    a.W = M->W;
    a.T = M->T;
    a.L = M->L;
    a.n_alpha = M->cfg.n_alpha;
    a.n_beta = M->cfg.n_beta;
    a.spt = 128 / M->T;
    a.n_tiles = (C + a.spt - 1) / a.spt;
    a.tok = V.tok;
    a.pos = V.pos;
    a.lnf_g = V.lnf_g;
    a.lnf_b = V.lnf_b;
    a.hw = V.hw;
    a.hb = V.hb;
    const __nv_bfloat16 *tiles = static_cast<const __nv_bfloat16 *>(tcw.tiles);
    for (int l = 0; l < M->L; ++l) {
        const auto &Lw = V.layer[l];
        a.ln1g[l] = Lw.ln1g;
        a.ln1b[l] = Lw.ln1b;
        a.bqkv[l] = Lw.bqkv;
        a.bo[l] = Lw.bo;
        a.ln2g[l] = Lw.ln2g;
        a.ln2b[l] = Lw.ln2b;
        a.b1[l] = Lw.b1;
        a.b2[l] = Lw.b2;
        a.tqkv[l] = tiles + tcw.tile_off[tc_slot(l, 0)];
        a.to[l] = tiles + tcw.tile_off[tc_slot(l, 1)];
        a.t1[l] = tiles + tcw.tile_off[tc_slot(l, 2)];
        a.t2[l] = tiles + tcw.tile_off[tc_slot(l, 3)];
    }
    a.out = out;
    a.st = st;
    a.row_offset = row_offset;
    return a;
}

// Forward of C samples keeping every activation for the reverse mode: the
// fused kernel in keep mode where it applies (BF16 / split BF16, d = 64),
// else the layer-by-layer forward.
template <class R>
nnqs_status forward_keep(const nnqs_model *M, const Views<R> &V, const uint64_t *x, int64_t C, Acts<R> &A,
                         double2 *out, DevStatus *st, int64_t row_offset, const TcWeights *tcw, cudaStream_t s) {
    if constexpr (sizeof(R) == 4) {
        // the fused reverse mode recomputes each layer from its input and
        // hmid: the fused forward then writes only those (and the head's)
        // (a workspace without the per-layer activations, A.a null, holds only those)
        const bool lite = !A.a || fused_bwd_applies(M, tcw);
        if (!A.a && !(tcw && fused_fwd_supported(M->d, M->F, M->dh, M->T, M->L)))
            return set_error(NNQS_E_INVAL, "lite reverse-mode workspace without the fused forward");
        if (tcw && !tcw->fp8 && A.keep && (fused_fwd_level() >= 2 || (lite && fused_fwd_level() >= 1)) &&
            fused_fwd_supported(M->d, M->F, M->dh, M->T, M->L)) {
            FusedFwdArgs a = fused_args(M, V, *tcw, x, C, out, st, row_offset);
            if (!fused_fwd_aligned(a)) {
                if (!A.a) return set_error(NNQS_E_INVAL, "fused forward: parameters not 16-byte aligned");
                return forward_chunk<R>(M, V, x, C, A, out, st, row_offset, tcw, s);
            }
            a.rows = C * M->T;
            a.hbuf = A.hbuf;
            a.hmid = A.hmid;
            if (!lite) {
                a.a = A.a;
                a.a2 = A.a2;
                a.o = A.o;
                a.qkv = A.qkv;
                a.u = A.u;
                a.gu = A.gu;
                a.mean1 = A.mean1;
                a.rstd1 = A.rstd1;
                a.mean2 = A.mean2;
                a.rstd2 = A.rstd2;
                a.lse = A.lse;
            }
            a.hf = A.hf;
            a.meanf = A.meanf;
            a.rstdf = A.rstdf;
            a.pi = A.pi;
            a.tok_out = A.tok;
            NNQS_TRY(fused_fwd_launch(a, tcw->split, M->dh, s));
            return phase_mlp<R>(M, V, x, C, A, out, tcw, s);
        }
    }
    return forward_chunk<R>(M, V, x, C, A, out, st, row_offset, tcw, s);
}

template <class R>
nnqs_status forward_impl(const nnqs_model *M, const float *params, const uint64_t *x, int64_t n, double *out, Arena &ws,
                         DevStatus *st, int tcm, cudaStream_t s) {
    const bool tensor = tcm != 0;
    R *pr = ws.take<R>(M->lay.total);
    TcWeights tcw{};
    if (tensor) tc_weights_take(M, ws, &tcw);
    tcw.st = st;
    tcw.split = tcm == 2;
    tcw.fp8 = tcm == 3;
    const int64_t C = chunk_for(M, n, sizeof(R), false);
    Acts<R> A;
    take_acts<R>(M, C, false, ws, A);
    NNQS_LAUNCH("k_convert_params", s, k_convert_params<R><<<grid_for(M->lay.total, 256), 256, 0, s>>>(params, pr, M->lay.total));
    if (tensor) NNQS_TRY(tc_weights_prepare(M, params, tcw, s));
    const Views<R> V = make_views<R>(M, pr);
    // BF16 (split or not) with d = 64: the whole transformer of a 128-row
    // tile in one persistent kernel (fwd_fused.cu); the phase MLP after it
    const bool fused = tensor && !tcw.fp8 && sizeof(R) == 4 && fused_fwd_enabled() &&
                       fused_fwd_supported(M->d, M->F, M->dh, M->T, M->L);
    for (int64_t c0 = 0; c0 < n; c0 += C) {
        const int64_t cn = std::min(C, n - c0);
        double2 *oc = reinterpret_cast<double2 *>(out) + c0;
        if constexpr (sizeof(R) == 4) {
            if (fused) {
                const FusedFwdArgs fa = fused_args(M, V, tcw, x + c0 * M->W, cn, oc, st, c0);
                if (fused_fwd_aligned(fa)) {
                    NNQS_TRY(fused_fwd_launch(fa, tcw.split, M->dh, s));
                    NNQS_TRY(phase_mlp<R>(M, V, x + c0 * M->W, cn, A, oc, &tcw, s));
                    continue;
                }
            }
        }
        NNQS_TRY(forward_chunk<R>(M, V, x + c0 * M->W, cn, A, oc, st, c0, tensor ? &tcw : nullptr, s));
    }
    return NNQS_OK;
}

template <class R>
nnqs_status backward_impl(const nnqs_model *M, const float *params, const uint64_t *x, int64_t n, const double *seed,
                          double *g64, float *g32, Arena &ws, DevStatus *st, int tcm, cudaStream_t s) {
    const bool tensor = tcm != 0;
    R *pr = ws.take<R>(M->lay.total);
    R *gacc = ws.take<R>(M->lay.total);
    TcWeights tcw{};
    if (tensor) tc_weights_take(M, ws, &tcw);
    tcw.st = st;
    tcw.split = tcm == 2;
    tcw.fp8 = tcm == 3;
    const int64_t C = chunk_for(M, std::max<int64_t>(n, 1), sizeof(R), true);
    const bool lite = sizeof(R) == 4 && reverse_lite(M, tcm);
    Acts<R> A;
    take_acts<R>(M, C, true, ws, A, lite);
    Grads<R> G;
    take_grads<R>(M, C, ws, G, lite);
    NNQS_CUDA_TRY(cudaMemsetAsync(A.scr.ctr, 0, sizeof(unsigned), s));
    NNQS_LAUNCH("k_convert_params", s, k_convert_params<R><<<grid_for(M->lay.total, 256), 256, 0, s>>>(params, pr, M->lay.total));
    NNQS_LAUNCH("k_fill", s, k_fill<R><<<grid_for(M->lay.total, 256), 256, 0, s>>>(gacc, M->lay.total, R(0)));
    if (tensor) NNQS_TRY(tc_weights_prepare(M, params, tcw, s));
    const Views<R> V = make_views<R>(M, pr);
    for (int64_t c0 = 0; c0 < n; c0 += C) {
        const int64_t cn = std::min(C, n - c0);
        const uint64_t *xc = x + c0 * M->W;
        // recompute the forward (tensor cores for NNQS_MIXED), keeping activations
        NNQS_TRY(forward_keep<R>(M, V, xc, cn, A, G.lp, st, c0, tensor ? &tcw : nullptr, s));
        NNQS_TRY(backward_chunk<R>(M, V, xc, cn, A, G, reinterpret_cast<const double2 *>(seed) + c0, gacc,
                                   tensor ? &tcw : nullptr, s));
    }
    NNQS_LAUNCH("k_grad_out", s, k_grad_out<R><<<grid_for(M->lay.total, 256), 256, 0, s>>>(gacc, M->lay.total, g64, g32));
    return NNQS_OK;
}

// forward with the activations kept, then `between` (which fills `seed`),
// then the reverse mode on those activations: one forward instead of two
template <class R>
nnqs_status fwd_bwd_impl(const nnqs_model *M, const float *params, const uint64_t *x, int64_t n, double *lp_out,
                         const double *seed, double *g64, float *g32, Arena &ws, DevStatus *st, int tcm,
                         cudaStream_t s, const std::function<nnqs_status()> &between) {
    const bool tensor = tcm != 0;
    R *pr = ws.take<R>(M->lay.total);
    R *gacc = ws.take<R>(M->lay.total);
    TcWeights tcw{};
    if (tensor) tc_weights_take(M, ws, &tcw);
    tcw.st = st;
    tcw.split = tcm == 2;
    tcw.fp8 = tcm == 3;
    const int64_t C = chunk_for(M, std::max<int64_t>(n, 1), sizeof(R), true);
    if (C < n) return set_error(NNQS_E_INVAL, "fused forward/backward needs one chunk");
    const bool lite = sizeof(R) == 4 && reverse_lite(M, tcm);
    Acts<R> A;
    take_acts<R>(M, C, true, ws, A, lite);
    Grads<R> G;
    take_grads<R>(M, C, ws, G, lite);
    NNQS_CUDA_TRY(cudaMemsetAsync(A.scr.ctr, 0, sizeof(unsigned), s));
    NNQS_LAUNCH("k_convert_params", s, k_convert_params<R><<<grid_for(M->lay.total, 256), 256, 0, s>>>(params, pr, M->lay.total));
    NNQS_LAUNCH("k_fill", s, k_fill<R><<<grid_for(M->lay.total, 256), 256, 0, s>>>(gacc, M->lay.total, R(0)));
    if (tensor) NNQS_TRY(tc_weights_prepare(M, params, tcw, s));
    const Views<R> V = make_views<R>(M, pr);
    NNQS_TRY(forward_keep<R>(M, V, x, n, A, reinterpret_cast<double2 *>(lp_out), st, 0, tensor ? &tcw : nullptr, s));
    NNQS_TRY(between());
    NNQS_TRY(backward_chunk<R>(M, V, x, n, A, G, reinterpret_cast<const double2 *>(seed), gacc,
                               tensor ? &tcw : nullptr, s));
    NNQS_LAUNCH("k_grad_out", s, k_grad_out<R><<<grid_for(M->lay.total, 256), 256, 0, s>>>(gacc, M->lay.total, g64, g32));
    return NNQS_OK;
}

template <class R>
size_t cond_workspace_impl(const nnqs_model *M, int64_t max_prefixes, bool tensor, int64_t kv_nodes) {
    Arena a(nullptr);
    a.take<R>(M->lay.total);
    a.take<R>(size_t(kv_nodes) * M->L * 3 * M->d);
    if (tensor) tc_weights_take(M, a);
    const int64_t C = chunk_for(M, std::max<int64_t>(max_prefixes, 1), sizeof(R), false);
    Acts<R> A;
    take_acts<R>(M, C, false, a, A);
    return a.used + 1024;
}

}  // namespace

template <int DH_, class R>
nnqs_status launch_attn_decode(cudaStream_t s, const R *pool, const int32_t *anc, int64_t anc_stride, int64_t g0, int64_t n, int t,
                               int L, int l, int H, int d, R *o) {
    NNQS_LAUNCH("k_attn_decode", s,
                k_attn_decode<R, DH_><<<grid_for(n * H, 128), 128, 0, s>>>(pool, anc, anc_stride, g0, n, t, L, l, H, d, o));
    return NNQS_OK;
}

template <class R>
nnqs_status attn_decode(cudaStream_t s, int dh, const R *pool, const int32_t *anc, int64_t anc_stride, int64_t g0, int64_t n, int t,
                        int L, int l, int H, int d, R *o) {
    switch (dh) {
        case 1: return launch_attn_decode<1>(s, pool, anc, anc_stride, g0, n, t, L, l, H, d, o);
        case 2: return launch_attn_decode<2>(s, pool, anc, anc_stride, g0, n, t, L, l, H, d, o);
        case 4: return launch_attn_decode<4>(s, pool, anc, anc_stride, g0, n, t, L, l, H, d, o);
        case 8: return launch_attn_decode<8>(s, pool, anc, anc_stride, g0, n, t, L, l, H, d, o);
        case 16: return launch_attn_decode<16>(s, pool, anc, anc_stride, g0, n, t, L, l, H, d, o);
        case 32: return launch_attn_decode<32>(s, pool, anc, anc_stride, g0, n, t, L, l, H, d, o);
        case 64: return launch_attn_decode<64>(s, pool, anc, anc_stride, g0, n, t, L, l, H, d, o);
        default: return set_error(NNQS_E_UNSUPPORTED, "head dimension must be a power of two <= 64");
    }
}

// one decoding step for C prefixes at depth t (global node ids g0 ...)
bool decode_fused_ok(const nnqs_model *M, const TcWeights &w) {
    if (M->d != dec::kD || M->F != dec::kF || (M->dh != 8 && M->dh != 16) || M->L > kDecMaxLayers) return false;
    for (int l = 0; l < M->L; ++l) {
        if (w.pcols[tc_slot(l, 0)] != 64 || w.pcols[tc_slot(l, 1)] != 64 || w.pcols[tc_slot(l, 2)] != 64 ||
            w.pcols[tc_slot(l, 3)] != 256)
            return false;
    }
    return true;
}

template <bool SPLIT, int DH>
nnqs_status launch_decode_step(const DecodeArgs &g, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        NNQS_CUDA_TRY(cudaFuncSetAttribute(k_decode_step<SPLIT, DH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           dec::kSmem));
        attr = true;
    }
    // device-side counts: enough CTAs for any n <= g.n (the capacity)
    const unsigned grid = g.n_dev ? (unsigned)std::max<int64_t>(g.n_sms, (g.n + dec::kRows - 1) / dec::kRows)
                                  : (unsigned)((g.n + g.rpc - 1) / g.rpc);
    NNQS_LAUNCH("k_decode_step", s, (k_decode_step<SPLIT, DH><<<grid, dec::kThreads, dec::kSmem, s>>>(g)));
    return NNQS_OK;
}

// the four GEMMs of every layer of one fused decoding step over n prefixes at
// depth t (method FLOPs) and its bytes: per layer and prefix the keys and
// values of its t ancestors and itself read, its q | k | v row written, and
// the weight images once
// method FLOPs of the step's products; bytes: per row and layer the keys and
// values of its t + 1 ancestors (itself included) read and its own k|v row
// written, and the layer's BF16 weight images
void note_decode_work(int64_t n, bool split, int L, int t) {
    note_work("k_decode_step", L * 2.0 * double(n) * (4.0 * dec::kD * dec::kD + 2.0 * dec::kD * dec::kF),
              L * (double(n) * 4.0 * (2.0 * dec::kD * (t + 1) + 2.0 * dec::kD) +
                   2.0 * (split ? 2.0 : 1.0) * (4.0 * dec::kD * dec::kD + 2.0 * dec::kD * dec::kF)));
}

// One decoding step of all layers for n prefixes at depth t (global node ids
// g0 ...): the embeddings of their last tokens in, the conditionals of the
// next token out (k_decode_step)
nnqs_status decode_step_fused(const nnqs_model *M, const Views<float> &V, const TcWeights &w, const uint64_t *x,
                              int64_t n, float *pool, const int32_t *anc, int64_t anc_stride, int t, int64_t g0,
                              double *cond, DevStatus *st, cudaStream_t s, const int64_t *n_dev = nullptr,
                              const int64_t *g0_dev = nullptr, float *act = nullptr, float *fin = nullptr) {
    if (n == 0) return NNQS_OK;
    DecodeArgs g{};
    g.n = n;
    g.n_dev = n_dev;
    g.g0_dev = g0_dev;
    g.n_sms = sm_count();
    // prefixes per CTA: once there are more prefixes than SMs every SM gets a
    // CTA (the late steps' attention is bound by memory traffic; the MMA
    // tiles stay 128 rows, the rows past rpc idle)
    g.rpc = (int)std::min<int64_t>(dec::kRows, std::max<int64_t>(1, (n + sm_count() - 1) / sm_count()));
    g.pool = pool;
    g.L = M->L;
    g.Tm = M->T;
    g.t = t;
    g.g0 = g0;
    g.anc = anc;
    g.anc_stride = anc_stride;
    const __nv_bfloat16 *tiles = static_cast<const __nv_bfloat16 *>(w.tiles);
    for (int l = 0; l < M->L; ++l) {
        const auto &Lw = V.layer[l];
        g.ln1g[l] = Lw.ln1g;
        g.ln1b[l] = Lw.ln1b;
        g.ln2g[l] = Lw.ln2g;
        g.ln2b[l] = Lw.ln2b;
        g.bqkv[l] = Lw.bqkv;
        g.bo[l] = Lw.bo;
        g.b1[l] = Lw.b1;
        g.b2[l] = Lw.b2;
        g.tqkv[l] = tiles + w.tile_off[tc_slot(l, 0)];
        g.to[l] = tiles + w.tile_off[tc_slot(l, 1)];
        g.t1[l] = tiles + w.tile_off[tc_slot(l, 2)];
        g.t2[l] = tiles + w.tile_off[tc_slot(l, 3)];
    }
    g.x = x;
    g.W = M->W;
    g.n_alpha = M->cfg.n_alpha;
    g.n_beta = M->cfg.n_beta;
    g.tok_emb = V.tok;
    g.pos_emb = V.pos;
    g.lnf_g = V.lnf_g;
    g.lnf_b = V.lnf_b;
    g.hw = V.hw;
    g.hb = V.hb;
    g.cond = cond;
    g.st = st;
    g.act = act;
    g.fin = fin;
    // work per launch (for the profile); with the level size on the device
    // the walk notes it once the size is known (n is the capacity here)
    if (!n_dev) note_decode_work(n, w.split, M->L, t);
    if (w.split) return M->dh == 8 ? launch_decode_step<true, 8>(g, s) : launch_decode_step<true, 16>(g, s);
    return M->dh == 8 ? launch_decode_step<false, 8>(g, s) : launch_decode_step<false, 16>(g, s);
}

template <class R>
nnqs_status decode_chunk(const nnqs_model *M, const Views<R> &V, const uint64_t *x, int64_t C, int t, int64_t g0,
                         R *pool, const int32_t *anc, int64_t anc_stride, Acts<R> &A, double *cond, DevStatus *st,
                         const TcWeights *tcw, cudaStream_t s) {
    const int T = M->T, d = M->d, L = M->L, F = M->F, H = M->H, W = M->W;
    const int64_t rows = C;
    R *h = A.hbuf;
    if constexpr (sizeof(R) == 4) {
        // fused: embedding in the first layer, conditionals in the last
        if (tcw && decode_fused_ok(M, *tcw))
            return decode_step_fused(M, V, *tcw, x, C, pool, anc, anc_stride, t, g0, cond, st, s);
    }
    NNQS_LAUNCH("k_embed", s, k_embed_decode<R><<<grid_for(rows * d, 256), 256, 0, s>>>(x, W, C, t, T, d, V.tok, V.pos, h));
    for (int l = 0; l < L; ++l) {
        const auto &Lw = V.layer[l];
        R *qkv = pool + (g0 * L + l) * 3 * (int64_t)d;
        NNQS_TRY(ln_fwd<R>(s, h, Lw.ln1g, Lw.ln1b, A.a, nullptr, nullptr, rows, d));
        if (tcw) {
            NNQS_TRY(tc_linear_fwd_ld<R>(s, *tcw, tc_slot(l, 0), EPI_STORE, A.a, rows, d, Lw.bqkv, qkv, (int64_t)L * 3 * d,
                                         nullptr, nullptr));
        } else {
            NNQS_TRY(gemm<R>(s, EPI_STORE, A.a, d, 1, Lw.wqkv, d, 1, qkv, (int64_t)L * 3 * d, nullptr, Lw.bqkv, nullptr,
                             rows, 3 * d, d, A.scr));
        }
        NNQS_TRY(attn_decode<R>(s, M->dh, pool, anc, anc_stride, g0, C, t, L, l, H, d, A.o));
        if (tcw) {
            NNQS_TRY(tc_linear_fwd<R>(s, *tcw, tc_slot(l, 1), EPI_RESID, A.o, rows, d, Lw.bo, h, nullptr, h));
        } else {
            NNQS_TRY(linear_fwd<R>(s, EPI_RESID, A.o, rows, d, Lw.wo, d, Lw.bo, h, nullptr, h, A.scr));
        }
        NNQS_TRY(ln_fwd<R>(s, h, Lw.ln2g, Lw.ln2b, A.a2, nullptr, nullptr, rows, d));
        if (tcw) {
            NNQS_TRY(tc_linear_fwd<R>(s, *tcw, tc_slot(l, 2), EPI_GELU, A.a2, rows, d, Lw.b1, A.u, A.gu, nullptr));
            NNQS_TRY(tc_linear_fwd<R>(s, *tcw, tc_slot(l, 3), EPI_RESID, A.gu, rows, F, Lw.b2, h, nullptr, h));
        } else {
            NNQS_TRY(linear_fwd<R>(s, EPI_GELU, A.a2, rows, d, Lw.w1, F, Lw.b1, A.u, A.gu, nullptr, A.scr));
            NNQS_TRY(linear_fwd<R>(s, EPI_RESID, A.gu, rows, F, Lw.w2, d, Lw.b2, h, nullptr, h, A.scr));
        }
    }
    NNQS_TRY(ln_fwd<R>(s, h, V.lnf_g, V.lnf_b, A.hf, nullptr, nullptr, rows, d));
    NNQS_LAUNCH("k_cond_last", s, k_cond_last<R><<<grid_for(C, 128), 128, 0, s>>>(x, W, A.hf, V.hw, V.hb, C, 1, t, T, d,
                                                                             M->cfg.n_alpha, M->cfg.n_beta, cond, st));
    return NNQS_OK;
}

struct CondCtx {
    int prec = NNQS_FP64;
    bool tensor = false;
    void *params = nullptr;  // converted copy (double or float)
    int64_t C = 0;
    TcWeights tcw;
    Acts<float> Af;
    Acts<double> Ad;
    void *pool = nullptr;  // key/value cache [nodes][L][3d]
    int64_t pool_nodes = 0;
    int64_t anc_stride = 0;  // rows of the depth-major ancestor tables (the prefix capacity)
};

size_t cond_workspace(const nnqs_model *M, int64_t max_prefixes, int prec, int64_t kv_nodes) {
    if (prec == NNQS_FP64) return cond_workspace_impl<double>(M, max_prefixes, false, kv_nodes);
    return cond_workspace_impl<float>(M, max_prefixes, tc_mode(prec) != 0, kv_nodes);
}

nnqs_status cond_create(const nnqs_model *M, const float *params, int prec, int64_t max_prefixes, int64_t kv_nodes,
                        Arena &ws, CondCtx **out, cudaStream_t s) {
    CondCtx *c = new (std::nothrow) CondCtx();
    if (!c) return set_error(NNQS_E_NOMEM, "host allocation failed");
    *out = c;
    c->prec = prec;
    c->tensor = tc_mode(prec) != 0;
    c->pool_nodes = kv_nodes;
    c->anc_stride = max_prefixes;
    if (prec == NNQS_FP64) {
        double *pr = ws.take<double>(M->lay.total);
        c->pool = ws.take<double>(size_t(kv_nodes) * M->L * 3 * M->d);
        c->params = pr;
        c->C = chunk_for(M, std::max<int64_t>(max_prefixes, 1), sizeof(double), false);
        take_acts<double>(M, c->C, false, ws, c->Ad);
        NNQS_LAUNCH("k_convert_params", s, k_convert_params<double><<<grid_for(M->lay.total, 256), 256, 0, s>>>(params, pr, M->lay.total));
    } else {
        float *pr = ws.take<float>(M->lay.total);
        c->pool = ws.take<float>(size_t(kv_nodes) * M->L * 3 * M->d);
        c->params = pr;
        if (c->tensor) tc_weights_take(M, ws, &c->tcw);
        c->tcw.split = tc_mode(prec) == 2;
        c->tcw.fp8 = false;  // NNQS_FP8 samples with BF16 operands (as NNQS_MIXED)
        c->C = chunk_for(M, std::max<int64_t>(max_prefixes, 1), sizeof(float), false);
        take_acts<float>(M, c->C, false, ws, c->Af);
        NNQS_LAUNCH("k_convert_params", s, k_convert_params<float><<<grid_for(M->lay.total, 256), 256, 0, s>>>(params, pr, M->lay.total));
        if (c->tensor) NNQS_TRY(tc_weights_prepare(M, params, c->tcw, s));
    }
    NNQS_CUDA_TRY(cudaGetLastError());
    return NNQS_OK;
}

void cond_destroy(CondCtx *c) { delete c; }

nnqs_status cond_step_cached(const nnqs_model *M, CondCtx *ctx, const uint64_t *prefixes, int64_t n, int t,
                             int64_t g0, const int32_t *anc, double *cond, DevStatus *st, cudaStream_t s) {
    if (t >= kMaxDepth) return set_error(NNQS_E_UNSUPPORTED, "more than 64 tokens");
    if (g0 + n > ctx->pool_nodes) return set_error(NNQS_E_TABLE_FULL, "key/value cache full");
    ctx->tcw.st = st;
    for (int64_t c0 = 0; c0 < n; c0 += ctx->C) {
        const int64_t cn = std::min(ctx->C, n - c0);
        if (ctx->prec == NNQS_FP64) {
            const Views<double> V = make_views<double>(M, static_cast<double *>(ctx->params));
            NNQS_TRY(decode_chunk<double>(M, V, prefixes + c0 * M->W, cn, t, g0 + c0, static_cast<double *>(ctx->pool),
                                          anc + c0, ctx->anc_stride, ctx->Ad, cond + c0 * 4, st, nullptr, s));
        } else {
            const Views<float> V = make_views<float>(M, static_cast<float *>(ctx->params));
            NNQS_TRY(decode_chunk<float>(M, V, prefixes + c0 * M->W, cn, t, g0 + c0, static_cast<float *>(ctx->pool),
                                         anc + c0, ctx->anc_stride, ctx->Af, cond + c0 * 4, st,
                                         ctx->tensor ? &ctx->tcw : nullptr, s));
        }
    }
    return NNQS_OK;
}

bool cond_dev_walk_ok(const nnqs_model *M, int prec, int64_t cap) {
    return prec != NNQS_FP64 && tc_mode(prec) != 0 && M->d == dec::kD && M->F == dec::kF &&
           (M->dh == 8 || M->dh == 16) && cap <= chunk_for(M, std::max<int64_t>(cap, 1), sizeof(float), false);
}

bool cond_cached_dev_ok(const nnqs_model *M, const CondCtx *ctx, int64_t cap) {
    return ctx->prec != NNQS_FP64 && ctx->tensor && decode_fused_ok(M, ctx->tcw) && cap <= ctx->C;
}

nnqs_status cond_step_cached_dev(const nnqs_model *M, CondCtx *ctx, const uint64_t *prefixes, const int64_t *n_dev,
                                 const int64_t *g0_dev, int64_t cap, int t, const int32_t *anc, double *cond,
                                 DevStatus *st, cudaStream_t s, float *act, float *fin) {
    if (t >= kMaxDepth) return set_error(NNQS_E_UNSUPPORTED, "more than 64 tokens");
    if (!cond_cached_dev_ok(M, ctx, cap)) return set_error(NNQS_E_UNSUPPORTED, "no fused decode for this model");
    ctx->tcw.st = st;
    const Views<float> V = make_views<float>(M, static_cast<float *>(ctx->params));
    if (profiling_on()) {  // the level's size, for the profile's work count (profiling runs wait anyway)
        int64_t n = 0;
        NNQS_CUDA_TRY(cudaMemcpyAsync(&n, n_dev, 8, cudaMemcpyDeviceToHost, s));
        NNQS_CUDA_TRY(cudaStreamSynchronize(s));
        note_decode_work(n, ctx->tcw.split, M->L, t);
    }
    NNQS_TRY(decode_step_fused(M, V, ctx->tcw, prefixes, cap, static_cast<float *>(ctx->pool), anc, ctx->anc_stride, t,
                               0, cond, st, s, n_dev, g0_dev, act, fin));
    return NNQS_OK;
}

nnqs_status cond_step(const nnqs_model *M, CondCtx *ctx, const uint64_t *prefixes, int64_t n, int S, double *cond,
                      DevStatus *st, cudaStream_t s) {
    ctx->tcw.st = st;
    for (int64_t c0 = 0; c0 < n; c0 += ctx->C) {
        const int64_t cn = std::min(ctx->C, n - c0);
        if (ctx->prec == NNQS_FP64) {
            const Views<double> V = make_views<double>(M, static_cast<double *>(ctx->params));
            NNQS_TRY(forward_chunk<double>(M, V, prefixes + c0 * M->W, cn, ctx->Ad, nullptr, st, c0, nullptr, s, S,
                                           cond + c0 * 4));
        } else {
            const Views<float> V = make_views<float>(M, static_cast<float *>(ctx->params));
            NNQS_TRY(forward_chunk<float>(M, V, prefixes + c0 * M->W, cn, ctx->Af, nullptr, st, c0,
                                          ctx->tensor ? &ctx->tcw : nullptr, s, S, cond + c0 * 4));
        }
    }
    return NNQS_OK;
}

size_t logpsi_workspace(const nnqs_model *M, int64_t n, int prec, bool backward) {
    if (prec == NNQS_FP64) return workspace_impl<double>(M, n, backward, 0);
    return workspace_impl<float>(M, n, backward, tc_mode(prec));
}

nnqs_status logpsi_forward(const nnqs_model *M, const float *params, const uint64_t *x, int64_t n, int prec,
                           double *out, Arena &ws, DevStatus *st, cudaStream_t s) {
    if (prec == NNQS_FP64) return forward_impl<double>(M, params, x, n, out, ws, st, 0, s);
    return forward_impl<float>(M, params, x, n, out, ws, st, tc_mode(prec), s);
}

nnqs_status logpsi_backward(const nnqs_model *M, const float *params, const uint64_t *x, int64_t n, int prec,
                            const double *seed, double *g64, float *g32, Arena &ws, DevStatus *st, cudaStream_t s) {
    if (prec == NNQS_FP64) return backward_impl<double>(M, params, x, n, seed, g64, g32, ws, st, 0, s);
    return backward_impl<float>(M, params, x, n, seed, g64, g32, ws, st, tc_mode(prec), s);
}

bool logpsi_single_chunk(const nnqs_model *M, int64_t n, int prec) {
    return chunk_for(M, std::max<int64_t>(n, 1), prec == NNQS_FP64 ? sizeof(double) : sizeof(float), true) >= n;
}

// ---------------------------------------------------------------- rows from the sampler's tree
// The activations of every token row (sample i, position t) as the sampler's
// decode step left them at row t's tree node anc[t * stride + i]
// (NNQS_SAMPLE_KEEP): the final residual and, when `layers` is set, each
// layer's input and mid residual (the fused reverse mode reads those from the
// nodes itself); then the final LayerNorm, the head and the masked
// log-softmax of the row's token, as the forward's last part computes them.
// 4 lanes per row, 16 columns each; lane 0 of a row writes its conditionals,
// token and log probability (lprow), k_rows_logpsi adds a sample's rows.
constexpr int kRowsPerBlock = 64;
__global__ void __launch_bounds__(4 * kRowsPerBlock) k_rows_from_nodes(
    const uint64_t *__restrict__ x, int W, int64_t n, int T, int L, const float *__restrict__ act,
    const float *__restrict__ fin, const int32_t *__restrict__ anc, int64_t stride, const float *__restrict__ lnf_g,
    const float *__restrict__ lnf_b, const float *__restrict__ hw, const float *__restrict__ hb, int n_alpha,
    int n_beta, bool layers, float *__restrict__ hbuf, float *__restrict__ hmid, float *__restrict__ hf,
    float *__restrict__ meanf, float *__restrict__ rstdf, float *__restrict__ pi, uint8_t *__restrict__ tok,
    float *__restrict__ lprow) {
    constexpr int d = 64;
    const int64_t rows = n * T;
    const int64_t r = blockIdx.x * (int64_t)kRowsPerBlock + (threadIdx.x >> 2);
    const int q = threadIdx.x & 3;
    const bool valid = r < rows;
    const int64_t i = valid ? r / T : 0;
    const int t = valid ? (int)(r - i * T) : 0;
    const int64_t node = valid ? (int64_t)anc[t * stride + i] : 0;
    if (valid && layers) {
        for (int l = 0; l < L; ++l) {
            const float4 *a0 = reinterpret_cast<const float4 *>(act + ((node * L + l) * 2) * d + 16 * q);
            const float4 *a1 = reinterpret_cast<const float4 *>(act + ((node * L + l) * 2 + 1) * d + 16 * q);
            float4 *h0 = reinterpret_cast<float4 *>(hbuf + ((int64_t)l * rows + r) * d + 16 * q);
            float4 *h1 = reinterpret_cast<float4 *>(hmid + ((int64_t)l * rows + r) * d + 16 * q);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                h0[k] = __ldg(a0 + k);
                h1[k] = __ldg(a1 + k);
            }
        }
    }
    float v[16];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float4 f = valid ? __ldg(reinterpret_cast<const float4 *>(fin + node * d + 16 * q) + k)
                               : make_float4(0.f, 0.f, 0.f, 0.f);
        v[4 * k] = f.x;
        v[4 * k + 1] = f.y;
        v[4 * k + 2] = f.z;
        v[4 * k + 3] = f.w;
    }
    if (valid) {
        float4 *hl = reinterpret_cast<float4 *>(hbuf + ((int64_t)L * rows + r) * d + 16 * q);
#pragma unroll
        for (int k = 0; k < 4; ++k) hl[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
    }
    // final LayerNorm (eps 1e-5) over the row's 64 columns
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < 16; ++c) s += v[c];
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    const float mu = s / float(d);
    float qv = 0.f;
#pragma unroll
    for (int c = 0; c < 16; ++c) qv += (v[c] - mu) * (v[c] - mu);
    qv += __shfl_xor_sync(0xffffffffu, qv, 1);
    qv += __shfl_xor_sync(0xffffffffu, qv, 2);
    const float rs = 1.0f / sqrtf(qv / float(d) + 1e-5f);
    float y[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) y[c] = (v[c] - mu) * rs * __ldg(lnf_g + 16 * q + c) + __ldg(lnf_b + 16 * q + c);
    if (valid) {
        float4 *ho = reinterpret_cast<float4 *>(hf + r * d + 16 * q);
#pragma unroll
        for (int k = 0; k < 4; ++k) ho[k] = make_float4(y[4 * k], y[4 * k + 1], y[4 * k + 2], y[4 * k + 3]);
        if (q == 0) {
            meanf[r] = mu;
            rstdf[r] = rs;
        }
    }
    // head logits and the masked log-softmax of the row's token
    float z[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float a = 0.f;
#pragma unroll
        for (int c = 0; c < 16; ++c) a += y[c] * __ldg(hw + k * d + 16 * q + c);
        a += __shfl_xor_sync(0xffffffffu, a, 1);
        a += __shfl_xor_sync(0xffffffffu, a, 2);
        z[k] = a + __ldg(hb + k);
    }
    if (!valid || q != 0) return;
    const uint64_t *xi = x + i * W;
    int ca = 0, cb = 0;  // electrons on the orbitals of tokens < t
    for (int p2 = T - t; p2 < T; ++p2) {
        ca += bit_of(xi, 2 * p2);
        cb += bit_of(xi, 2 * p2 + 1);
    }
    const int rem = T - 1 - t;
    bool okv[4];
    float zmax = -INFINITY;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int a = ca + (k & 1), b = cb + (k >> 1);
        okv[k] = a <= n_alpha && b <= n_beta && a + rem >= n_alpha && b + rem >= n_beta;
        if (okv[k] && z[k] > zmax) zmax = z[k];
    }
    float se = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (okv[k]) se += expf(z[k] - zmax);
    const float lse = zmax + logf(se);
    const int tk = token_at(xi, T, t);
#pragma unroll
    for (int k = 0; k < 4; ++k) pi[r * 4 + k] = okv[k] ? expf(z[k] - lse) : 0.f;
    tok[r] = (uint8_t)tk;
    lprow[r] = okv[tk] ? z[tk] - lse : -INFINITY;
}

// log|psi| of each sample: half the sum of its rows' log probabilities (in
// position order); an out-of-sector token gives -inf and NNQS_E_SECTOR
__global__ void k_rows_logpsi(const float *__restrict__ lprow, int64_t n, int T, double2 *__restrict__ out,
                              DevStatus *st) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float sum = 0.f;
    bool bad = false;
    for (int t = 0; t < T; ++t) {
        const float v = lprow[i * T + t];
        if (v == -INFINITY)
            bad = true;
        else
            sum += v;
    }
    out[i].x = bad ? -(double)INFINITY : 0.5 * (double)sum;
    if (bad) record_status(st, NNQS_E_SECTOR, i);
}

// the samples must be the last level of the kept tree, row for row
__global__ void k_rows_match(const uint64_t *__restrict__ x, const uint64_t *__restrict__ pref, int64_t n, int W,
                             DevStatus *st) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int w = 0; w < W; ++w)
        if (x[i * W + w] != pref[i * W + w]) {
            record_status(st, NNQS_E_INVAL, i);
            return;
        }
}

// forward quantities of the reverse mode from the sampler's tree, then
// `between` (which fills `seed`), then the fused reverse mode
nnqs_status rows_fwd_bwd_impl(const nnqs_model *M, const float *params, const uint64_t *x, int64_t n, double *lp_out,
                              const double *seed, double *g64, float *g32, Arena &ws, DevStatus *st, int tcm,
                              cudaStream_t s, const std::function<nnqs_status()> &between, const SampleKept &kept) {
    using R = float;
    if (!reverse_lite(M, tcm)) return set_error(NNQS_E_UNSUPPORTED, "no fused reverse mode for this model or precision");
    R *pr = ws.take<R>(M->lay.total);
    R *gacc = ws.take<R>(M->lay.total);
    TcWeights tcw{};
    tc_weights_take(M, ws, &tcw);
    tcw.st = st;
    tcw.split = tcm == 2;
    tcw.fp8 = false;
    const int64_t C = chunk_for(M, std::max<int64_t>(n, 1), sizeof(R), true);
    if (C < n) return set_error(NNQS_E_INVAL, "forward/backward from the sampler's rows needs one chunk");
    Acts<R> A;
    take_acts<R>(M, C, true, ws, A, true);
    Grads<R> G;
    take_grads<R>(M, C, ws, G, true);
    const int T = M->T;
    const int64_t rows = n * T;
    NNQS_CUDA_TRY(cudaMemsetAsync(A.scr.ctr, 0, sizeof(unsigned), s));
    NNQS_LAUNCH("k_convert_params", s, k_convert_params<R><<<grid_for(M->lay.total, 256), 256, 0, s>>>(params, pr, M->lay.total));
    NNQS_LAUNCH("k_fill", s, k_fill<R><<<grid_for(M->lay.total, 256), 256, 0, s>>>(gacc, M->lay.total, R(0)));
    NNQS_TRY(tc_weights_prepare(M, params, tcw, s));
    const Views<R> V = make_views<R>(M, pr);
    NNQS_LAUNCH("k_rows_match", s, k_rows_match<<<grid_for(n, 256), 256, 0, s>>>(x, kept.pref, n, M->W, st));
    NNQS_LAUNCH("k_rows_from_nodes", s,
                k_rows_from_nodes<<<(unsigned)((rows + kRowsPerBlock - 1) / kRowsPerBlock), 4 * kRowsPerBlock, 0, s>>>(
                    x, M->W, n, T, M->L, kept.act, kept.fin, kept.anc, kept.stride, V.lnf_g, V.lnf_b, V.hw, V.hb,
                    M->cfg.n_alpha, M->cfg.n_beta, false, A.hbuf, A.hmid, A.hf, A.meanf, A.rstdf, A.pi, A.tok,
                    G.dtmp));
    double2 *out = reinterpret_cast<double2 *>(lp_out);
    NNQS_LAUNCH("k_rows_logpsi", s, k_rows_logpsi<<<grid_for(n, 256), 256, 0, s>>>(G.dtmp, n, T, out, st));
    NNQS_TRY(phase_mlp<R>(M, V, x, n, A, out, &tcw, s));
    NNQS_TRY(between());
    NNQS_TRY(backward_chunk<R>(M, V, x, n, A, G, reinterpret_cast<const double2 *>(seed), gacc, &tcw, s, &kept));
    NNQS_LAUNCH("k_grad_out", s, k_grad_out<R><<<grid_for(M->lay.total, 256), 256, 0, s>>>(gacc, M->lay.total, g64, g32));
    return NNQS_OK;
}

nnqs_status logpsi_forward_backward(const nnqs_model *M, const float *params, const uint64_t *x, int64_t n, int prec,
                                    double *lp_out, const double *seed, double *g64, float *g32, Arena &ws,
                                    DevStatus *st, cudaStream_t s, const std::function<nnqs_status()> &between) {
    if (prec == NNQS_FP64)
        return fwd_bwd_impl<double>(M, params, x, n, lp_out, seed, g64, g32, ws, st, 0, s, between);
    return fwd_bwd_impl<float>(M, params, x, n, lp_out, seed, g64, g32, ws, st, tc_mode(prec), s, between);
}

bool reverse_lite_ok(const nnqs_model *M, int tcm) { return reverse_lite(M, tcm); }

nnqs_status logpsi_forward_backward_rows(const nnqs_model *M, const float *params, const uint64_t *x, int64_t n,
                                         int prec, double *lp_out, const double *seed, double *g64, float *g32,
                                         Arena &ws, DevStatus *st, cudaStream_t s,
                                         const std::function<nnqs_status()> &between, const SampleKept &kept) {
    const int tcm = tc_mode(prec);
    if (tcm != 1 && tcm != 2) return set_error(NNQS_E_UNSUPPORTED, "rows from the sampler: BF16 or split BF16 only");
    return rows_fwd_bwd_impl(M, params, x, n, lp_out, seed, g64, g32, ws, st, tcm, s, between, kept);
}

}  // namespace nnqs
