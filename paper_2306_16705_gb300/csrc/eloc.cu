// Local energy, Eq. (Eloc), sample-aware form (Sec. 3.4 (2)-(5), Alg. 2),
// re-mapped to sm_103a.
//
// E_loc(x) = sum_{x' in S} H_{x x'} psi(x') / psi(x),
// H_{x x'} = sum_{t in group(x ^ x')} coef_t (-1)^{popc(x & yz_t)}.
//
// The paper gives one thread a whole sample and walks every X/Y group of
// the Hamiltonian for it (Alg. 2).  Here a CTA takes a tile of rows x and a
// chunk of the work so that the grid fills 152 SMs, and writes one partial
// sum per (chunk, row); a second kernel adds the partials in chunk order so
// the result does not depend on scheduling.  The diagonal group (x' = x,
// the largest group) is evaluated by one warp per row in its own kernel so
// that it does not serialise a warp of the sweep.
//
// Two sweeps give the same sum:
//   GROUPS  for each row and each non-diagonal group m: x' = x ^ m kept iff
//           it has the sector's electron counts, then probed in the hash of
//           S (the role of the sorted id_lut search of Alg. 2).
//   PAIRS   for each row x and each sample y in S: m = x ^ y is looked up
//           in the hash of group X/Y masks when popc(m) is at most the
//           largest group weight.  Cost |rows| x |S| instead of
//           |rows| x N_XY.
#include <cuda_runtime.h>

#include <algorithm>

#include "dev_common.cuh"
#include "internal.h"
#include "sweep_common.cuh"

namespace nnqs {
namespace {

constexpr int kSweepThreads = 128;
constexpr int kGroupTile = 256;   // groups staged in shared memory per step
constexpr int kPairTile = 512;    // samples staged in shared memory per step
constexpr int kPairRows = 2;      // rows per thread in the pair sweep

template <int W>
__global__ void k_build_lut_hash(const uint64_t *__restrict__ lut, int64_t n_lut, int n_qubits,
                                 int n_alpha, int n_beta, HashTab<W> tab, DevStatus *st) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_lut) return;
    Bits<W> k = load_bits<W>(lut, i);
    int na = 0, nb = 0;
    bool high = false;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        na += __popcll(k.w[w] & kEven);
        nb += __popcll(k.w[w] & ~kEven);
        int lo = n_qubits - 64 * w;  // valid bits in this word
        if (lo < 64) high |= (lo <= 0) ? (k.w[w] != 0) : ((k.w[w] >> lo) != 0);
    }
    if (high) {
        record_status(st, NNQS_E_INVAL, i);
        return;
    }
    if (na != n_alpha || nb != n_beta) {
        record_status(st, NNQS_E_SECTOR, i);
        return;
    }
    bool fresh = false;
    int64_t slot = tab.insert(k, &fresh);
    if (slot < 0) {
        record_status(st, NNQS_E_TABLE_FULL, i);
        return;
    }
    if (!fresh) {
        record_status(st, NNQS_E_DUPLICATE, i);
        return;
    }
    tab.vals[slot] = (int32_t)i;
}

// the table's largest log|psi| (one block; max is order-free)
__global__ void k_lp_max(const double2 *__restrict__ lp, int64_t n, double *__restrict__ amax) {
    __shared__ double sh[1024];
    double m = -INFINITY;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, lp[i].x);
    sh[threadIdx.x] = m;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + off]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *amax = sh[0];
}

// psi[j] = exp(log|psi_j| - A) (cos phase_j, sin phase_j)
__global__ void k_lut_psi(const double2 *__restrict__ lp, int64_t n, const double *__restrict__ amax,
                          double2 *__restrict__ psi) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    const double2 v = lp[j];
    const double m = exp(v.x - *amax);
    double s, c;
    sincos(v.y, &s, &c);
    psi[j] = make_double2(m * c, m * s);
}

// GROUPS sweep.  grid = (row tiles of 128, group chunks).
template <int W>
__global__ void __launch_bounds__(kSweepThreads)
    k_sweep_groups(const uint64_t *__restrict__ gxy, const uint32_t *__restrict__ goff,
                   const uint8_t *__restrict__ gspin, int64_t g_begin, int64_t g_end,
                   int64_t groups_per_chunk, const uint64_t *__restrict__ tyz,
                   const double *__restrict__ tcoef, const uint64_t *__restrict__ lut,
                   const double2 *__restrict__ lut_lp, const double2 *__restrict__ psi,
                   const double *__restrict__ amax, HashTab<W> tab, int64_t row_begin,
                   int64_t n_rows, double2 *__restrict__ partial) {
    __shared__ uint64_t s_xy[kGroupTile * W];
    __shared__ uint8_t s_spin[kGroupTile];
    const int64_t r = blockIdx.x * (int64_t)kSweepThreads + threadIdx.x;
    const bool active = r < n_rows;
    Bits<W> x{};
    RowRatio rx;
    rx.init(make_double2(0.0, 0.0), nullptr);
    if (active) {
        x = load_bits<W>(lut, row_begin + r);
        rx.init(lut_lp[row_begin + r], amax);
    }
    const int64_t c0 = g_begin + blockIdx.y * groups_per_chunk;
    const int64_t c1 = min(g_end, c0 + groups_per_chunk);
    double er = 0.0, ei = 0.0;
    for (int64_t gt = c0; gt < c1; gt += kGroupTile) {
        const int ntile = (int)min((int64_t)kGroupTile, c1 - gt);
        __syncthreads();
        for (int k = threadIdx.x; k < ntile * W; k += kSweepThreads) s_xy[k] = gxy[gt * W + k];
        for (int k = threadIdx.x; k < ntile; k += kSweepThreads) s_spin[k] = gspin[gt + k];
        __syncthreads();
        if (!active) continue;
        for (int k = 0; k < ntile; ++k) {
            const uint8_t sp = s_spin[k];
            int ra = 0, rb = 0;  // electrons the mask removes, per spin
#pragma unroll
            for (int w = 0; w < W; ++w) {
                uint64_t v = s_xy[k * W + w] & x.w[w];
                ra += __popcll(v & kEven);
                rb += __popcll(v & ~kEven);
            }
            if (sp == 0xFF || ra != (sp & 15) || rb != (sp >> 4)) continue;
            Bits<W> xp;
#pragma unroll
            for (int w = 0; w < W; ++w) xp.w[w] = x.w[w] ^ s_xy[k * W + w];
            const int32_t j = tab.find(xp);
            if (j < 0) continue;
            const int64_t g = gt + k;
            const double coef = group_coef<W>(x, __ldg(goff + g), __ldg(goff + g + 1), tyz, tcoef);
            const double2 q = rx.of(psi, lut_lp, j);
            er += coef * q.x;
            ei += coef * q.y;
        }
    }
    if (active) partial[blockIdx.y * n_rows + r] = make_double2(er, ei);
}

// TERMS sweep over the ungrouped layout: every string t carries its own X/Y
// mask, so each string tests its coupled x' = x ^ xy_t on its own (spin
// counts, table probe) and adds coef_t (-1)^{popc(x & yz_t)} psi(x')/psi(x).
// The cost the grouping of Alg. 1 removes: N_h probes per row instead of
// N_XY.  grid = (row tiles of 128, string chunks).
constexpr int kTermTile = 256;
template <int W>
__global__ void __launch_bounds__(kSweepThreads)
    k_sweep_terms(const uint64_t *__restrict__ txy, const uint64_t *__restrict__ tyz,
                  const double *__restrict__ tcoef, int64_t t_begin, int64_t t_end, int64_t terms_per_chunk,
                  const uint64_t *__restrict__ lut, const double2 *__restrict__ lut_lp,
                  const double2 *__restrict__ psi, const double *__restrict__ amax, HashTab<W> tab,
                  int64_t row_begin, int64_t n_rows, double2 *__restrict__ partial) {
    __shared__ uint64_t s_xy[kTermTile * W], s_yz[kTermTile * W];
    __shared__ double s_c[kTermTile];
    const int64_t r = blockIdx.x * (int64_t)kSweepThreads + threadIdx.x;
    const bool active = r < n_rows;
    Bits<W> x{};
    RowRatio rx;
    rx.init(make_double2(0.0, 0.0), nullptr);
    if (active) {
        x = load_bits<W>(lut, row_begin + r);
        rx.init(lut_lp[row_begin + r], amax);
    }
    const int64_t c0 = t_begin + blockIdx.y * terms_per_chunk;
    const int64_t c1 = min(t_end, c0 + terms_per_chunk);
    double er = 0.0, ei = 0.0;
    for (int64_t tt = c0; tt < c1; tt += kTermTile) {
        const int nt = (int)min((int64_t)kTermTile, c1 - tt);
        __syncthreads();
        for (int k = threadIdx.x; k < nt * W; k += kSweepThreads) {
            s_xy[k] = txy[tt * W + k];
            s_yz[k] = tyz[tt * W + k];
        }
        for (int k = threadIdx.x; k < nt; k += kSweepThreads) s_c[k] = tcoef[tt + k];
        __syncthreads();
        if (!active) continue;
        for (int k = 0; k < nt; ++k) {
            int ma = 0, mb = 0, ra = 0, rb = 0;  // mask bits and electrons it removes, per spin
            int par = 0;
#pragma unroll
            for (int w = 0; w < W; ++w) {
                const uint64_t m = s_xy[k * W + w], v = m & x.w[w];
                ma += __popcll(m & kEven);
                mb += __popcll(m & ~kEven);
                ra += __popcll(v & kEven);
                rb += __popcll(v & ~kEven);
                par += __popcll(x.w[w] & s_yz[k * W + w]);
            }
            if (2 * ra != ma || 2 * rb != mb) continue;
            Bits<W> xp;
#pragma unroll
            for (int w = 0; w < W; ++w) xp.w[w] = x.w[w] ^ s_xy[k * W + w];
            const int32_t j = tab.find(xp);
            if (j < 0) continue;
            const double c = (par & 1) ? -s_c[k] : s_c[k];
            const double2 q = rx.of(psi, lut_lp, j);
            er += c * q.x;
            ei += c * q.y;
        }
    }
    if (active) partial[blockIdx.y * n_rows + r] = make_double2(er, ei);
}

// PAIRS sweep.  grid = (row tiles of 128 * kPairRows, sample chunks).
template <int W>
__global__ void __launch_bounds__(kSweepThreads)
    k_sweep_pairs(const uint64_t *__restrict__ lut, const double2 *__restrict__ lut_lp,
                  const double2 *__restrict__ psi, const double *__restrict__ amax,
                  int64_t n_lut, int64_t cols_per_chunk, int max_weight, HashTab<W> gtab,
                  const uint32_t *__restrict__ goff, const uint64_t *__restrict__ tyz,
                  const double *__restrict__ tcoef, int64_t row_begin, int64_t n_rows,
                  double2 *__restrict__ partial) {
    __shared__ uint64_t s_y[kPairTile * W];
    const int64_t rbase = blockIdx.x * (int64_t)(kSweepThreads * kPairRows);
    Bits<W> x[kPairRows];
    RowRatio rx[kPairRows];
    bool act[kPairRows];
    double er[kPairRows], ei[kPairRows];
#pragma unroll
    for (int q = 0; q < kPairRows; ++q) {
        const int64_t r = rbase + q * kSweepThreads + threadIdx.x;
        act[q] = r < n_rows;
        er[q] = ei[q] = 0.0;
        if (act[q]) {
            x[q] = load_bits<W>(lut, row_begin + r);
            rx[q].init(lut_lp[row_begin + r], amax);
        } else {
#pragma unroll
            for (int w = 0; w < W; ++w) x[q].w[w] = 0;
            rx[q].init(make_double2(0.0, 0.0), nullptr);
        }
    }
    const int64_t c0 = blockIdx.y * cols_per_chunk;
    const int64_t c1 = min(n_lut, c0 + cols_per_chunk);
    for (int64_t ct = c0; ct < c1; ct += kPairTile) {
        const int ntile = (int)min((int64_t)kPairTile, c1 - ct);
        __syncthreads();
        for (int k = threadIdx.x; k < ntile * W; k += kSweepThreads) s_y[k] = lut[ct * W + k];
        __syncthreads();
        for (int k = 0; k < ntile; ++k) {
            Bits<W> y;
#pragma unroll
            for (int w = 0; w < W; ++w) y.w[w] = s_y[k * W + w];
            int32_t g[kPairRows];
            bool any = false;
#pragma unroll
            for (int q = 0; q < kPairRows; ++q) {
                int d = 0;
                Bits<W> m;
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    m.w[w] = x[q].w[w] ^ y.w[w];
                    d += __popcll(m.w[w]);
                }
                // d == 0 is the diagonal, handled by k_diag
                g[q] = (d == 0 || d > max_weight || !act[q]) ? -1 : gtab.find(m);
                any |= g[q] >= 0;
            }
            if (!any) continue;
            // each lane its own hits: the ratio psi(y)/psi(x) and the popcount
            // signs over the hit's group, the group's strings in order (the
            // sampler's samples cluster, so hits are common and the lanes'
            // dependent loads overlap; a group averages about five strings)
#pragma unroll
            for (int q = 0; q < kPairRows; ++q) {
                if (g[q] < 0) continue;
                const double2 rr = rx[q].of(psi, lut_lp, ct + k);
                const uint32_t t0 = __ldg(goff + g[q]), t1 = __ldg(goff + g[q] + 1);
                double c = 0.0;
                for (uint32_t t = t0; t < t1; ++t) {
                    const Bits<W> yz = load_bits<W>(tyz, t);
                    const double v = __ldg(tcoef + t);
                    c += (popc_and<W>(x[q], yz) & 1) ? -v : v;
                }
                er[q] += c * rr.x;
                ei[q] += c * rr.y;
            }
        }
    }
#pragma unroll
    for (int q = 0; q < kPairRows; ++q) {
        const int64_t r = rbase + q * kSweepThreads + threadIdx.x;
        if (act[q]) partial[blockIdx.y * n_rows + r] = make_double2(er[q], ei[q]);
    }
}

struct SaPlan {
    bool pairs, terms;
    int64_t row_tiles, chunks, per_chunk;
    int64_t g_begin, g_end;
    bool has_diag;
};


SaPlan plan_sa(const nnqs_ham *H, int64_t n_lut, int64_t n_rows, int flags) {
    SaPlan p{};
    p.has_diag = H->n_groups > 0 && H->gxy[0] == 0 && (H->W == 1 || H->gxy[1] == 0);
    p.g_begin = p.has_diag ? 1 : 0;
    p.g_end = H->n_groups;
    const int64_t work_groups = n_rows * (p.g_end - p.g_begin);
    const int64_t work_pairs = n_rows * n_lut;
    if (flags == NNQS_SWEEP_GROUPS)
        p.pairs = false;
    else if (flags == NNQS_SWEEP_PAIRS)
        p.pairs = true;
    else
        p.pairs = work_pairs < work_groups;
    // enough CTAs for ~8 per SM
    const int64_t target = 8 * (int64_t)num_sms();
    p.terms = flags == NNQS_SWEEP_TERMS;
    if (p.terms) {
        // strings of the non-diagonal groups
        p.pairs = false;
        p.g_begin = p.has_diag ? H->goff[1] : 0;
        p.g_end = H->n_terms;
        const int64_t nt = p.g_end - p.g_begin;
        p.row_tiles = std::max<int64_t>(1, (n_rows + kSweepThreads - 1) / kSweepThreads);
        int64_t max_chunks = std::max<int64_t>(1, (nt + kTermTile - 1) / kTermTile);
        p.chunks = std::min(max_chunks, std::max<int64_t>(1, (target + p.row_tiles - 1) / p.row_tiles));
        p.per_chunk = std::max<int64_t>(1, (nt + p.chunks - 1) / p.chunks);
        p.chunks = nt > 0 ? (nt + p.per_chunk - 1) / p.per_chunk : 0;
        return p;
    }
    if (p.pairs) {
        p.row_tiles = std::max<int64_t>(1, (n_rows + kSweepThreads * kPairRows - 1) / (kSweepThreads * kPairRows));
        int64_t max_chunks = std::max<int64_t>(1, (n_lut + kPairTile - 1) / kPairTile);
        p.chunks = std::min(max_chunks, std::max<int64_t>(1, (target + p.row_tiles - 1) / p.row_tiles));
        p.per_chunk = (n_lut + p.chunks - 1) / p.chunks;
        p.per_chunk = std::max<int64_t>(1, p.per_chunk);
        p.chunks = std::max<int64_t>(1, (n_lut + p.per_chunk - 1) / p.per_chunk);
    } else {
        const int64_t ng = p.g_end - p.g_begin;
        p.row_tiles = std::max<int64_t>(1, (n_rows + kSweepThreads - 1) / kSweepThreads);
        int64_t max_chunks = std::max<int64_t>(1, (ng + kGroupTile - 1) / kGroupTile);
        p.chunks = std::min(max_chunks, std::max<int64_t>(1, (target + p.row_tiles - 1) / p.row_tiles));
        p.per_chunk = std::max<int64_t>(1, (ng + p.chunks - 1) / p.chunks);
        p.chunks = ng > 0 ? (ng + p.per_chunk - 1) / p.per_chunk : 0;
    }
    return p;
}

template <int W>
nnqs_status eloc_sa_impl(const nnqs_ham *H, const uint64_t *lut, const double *lut_lp, int64_t n_lut,
                         int64_t row_begin, int64_t n_rows, int n_alpha, int n_beta, int flags,
                         double *out, Arena &ws, DevStatus *status, cudaStream_t s) {
    const SaPlan p = plan_sa(H, n_lut, n_rows, flags);
    const int64_t cap = pow2_at_least(std::max<int64_t>(2, 2 * n_lut));
    uint64_t *hkeys = ws.take<uint64_t>(size_t(cap) * W);
    int32_t *hvals = ws.take<int32_t>(size_t(cap));
    double *diag = ws.take<double>(size_t(std::max<int64_t>(1, n_rows)));
    double2 *partial = ws.take<double2>(size_t(std::max<int64_t>(1, p.chunks * n_rows)));
    double2 *psi = ws.take<double2>(size_t(std::max<int64_t>(1, n_lut)));
    double *amax = ws.take<double>(1);
    if (ws.base == nullptr) return NNQS_OK;  // sizing pass

    if (n_rows == 0) return NNQS_OK;
    NNQS_CUDA_TRY(cudaMemsetAsync(hkeys, 0xFF, size_t(cap) * W * 8, s));
    HashTab<W> tab{hkeys, hvals, uint64_t(cap - 1)};
    NNQS_LAUNCH("k_build_lut_hash", s, k_build_lut_hash<W><<<grid_for(n_lut, 256), 256, 0, s>>>(lut, n_lut, H->n_qubits, n_alpha, n_beta, tab, status));
    if (p.has_diag) {
        NNQS_LAUNCH("k_diag", s, k_diag<W><<<grid_for(n_rows * 32, 256), 256, 0, s>>>(lut, row_begin, n_rows, (uint32_t)H->goff[0],
                                                             (uint32_t)H->goff[1], H->d_tyz, H->d_tcoef, diag));
    }
    const double2 *lp2 = reinterpret_cast<const double2 *>(lut_lp);
    if (p.chunks > 0) {
        NNQS_LAUNCH("k_lut_psi", s, k_lp_max<<<1, 1024, 0, s>>>(lp2, n_lut, amax));
        NNQS_LAUNCH("k_lut_psi", s, k_lut_psi<<<grid_for(n_lut, 256), 256, 0, s>>>(lp2, n_lut, amax, psi));
    }
    if (p.chunks > 0) {
        dim3 grid((unsigned)p.row_tiles, (unsigned)p.chunks);
        if (p.terms) {
            if (!H->d_txy) return set_error(NNQS_E_INVAL, "ungrouped layout not built");
            note_work("k_sweep_terms", double(n_rows) * double(p.g_end - p.g_begin),
                      double(p.row_tiles) * double(p.g_end - p.g_begin) * (16.0 * W + 8.0));
            NNQS_LAUNCH("k_sweep_terms", s, k_sweep_terms<W><<<grid, kSweepThreads, 0, s>>>(H->d_txy, H->d_tyz, H->d_tcoef, p.g_begin, p.g_end,
                                                             p.per_chunk, lut, lp2, psi, amax, tab, row_begin, n_rows, partial));
        } else if (p.pairs) {
            const int maxw = H->max_xy_weight;
            // algorithmic work: one (row, sample) mask test each; bytes = one
            // read of the sample table per row tile
            note_work("k_sweep_pairs", double(n_rows) * double(n_lut),
                      double(p.row_tiles) * double(n_lut) * (8.0 * W + 16.0));
            HashTab<W> gtab{H->d_ghkeys, H->d_ghvals, uint64_t(H->ghcap - 1)};
            NNQS_LAUNCH("k_sweep_pairs", s, k_sweep_pairs<W><<<grid, kSweepThreads, 0, s>>>(lut, lp2, psi, amax, n_lut, p.per_chunk, maxw, gtab, H->d_goff,
                                                            H->d_tyz, H->d_tcoef, row_begin, n_rows, partial));
        } else {
            note_work("k_sweep_groups", double(n_rows) * double(p.g_end - p.g_begin),
                      double(p.row_tiles) * double(p.g_end - p.g_begin) * (8.0 * W + 1.0));
            NNQS_LAUNCH("k_sweep_groups", s, k_sweep_groups<W><<<grid, kSweepThreads, 0, s>>>(H->d_gxy, H->d_goff, H->d_gspin, p.g_begin, p.g_end,
                                                             p.per_chunk, H->d_tyz, H->d_tcoef, lut, lp2, psi, amax, tab,
                                                             row_begin, n_rows, partial));
        }
        NNQS_CUDA_TRY(cudaGetLastError());
    }
    NNQS_LAUNCH("k_reduce_partials", s, k_reduce_partials<<<grid_for(n_rows, 256), 256, 0, s>>>(p.has_diag ? diag : nullptr, partial, p.chunks, n_rows,
                                                            reinterpret_cast<double2 *>(out)));
    return NNQS_OK;
}

// Energy statistics over 128 fixed row ranges (the FP64 sums of one block
// were bound by a single SM's FP64 pipe): pass 0 gives the blocks' (sum w,
// sum w Re E_loc, sum w Im E_loc), pass 1 the blocks' sum w |E_loc - E|^2 with
// E from pass 0; k_stats_fin adds the block sums by a fixed tree.
constexpr int kStatBlocks = 128, kStatPartThreads = 256;

__global__ void __launch_bounds__(kStatPartThreads)
    k_stats_part(const double2 *__restrict__ e, const uint64_t *__restrict__ w, int64_t n, int pass,
                 const double *__restrict__ stats, double *__restrict__ part) {
    __shared__ double sh[3][kStatPartThreads];
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t i0 = blockIdx.x * chunk, i1 = min(n, i0 + chunk);
    double a = 0.0, b = 0.0, c = 0.0;
    const double er = pass ? stats[0] : 0.0, ei = pass ? stats[1] : 0.0;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += kStatPartThreads) {
        const double wi = (double)w[i];
        const double2 v = e[i];
        if (pass == 0) {
            a += wi;
            b += wi * v.x;
            c += wi * v.y;
        } else {
            const double dr = v.x - er, di = v.y - ei;
            a += wi * (dr * dr + di * di);
        }
    }
    const int t = threadIdx.x;
    sh[0][t] = a;
    sh[1][t] = b;
    sh[2][t] = c;
    __syncthreads();
    for (int off = kStatPartThreads / 2; off > 0; off >>= 1) {
        if (t < off) {
            sh[0][t] += sh[0][t + off];
            sh[1][t] += sh[1][t + off];
            sh[2][t] += sh[2][t + off];
        }
        __syncthreads();
    }
    if (t == 0) {
        part[3 * blockIdx.x] = sh[0][0];
        part[3 * blockIdx.x + 1] = sh[1][0];
        part[3 * blockIdx.x + 2] = sh[2][0];
    }
}

__global__ void __launch_bounds__(kStatBlocks) k_stats_fin(const double *__restrict__ part, int nb, int pass,
                                                           double *__restrict__ stats) {
    // the block sums added by a fixed tree (nb <= kStatBlocks, a power of two)
    __shared__ double sh[3][kStatBlocks];
    const int t = threadIdx.x;
#pragma unroll
    for (int c = 0; c < 3; ++c) sh[c][t] = t < nb ? part[3 * t + c] : 0.0;
    __syncthreads();
    for (int off = kStatBlocks / 2; off > 0; off >>= 1) {
        if (t < off) {
#pragma unroll
            for (int c = 0; c < 3; ++c) sh[c][t] += sh[c][t + off];
        }
        __syncthreads();
    }
    if (t != 0) return;
    const double a = sh[0][0], b = sh[1][0], c = sh[2][0];
    if (pass == 0) {
        stats[0] = b / a;
        stats[1] = c / a;
        stats[3] = a;
    } else {
        stats[2] = a / stats[3];
    }
}
}  // namespace

// bytes for either sweep (the size query does not know which one a call forces)
size_t eloc_sa_workspace(const nnqs_ham *H, int64_t n_lut, int64_t n_rows, int) {
    size_t best = 0;
    for (int f : {NNQS_SWEEP_GROUPS, NNQS_SWEEP_PAIRS, NNQS_SWEEP_TERMS}) {
        Arena a(nullptr);
        a.take<char>(kStatusBytes);
        if (H->W == 1)
            eloc_sa_impl<1>(H, nullptr, nullptr, n_lut, 0, n_rows, 0, 0, f, nullptr, a, nullptr, nullptr);
        else
            eloc_sa_impl<2>(H, nullptr, nullptr, n_lut, 0, n_rows, 0, 0, f, nullptr, a, nullptr, nullptr);
        best = std::max(best, a.used + 256);
    }
    return best;
}

size_t eloc_sa_workspace_for(const nnqs_ham *H, int64_t n_lut, int64_t n_rows, int flags) {
    Arena a(nullptr);
    a.take<char>(kStatusBytes);
    if (H->W == 1)
        eloc_sa_impl<1>(H, nullptr, nullptr, n_lut, 0, n_rows, 0, 0, flags, nullptr, a, nullptr, nullptr);
    else
        eloc_sa_impl<2>(H, nullptr, nullptr, n_lut, 0, n_rows, 0, 0, flags, nullptr, a, nullptr, nullptr);
    return a.used + 256;
}

nnqs_status eloc_sa(const nnqs_ham *H, const uint64_t *lut, const double *lut_lp, int64_t n_lut,
                    int64_t row_begin, int64_t n_rows, int n_alpha, int n_beta, int flags, double *out,
                    Arena &ws, DevStatus *status, cudaStream_t s) {
    if (H->W == 1)
        return eloc_sa_impl<1>(H, lut, lut_lp, n_lut, row_begin, n_rows, n_alpha, n_beta, flags, out, ws, status, s);
    return eloc_sa_impl<2>(H, lut, lut_lp, n_lut, row_begin, n_rows, n_alpha, n_beta, flags, out, ws, status, s);
}

size_t stats_workspace(int64_t) { return kStatusBytes + 256 + 3 * kStatBlocks * sizeof(double) + 256; }

nnqs_status energy_stats(const double *eloc, const uint64_t *w, int64_t n, double *stats, Arena &ws, cudaStream_t s) {
    double *part = ws.take<double>(3 * kStatBlocks);
    if (ws.base == nullptr) return NNQS_OK;
    const double2 *e = reinterpret_cast<const double2 *>(eloc);
    for (int pass = 0; pass < 2; ++pass) {
        NNQS_LAUNCH("k_stats", s, k_stats_part<<<kStatBlocks, kStatPartThreads, 0, s>>>(e, w, n, pass, stats, part));
        NNQS_LAUNCH("k_stats", s, k_stats_fin<<<1, kStatBlocks, 0, s>>>(part, kStatBlocks, pass, stats));
    }
    return NNQS_OK;
}

int num_sms() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
            sms = 152;
    }
    return sms;
}

}  // namespace nnqs

// ---------------------------------------------------------------- no-allocation variant
// Scratch for nnqs_eloc_sa_noalloc: one file-scope device array, present on
// every GPU that loads this library until the process exits.  Host code must
// not use the symbol itself as a device address: its device address is
// looked up with cudaGetSymbolAddress.
namespace nnqs {
namespace {
constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;  // 64 MiB
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// device address of the scratch array in the current context, looked up on
// every call (an address kept from an earlier call would outlive a context
// reset)
nnqs_status noalloc_scratch(void **out) {
    void *p = nullptr;
    NNQS_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    *out = p;
    return NNQS_OK;
}
}  // namespace
}  // namespace nnqs

extern "C" nnqs_status nnqs_eloc_sa_noalloc(const nnqs_ham *H, const uint64_t *lut, const double *lut_logpsi,
                                            int64_t n_lut, int64_t row_begin, int64_t n_rows, int n_alpha,
                                            int n_beta, int flags, double *eloc_out, int check,
                                            nnqs_stream stream) {
    using namespace nnqs;
    NNQS_TRY(eloc_args(H, n_lut, row_begin, n_rows, n_alpha, n_beta, NNQS_SA));
    NNQS_TRY(eloc_flags(H, flags, NNQS_SA));
    if (n_rows > 0 && (!lut || !lut_logpsi || !eloc_out)) return set_error(NNQS_E_INVAL, "null device pointer");
    // sized by the sweep this call runs (AUTO resolved), not the largest one
    const size_t need = eloc_sa_workspace_for(H, n_lut, n_rows, flags);
    if (need > kNoAllocScratchBytes)
        return set_error(NNQS_E_INVAL, "nnqs_eloc_sa_noalloc: this table needs " + std::to_string(need) +
                                           " bytes of scratch, above the fixed " +
                                           std::to_string(kNoAllocScratchBytes) +
                                           "; use nnqs_eloc with a workspace");
    void *scratch = nullptr;
    NNQS_TRY(noalloc_scratch(&scratch));
    cudaStream_t s = (cudaStream_t)stream;
    // the array keeps the previous call's contents: the status word starts at
    // zero and the hash table is cleared inside eloc_sa
    NNQS_CUDA_TRY(cudaMemsetAsync(scratch, 0, sizeof(DevStatus), s));
    Arena a(scratch);
    DevStatus *st = a.take<DevStatus>(kStatusBytes / sizeof(DevStatus));
    NNQS_TRY(eloc_sa(H, lut, lut_logpsi, n_lut, row_begin, n_rows, n_alpha, n_beta, flags, eloc_out, a, st, s));
    if (!check) return NNQS_OK;
    NNQS_CUDA_TRY(cudaStreamSynchronize(s));
    DevStatus hst{};
    NNQS_CUDA_TRY(cudaMemcpy(&hst, scratch, sizeof hst, cudaMemcpyDeviceToHost));
    if (hst.code != 0)
        return set_error((nnqs_status)hst.code, std::string("device reported: ") + nnqs_status_string(hst.code) +
                                                    " at row " + std::to_string(hst.index));
    return NNQS_OK;
}
