// Local energy over every coupled configuration (Eq. Eloc as written, no
// sample restriction):
//   1. insert each row x and every x' = x ^ m (m a group X/Y mask that keeps
//      the electron counts) into a device hash table -- the coupled set,
//      deduplicated across rows;
//   2. number the distinct keys and run the ansatz forward once on them;
//   3. sweep again and add H_{x x'} psi(x')/psi(x), with log psi looked up
//      in the table (the fused accumulation of Sec. 3.4 (2)).
// The sample-aware mode of the paper skips step 2 by restricting x' to S;
// this mode is the plain definition the paper approximates, used for
// validation and small systems.
#include <cuda_runtime.h>

#include <algorithm>

#include "dev_common.cuh"
#include "internal.h"
#include "model.h"
#include "sweep_common.cuh"

namespace nnqs {
namespace {

constexpr int kThreads = 128;
constexpr int kTile = 256;

template <int W>
__global__ void k_insert_rows(const uint64_t *__restrict__ lut, int64_t row_begin, int64_t n_rows, int n_qubits,
                              int n_alpha, int n_beta, HashTab<W> tab, DevStatus *st) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n_rows) return;
    const Bits<W> k = load_bits<W>(lut, row_begin + r);
    int na = 0, nb = 0;
    bool high = false;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        na += __popcll(k.w[w] & kEven);
        nb += __popcll(k.w[w] & ~kEven);
        const int lo = n_qubits - 64 * w;
        if (lo < 64) high |= (lo <= 0) ? (k.w[w] != 0) : ((k.w[w] >> lo) != 0);
    }
    if (high) {
        record_status(st, NNQS_E_INVAL, row_begin + r);
        return;
    }
    if (na != n_alpha || nb != n_beta) {
        record_status(st, NNQS_E_SECTOR, row_begin + r);
        return;
    }
    bool fresh;
    if (tab.insert(k, &fresh) < 0) record_status(st, NNQS_E_TABLE_FULL, row_begin + r);
}

// every conserving x ^ m of every row into the table
template <int W>
__global__ void __launch_bounds__(kThreads)
    k_expand(const uint64_t *__restrict__ gxy, const uint8_t *__restrict__ gspin, int64_t g_begin, int64_t g_end,
             int64_t per_chunk, const uint64_t *__restrict__ lut, int64_t row_begin, int64_t n_rows, HashTab<W> tab,
             DevStatus *st) {
    __shared__ uint64_t s_xy[kTile * W];
    __shared__ uint8_t s_spin[kTile];
    const int64_t r = blockIdx.x * (int64_t)kThreads + threadIdx.x;
    const bool active = r < n_rows;
    Bits<W> x{};
    if (active) x = load_bits<W>(lut, row_begin + r);
    const int64_t c0 = g_begin + blockIdx.y * per_chunk, c1 = min(g_end, c0 + per_chunk);
    for (int64_t gt = c0; gt < c1; gt += kTile) {
        const int nt = (int)min((int64_t)kTile, c1 - gt);
        __syncthreads();
        for (int k = threadIdx.x; k < nt * W; k += kThreads) s_xy[k] = gxy[gt * W + k];
        for (int k = threadIdx.x; k < nt; k += kThreads) s_spin[k] = gspin[gt + k];
        __syncthreads();
        if (!active) continue;
        for (int k = 0; k < nt; ++k) {
            const uint8_t sp = s_spin[k];
            int ra = 0, rb = 0;
#pragma unroll
            for (int w = 0; w < W; ++w) {
                const uint64_t v = s_xy[k * W + w] & x.w[w];
                ra += __popcll(v & kEven);
                rb += __popcll(v & ~kEven);
            }
            if (sp == 0xFF || ra != (sp & 15) || rb != (sp >> 4)) continue;
            Bits<W> xp;
#pragma unroll
            for (int w = 0; w < W; ++w) xp.w[w] = x.w[w] ^ s_xy[k * W + w];
            bool fresh;
            if (tab.insert(xp, &fresh) < 0) record_status(st, NNQS_E_TABLE_FULL, row_begin + r);
        }
    }
}

// number the occupied slots; keys to the unique list
template <int W>
__global__ void k_compact(HashTab<W> tab, int64_t cap, uint64_t *__restrict__ ulist,
                          unsigned long long *__restrict__ counter) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= cap) return;
    Bits<W> k;
    bool used = false;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        k.w[w] = tab.keys[i * W + w];
        used |= k.w[w] != kEmpty;
    }
    if (!used) return;
    const unsigned long long idx = atomicAdd(counter, 1ull);
#pragma unroll
    for (int w = 0; w < W; ++w) ulist[idx * W + w] = k.w[w];
    tab.vals[i] = (int32_t)idx;
}

template <int W>
__global__ void __launch_bounds__(kThreads)
    k_sweep_exact(const uint64_t *__restrict__ gxy, const uint32_t *__restrict__ goff,
                  const uint8_t *__restrict__ gspin, int64_t g_begin, int64_t g_end, int64_t per_chunk,
                  const uint64_t *__restrict__ tyz, const double *__restrict__ tcoef, const uint64_t *__restrict__ lut,
                  int64_t row_begin, int64_t n_rows, HashTab<W> tab, const double2 *__restrict__ lpU,
                  double2 *__restrict__ partial, DevStatus *st) {
    __shared__ uint64_t s_xy[kTile * W];
    __shared__ uint8_t s_spin[kTile];
    const int64_t r = blockIdx.x * (int64_t)kThreads + threadIdx.x;
    bool active = r < n_rows;
    Bits<W> x{};
    double2 lx = make_double2(0.0, 0.0);
    if (active) {
        x = load_bits<W>(lut, row_begin + r);
        const int32_t self = tab.find(x);
        if (self < 0) {
            record_status(st, NNQS_E_TABLE_FULL, row_begin + r);
            active = false;
        } else {
            lx = lpU[self];
        }
    }
    const int64_t c0 = g_begin + blockIdx.y * per_chunk, c1 = min(g_end, c0 + per_chunk);
    double er = 0.0, ei = 0.0;
    for (int64_t gt = c0; gt < c1; gt += kTile) {
        const int nt = (int)min((int64_t)kTile, c1 - gt);
        __syncthreads();
        for (int k = threadIdx.x; k < nt * W; k += kThreads) s_xy[k] = gxy[gt * W + k];
        for (int k = threadIdx.x; k < nt; k += kThreads) s_spin[k] = gspin[gt + k];
        __syncthreads();
        if (!active) continue;
        for (int k = 0; k < nt; ++k) {
            const uint8_t sp = s_spin[k];
            int ra = 0, rb = 0;
#pragma unroll
            for (int w = 0; w < W; ++w) {
                const uint64_t v = s_xy[k * W + w] & x.w[w];
                ra += __popcll(v & kEven);
                rb += __popcll(v & ~kEven);
            }
            if (sp == 0xFF || ra != (sp & 15) || rb != (sp >> 4)) continue;
            Bits<W> xp;
#pragma unroll
            for (int w = 0; w < W; ++w) xp.w[w] = x.w[w] ^ s_xy[k * W + w];
            const int32_t j = tab.find(xp);
            if (j < 0) continue;  // cannot happen: every such x' was inserted
            const int64_t g = gt + k;
            const double coef = group_coef<W>(x, __ldg(goff + g), __ldg(goff + g + 1), tyz, tcoef);
            const double2 q = ratio(lx, lpU[j]);
            er += coef * q.x;
            ei += coef * q.y;
        }
    }
    if (r < n_rows) partial[blockIdx.y * n_rows + r] = make_double2(er, ei);
}

int sms() {
    static int v = 0;
    if (v == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
    }
    return v;
}

struct Plan {
    int64_t bound, cap, row_tiles, chunks, per_chunk, g_begin, g_end;
    bool has_diag;
};

Plan plan(const nnqs_ham *H, int64_t n_rows) {
    Plan p{};
    p.has_diag = H->n_groups > 0 && H->gxy[0] == 0 && (H->W == 1 || H->gxy[1] == 0);
    p.g_begin = p.has_diag ? 1 : 0;
    p.g_end = H->n_groups;
    p.bound = std::max<int64_t>(1, n_rows * std::max<int64_t>(1, H->n_groups));
    p.cap = pow2_at_least(2 * p.bound);
    const int64_t ng = p.g_end - p.g_begin;
    p.row_tiles = std::max<int64_t>(1, (n_rows + kThreads - 1) / kThreads);
    const int64_t target = 8 * (int64_t)sms();
    const int64_t maxc = std::max<int64_t>(1, (ng + kTile - 1) / kTile);
    p.chunks = std::min(maxc, std::max<int64_t>(1, (target + p.row_tiles - 1) / p.row_tiles));
    p.per_chunk = std::max<int64_t>(1, (ng + p.chunks - 1) / p.chunks);
    p.chunks = ng > 0 ? (ng + p.per_chunk - 1) / p.per_chunk : 0;
    return p;
}

// Steps 1 and 2a: the deduplicated coupled set of rows lut[row_begin, +n_rows)
// in the table (keys, vals) and the unique list ulist (n_U keys, numbered in
// slot order).  Synchronises once to read n_U.  *n_unique = -1 when a kernel
// recorded an error (reported through the status word).
template <int W>
nnqs_status build_coupled(const nnqs_ham *H, const Plan &p, const uint64_t *lut, int64_t row_begin, int64_t n_rows,
                          int n_alpha, int n_beta, HashTab<W> tab, uint64_t *ulist, unsigned long long *counter,
                          DevStatus *st, int64_t *n_unique, cudaStream_t s) {
    NNQS_CUDA_TRY(cudaMemsetAsync(tab.keys, 0xFF, size_t(p.cap) * W * 8, s));
    NNQS_CUDA_TRY(cudaMemsetAsync(counter, 0, 8, s));
    NNQS_LAUNCH("k_insert_rows", s, k_insert_rows<W><<<grid_for(n_rows, 256), 256, 0, s>>>(lut, row_begin, n_rows, H->n_qubits, n_alpha, n_beta, tab, st));
    if (p.chunks > 0) {
        dim3 grid((unsigned)p.row_tiles, (unsigned)p.chunks);
        NNQS_LAUNCH("k_expand", s, k_expand<W><<<grid, kThreads, 0, s>>>(H->d_gxy, H->d_gspin, p.g_begin, p.g_end, p.per_chunk, lut, row_begin,
                                               n_rows, tab, st));
    }
    NNQS_LAUNCH("k_compact", s, k_compact<W><<<grid_for(p.cap, 256), 256, 0, s>>>(tab, p.cap, ulist, counter));
    unsigned long long nU = 0;
    NNQS_CUDA_TRY(cudaMemcpyAsync(&nU, counter, 8, cudaMemcpyDeviceToHost, s));
    NNQS_CUDA_TRY(cudaStreamSynchronize(s));
    DevStatus hst{};
    NNQS_CUDA_TRY(cudaMemcpy(&hst, st, sizeof hst, cudaMemcpyDeviceToHost));
    *n_unique = hst.code != 0 ? -1 : (int64_t)nU;
    if (hst.code == 0 && (int64_t)nU > p.bound) return set_error(NNQS_E_TABLE_FULL, "coupled set larger than its bound");
    return NNQS_OK;
}

template <int W>
nnqs_status exact_impl(const nnqs_ham *H, const nnqs_model *M, const float *params, const uint64_t *lut,
                       int64_t row_begin, int64_t n_rows, int n_alpha, int n_beta, int prec, double *out, Arena &ws,
                       DevStatus *st, cudaStream_t s) {
    const Plan p = plan(H, n_rows);
    uint64_t *keys = ws.take<uint64_t>(size_t(p.cap) * W);
    int32_t *vals = ws.take<int32_t>(size_t(p.cap));
    uint64_t *ulist = ws.take<uint64_t>(size_t(p.bound) * W);
    double *lpU = ws.take<double>(size_t(p.bound) * 2);
    double *diag = ws.take<double>(size_t(std::max<int64_t>(1, n_rows)));
    double2 *partial = ws.take<double2>(size_t(std::max<int64_t>(1, p.chunks * n_rows)));
    unsigned long long *counter = ws.take<unsigned long long>(1);
    if (ws.base == nullptr) {  // sizing: add the forward's workspace over the bound
        ws.take<char>(logpsi_workspace(M, p.bound, prec, false));
        return NNQS_OK;
    }
    if (n_rows == 0) return NNQS_OK;
    HashTab<W> tab{keys, vals, uint64_t(p.cap - 1)};
    int64_t nU = 0;
    NNQS_TRY(build_coupled<W>(H, p, lut, row_begin, n_rows, n_alpha, n_beta, tab, ulist, counter, st, &nU, s));
    if (nU < 0) return NNQS_OK;  // reported through the status word
    NNQS_TRY(logpsi_forward(M, params, ulist, nU, prec, lpU, ws, st, s));
    if (p.has_diag) {
        NNQS_LAUNCH("k_diag", s, k_diag<W><<<grid_for(n_rows * 32, 256), 256, 0, s>>>(lut, row_begin, n_rows, (uint32_t)H->goff[0],
                                                             (uint32_t)H->goff[1], H->d_tyz, H->d_tcoef, diag));
    }
    if (p.chunks > 0) {
        dim3 grid((unsigned)p.row_tiles, (unsigned)p.chunks);
        NNQS_LAUNCH("k_sweep_exact", s, k_sweep_exact<W><<<grid, kThreads, 0, s>>>(H->d_gxy, H->d_goff, H->d_gspin, p.g_begin, p.g_end, p.per_chunk,
                                                   H->d_tyz, H->d_tcoef, lut, row_begin, n_rows, tab,
                                                   reinterpret_cast<const double2 *>(lpU), partial, st));
    }
    NNQS_LAUNCH("k_reduce_partials", s, k_reduce_partials<<<grid_for(n_rows, 256), 256, 0, s>>>(p.has_diag ? diag : nullptr, partial, p.chunks, n_rows,
                                                            reinterpret_cast<double2 *>(out)));
    return NNQS_OK;
}

// Per row, every conserving x' = x ^ m in group order (the identity group
// included, so x itself comes first when the Hamiltonian has a diagonal):
// its index in the unique list and H_{x x'}.  One thread per row walks all
// groups; rows with more than row_cap coupled states record
// NNQS_E_TABLE_FULL (their count is still written).
template <int W>
__global__ void __launch_bounds__(kThreads)
    k_rows_coupled(const uint64_t *__restrict__ gxy, const uint32_t *__restrict__ goff,
                   const uint8_t *__restrict__ gspin, int64_t n_groups, const uint64_t *__restrict__ tyz,
                   const double *__restrict__ tcoef, const uint64_t *__restrict__ lut, int64_t row_begin,
                   int64_t n_rows, HashTab<W> tab, int64_t row_cap, int32_t *__restrict__ row_count,
                   int32_t *__restrict__ row_idx, double *__restrict__ row_hxx, DevStatus *st) {
    __shared__ uint64_t s_xy[kTile * W];
    __shared__ uint8_t s_spin[kTile];
    const int64_t r = blockIdx.x * (int64_t)kThreads + threadIdx.x;
    const bool active = r < n_rows;
    Bits<W> x{};
    if (active) x = load_bits<W>(lut, row_begin + r);
    int64_t k = 0;
    for (int64_t gt = 0; gt < n_groups; gt += kTile) {
        const int nt = (int)min((int64_t)kTile, n_groups - gt);
        __syncthreads();
        for (int q = threadIdx.x; q < nt * W; q += kThreads) s_xy[q] = gxy[gt * W + q];
        for (int q = threadIdx.x; q < nt; q += kThreads) s_spin[q] = gspin[gt + q];
        __syncthreads();
        if (!active) continue;
        for (int q = 0; q < nt; ++q) {
            const uint8_t sp = s_spin[q];
            int ra = 0, rb = 0;
#pragma unroll
            for (int w = 0; w < W; ++w) {
                const uint64_t v = s_xy[q * W + w] & x.w[w];
                ra += __popcll(v & kEven);
                rb += __popcll(v & ~kEven);
            }
            if (sp == 0xFF || ra != (sp & 15) || rb != (sp >> 4)) continue;
            Bits<W> xp;
#pragma unroll
            for (int w = 0; w < W; ++w) xp.w[w] = x.w[w] ^ s_xy[q * W + w];
            const int64_t g = gt + q;
            if (k < row_cap) {
                row_idx[r * row_cap + k] = tab.find(xp);
                row_hxx[r * row_cap + k] = group_coef<W>(x, __ldg(goff + g), __ldg(goff + g + 1), tyz, tcoef);
            }
            ++k;
        }
    }
    if (!active) return;
    row_count[r] = (int32_t)(k < (int64_t)INT32_MAX ? k : (int64_t)INT32_MAX);
    if (k > row_cap) record_status(st, NNQS_E_TABLE_FULL, row_begin + r);
}

template <int W>
nnqs_status coupled_impl(const nnqs_ham *H, const uint64_t *lut, int64_t row_begin, int64_t n_rows, int n_alpha,
                         int n_beta, uint64_t *unique_out, int64_t cap_unique, int64_t *n_unique_out,
                         int32_t *row_count, int32_t *row_idx, double *row_hxx, int64_t row_cap, Arena &ws,
                         DevStatus *st, cudaStream_t s) {
    const Plan p = plan(H, n_rows);
    uint64_t *keys = ws.take<uint64_t>(size_t(p.cap) * W);
    int32_t *vals = ws.take<int32_t>(size_t(p.cap));
    uint64_t *ulist = ws.take<uint64_t>(size_t(p.bound) * W);
    unsigned long long *counter = ws.take<unsigned long long>(1);
    if (ws.base == nullptr || n_rows == 0) return NNQS_OK;
    HashTab<W> tab{keys, vals, uint64_t(p.cap - 1)};
    int64_t nU = 0;
    NNQS_TRY(build_coupled<W>(H, p, lut, row_begin, n_rows, n_alpha, n_beta, tab, ulist, counter, st, &nU, s));
    if (nU < 0) return NNQS_OK;  // reported through the status word
    *n_unique_out = nU;
    if (nU > cap_unique) return set_error(NNQS_E_INVAL, "cap_unique smaller than the coupled set");
    NNQS_CUDA_TRY(cudaMemcpyAsync(unique_out, ulist, size_t(nU) * W * 8, cudaMemcpyDeviceToDevice, s));
    NNQS_LAUNCH("k_rows_coupled", s, k_rows_coupled<W><<<grid_for(n_rows, kThreads), kThreads, 0, s>>>(H->d_gxy, H->d_goff, H->d_gspin, H->n_groups, H->d_tyz, H->d_tcoef, lut,
                                                    row_begin, n_rows, tab, row_cap, row_count, row_idx, row_hxx, st));
    return NNQS_OK;
}

}  // namespace

size_t eloc_exact_workspace(const nnqs_ham *H, const nnqs_model *M, int64_t, int64_t n_rows, int prec) {
    if (!M) return 0;
    Arena a(nullptr);
    a.take<char>(kStatusBytes);
    if (H->W == 1)
        exact_impl<1>(H, M, nullptr, nullptr, 0, n_rows, 0, 0, prec, nullptr, a, nullptr, nullptr);
    else
        exact_impl<2>(H, M, nullptr, nullptr, 0, n_rows, 0, 0, prec, nullptr, a, nullptr, nullptr);
    return a.used + 1024;
}

nnqs_status eloc_exact(const nnqs_ham *H, const nnqs_model *M, const float *params, const uint64_t *lut, int64_t,
                       int64_t row_begin, int64_t n_rows, int n_alpha, int n_beta, int prec, double *out, Arena &ws,
                       DevStatus *st, cudaStream_t s) {
    if (M->N != H->n_qubits) return set_error(NNQS_E_INVAL, "model and Hamiltonian disagree on the qubit count");
    if (M->cfg.n_alpha != n_alpha || M->cfg.n_beta != n_beta)
        return set_error(NNQS_E_INVAL, "model and call disagree on the electron counts");
    if (H->W == 1) return exact_impl<1>(H, M, params, lut, row_begin, n_rows, n_alpha, n_beta, prec, out, ws, st, s);
    return exact_impl<2>(H, M, params, lut, row_begin, n_rows, n_alpha, n_beta, prec, out, ws, st, s);
}

size_t exact_coupled_workspace(const nnqs_ham *H, int64_t n_rows) {
    Arena a(nullptr);
    a.take<char>(kStatusBytes);
    if (H->W == 1)
        coupled_impl<1>(H, nullptr, 0, n_rows, 0, 0, nullptr, 0, nullptr, nullptr, nullptr, nullptr, 0, a, nullptr,
                        nullptr);
    else
        coupled_impl<2>(H, nullptr, 0, n_rows, 0, 0, nullptr, 0, nullptr, nullptr, nullptr, nullptr, 0, a, nullptr,
                        nullptr);
    return a.used + 1024;
}

nnqs_status exact_coupled(const nnqs_ham *H, const uint64_t *lut, int64_t row_begin, int64_t n_rows, int n_alpha,
                          int n_beta, uint64_t *unique_out, int64_t cap_unique, int64_t *n_unique_out,
                          int32_t *row_count, int32_t *row_idx, double *row_hxx, int64_t row_cap, Arena &ws,
                          DevStatus *st, cudaStream_t s) {
    if (H->W == 1)
        return coupled_impl<1>(H, lut, row_begin, n_rows, n_alpha, n_beta, unique_out, cap_unique, n_unique_out,
                               row_count, row_idx, row_hxx, row_cap, ws, st, s);
    return coupled_impl<2>(H, lut, row_begin, n_rows, n_alpha, n_beta, unique_out, cap_unique, n_unique_out,
                           row_count, row_idx, row_hxx, row_cap, ws, st, s);
}

}  // namespace nnqs
