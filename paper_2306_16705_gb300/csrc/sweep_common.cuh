// Device pieces shared by the sample-aware and exact local-energy sweeps.
#pragma once
#include "dev_common.cuh"

namespace nnqs {
namespace {  // internal linkage: included by several translation units

// H_{x x'} for the group [t0, t1): sum_t coef_t (-1)^{popc(x & yz_t)}
template <int W>
__device__ __forceinline__ double group_coef(const Bits<W> &x, uint32_t t0, uint32_t t1,
                                             const uint64_t *__restrict__ tyz,
                                             const double *__restrict__ tcoef) {
    double c = 0.0;
    for (uint32_t t = t0; t < t1; ++t) {
        Bits<W> yz = load_bits<W>(tyz, t);
        double v = __ldg(tcoef + t);
        c += (popc_and<W>(x, yz) & 1) ? -v : v;
    }
    return c;
}

// psi(y)/psi(x) from (log|psi|, phase) pairs
__device__ __forceinline__ double2 ratio(double2 lx, double2 ly) {
    double mag = exp(ly.x - lx.x);
    double s, c;
    sincos(ly.y - lx.y, &s, &c);
    return make_double2(mag * c, mag * s);
}

// psi(y)/psi(x) for one row x against table samples y.  With the table
// psi[j] = exp(log|psi_j| - A) e^{i phase_j} (A = the table's largest
// log|psi|, k_lut_psi) a ratio is one complex product with the row factor
// exp(A - log|psi(x)|) e^{-i phase(x)}: no FP64 exp / sincos per coupled
// sample.  Rows far below the table's maximum (A - log|psi(x)| > 600, where
// the factor or psi[j] could leave the FP64 range) and tables whose maximum is
// not finite keep the direct form.  The two forms differ by a few ulp.
struct RowRatio {
    double2 lx, f;
    bool table;
    __device__ __forceinline__ void init(double2 lx_, const double *__restrict__ amax) {
        lx = lx_;
        const double a = amax ? *amax : 0.0;
        table = amax != nullptr && a - lx.x <= 600.0;
        f = make_double2(0.0, 0.0);
        if (table) {
            const double m = exp(a - lx.x);
            double s, c;
            sincos(lx.y, &s, &c);
            f = make_double2(m * c, -m * s);
        }
    }
    __device__ __forceinline__ double2 of(const double2 *__restrict__ psi, const double2 *__restrict__ lp,
                                          int64_t j) const {
        if (table) {
            const double2 p = psi[j];
            return make_double2(p.x * f.x - p.y * f.y, p.x * f.y + p.y * f.x);
        }
        return ratio(lx, lp[j]);
    }
};

// H_xx for each row: one warp per row over the diagonal group's terms,
// lane-strided then shuffled in a fixed order.
template <int W>
__global__ void k_diag(const uint64_t *__restrict__ lut, int64_t row_begin, int64_t n_rows,
                       uint32_t t0, uint32_t t1, const uint64_t *__restrict__ tyz,
                       const double *__restrict__ tcoef, double *__restrict__ diag) {
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (warp >= n_rows) return;
    Bits<W> x = load_bits<W>(lut, row_begin + warp);
    double c = 0.0;
    for (uint32_t t = t0 + lane; t < t1; t += 32) {
        Bits<W> yz = load_bits<W>(tyz, t);
        double v = __ldg(tcoef + t);
        c += (popc_and<W>(x, yz) & 1) ? -v : v;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) c += __shfl_down_sync(0xffffffffu, c, off);
    if (lane == 0) diag[warp] = c;
}

// out[r] = diag[r] + sum_c partial[c][r], chunks in order
__global__ void k_reduce_partials(const double *__restrict__ diag, const double2 *__restrict__ partial,
                                  int64_t n_chunks, int64_t n_rows, double2 *__restrict__ out) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n_rows) return;
    double re = diag ? diag[r] : 0.0, im = 0.0;
    for (int64_t c = 0; c < n_chunks; ++c) {
        double2 p = partial[c * n_rows + r];
        re += p.x;
        im += p.y;
    }
    out[r] = make_double2(re, im);
}


}  // namespace
}  // namespace nnqs
