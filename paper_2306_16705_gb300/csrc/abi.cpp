// extern "C" entry points of include/nnqs.h: argument checks, workspace
// layout, and dispatch to the kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "internal.h"
#include "model.h"

namespace nnqs {

static thread_local std::string g_last_error;

nnqs_status set_error(nnqs_status st, const std::string &msg) {
    g_last_error = msg;
    return st;
}

nnqs_status cuda_error(cudaError_t e, const char *where) {
    return set_error(NNQS_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

static nnqs_status check_ws(void *ws, size_t have, size_t need) {
    if (ws == nullptr) return set_error(NNQS_E_WORKSPACE, "workspace is null");
    if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return set_error(NNQS_E_WORKSPACE, "workspace not 256-byte aligned");
    if (have < need)
        return set_error(NNQS_E_WORKSPACE, "workspace too small: need " + std::to_string(need) + " bytes, have " +
                                               std::to_string(have));
    return NNQS_OK;
}

// zero the status word at the head of the workspace
static nnqs_status reset_status(void *ws, cudaStream_t s) {
    NNQS_CUDA_TRY(cudaMemsetAsync(ws, 0, sizeof(DevStatus), s));
    return NNQS_OK;
}

// argument checks shared by the local-energy entry points
nnqs_status eloc_args(const nnqs_ham *H, int64_t n_lut, int64_t row_begin, int64_t n_rows, int n_alpha,
                             int n_beta, int mode) {
    if (!H) return set_error(NNQS_E_INVAL, "null Hamiltonian");
    if (!H->d_gxy) return set_error(NNQS_E_INVAL, "Hamiltonian built with nnqs_build_pauli_host has no device tables");
    if (n_lut < 0 || n_rows < 0 || row_begin < 0 || row_begin + n_rows > n_lut)
        return set_error(NNQS_E_INVAL, "rows out of range of the sample table");
    if (n_lut >= (int64_t(1) << 31)) return set_error(NNQS_E_INVAL, "sample table larger than 2^31 rows");
    const int n = H->n_spatial;
    if (n_alpha < 0 || n_beta < 0 || n_alpha > n || n_beta > n)
        return set_error(NNQS_E_INVAL, "electron counts out of range");
    if (H->n_qubits % 64 == 0 && n_alpha == n && n_beta == n)
        return set_error(NNQS_E_UNSUPPORTED, "fully occupied 64/128-qubit sector (all-ones key is the empty marker)");
    if (mode != NNQS_SA && mode != NNQS_EXACT) return set_error(NNQS_E_INVAL, "unknown mode");
    return NNQS_OK;
}

nnqs_status eloc_flags(const nnqs_ham *H, int flags, int mode) {
    if (flags < NNQS_SWEEP_AUTO || flags > NNQS_SWEEP_TERMS) return set_error(NNQS_E_INVAL, "unknown flags");
    if (flags == NNQS_SWEEP_TERMS && mode == NNQS_SA && !H->d_txy)
        return set_error(NNQS_E_INVAL, "NNQS_SWEEP_TERMS needs nnqs_ham_build_ungrouped first");
    return NNQS_OK;
}

}  // namespace nnqs

using namespace nnqs;

extern "C" {

const char *nnqs_last_error(void) { return g_last_error.c_str(); }

const char *nnqs_status_string(int st) {
    switch (st) {
        case NNQS_OK: return "ok";
        case NNQS_E_INVAL: return "invalid argument";
        case NNQS_E_NOMEM: return "out of memory";
        case NNQS_E_CUDA: return "CUDA error";
        case NNQS_E_TABLE_FULL: return "hash table full";
        case NNQS_E_TIMEOUT: return "bounded wait timed out";
        case NNQS_E_SECTOR: return "sample outside the electron-number sector";
        case NNQS_E_NONFINITE: return "non-finite value";
        case NNQS_E_UNSUPPORTED: return "unsupported";
        case NNQS_E_DUPLICATE: return "duplicate sample";
        case NNQS_E_WORKSPACE: return "bad workspace";
        default: return "unknown status";
    }
}

const char *nnqs_version(void) { return "nnqs-gb300 0.1 (sm_103a)"; }

nnqs_status nnqs_workspace_status(const void *workspace, nnqs_stream stream, int64_t *bad_index) {
    if (bad_index) *bad_index = -1;
    if (workspace == nullptr) return set_error(NNQS_E_WORKSPACE, "workspace is null");
    NNQS_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    DevStatus st{};
    NNQS_CUDA_TRY(cudaMemcpy(&st, workspace, sizeof st, cudaMemcpyDeviceToHost));
    if (st.code == 0) return NNQS_OK;
    if (bad_index) *bad_index = st.index;
    return set_error((nnqs_status)st.code, std::string("device reported: ") + nnqs_status_string(st.code) +
                                               " at row " + std::to_string(st.index));
}

// ---------------------------------------------------------------- Hamiltonian
static nnqs_status build_common(int n_spatial, const double *h, const double *eri, double e_core, double drop_tol,
                                nnqs_ham **out, bool upload) {
    if (!out || !h || !eri) return set_error(NNQS_E_INVAL, "null argument");
    *out = nullptr;
    if (n_spatial < 1 || n_spatial > 64) return set_error(NNQS_E_INVAL, "n_spatial must be in 1..64");
    if (!(drop_tol >= 0.0) || !std::isfinite(e_core)) return set_error(NNQS_E_INVAL, "bad drop_tol or e_core");
    const size_t n = n_spatial;
    for (size_t i = 0; i < n * n; ++i)
        if (!std::isfinite(h[i])) return set_error(NNQS_E_NONFINITE, "non-finite one-electron integral");
    for (size_t i = 0; i < n * n * n * n; ++i)
        if (!std::isfinite(eri[i])) return set_error(NNQS_E_NONFINITE, "non-finite two-electron integral");
    nnqs_ham *H = new (std::nothrow) nnqs_ham();
    if (!H) return set_error(NNQS_E_NOMEM, "host allocation failed");
    nnqs_status st = build_pauli_host(n_spatial, h, eri, e_core, drop_tol, H);
    if (st == NNQS_OK && upload) st = upload_ham(H);
    if (st != NNQS_OK) {
        nnqs_ham_free(H);
        return st;
    }
    *out = H;
    return NNQS_OK;
}

nnqs_status nnqs_build_pauli(int n_spatial, const double *h, const double *eri, double e_core, double drop_tol,
                             nnqs_ham **out) {
    return build_common(n_spatial, h, eri, e_core, drop_tol, out, true);
}

nnqs_status nnqs_build_pauli_host(int n_spatial, const double *h, const double *eri, double e_core,
                                  double drop_tol, nnqs_ham **out) {
    return build_common(n_spatial, h, eri, e_core, drop_tol, out, false);
}

nnqs_status nnqs_ham_info(const nnqs_ham *H, int64_t info[6]) {
    if (!H || !info) return set_error(NNQS_E_INVAL, "null argument");
    info[0] = H->n_qubits;
    info[1] = H->W;
    info[2] = H->n_terms;
    info[3] = H->n_groups;
    info[4] = H->max_group;
    info[5] = (int64_t)H->device_bytes;
    return NNQS_OK;
}

nnqs_status nnqs_ham_export(const nnqs_ham *H, uint64_t *xy, int64_t *off, uint64_t *yz, double *coef) {
    if (!H) return set_error(NNQS_E_INVAL, "null handle");
    if (xy) std::memcpy(xy, H->gxy.data(), H->gxy.size() * 8);
    if (off) std::memcpy(off, H->goff.data(), H->goff.size() * 8);
    if (yz) std::memcpy(yz, H->tyz.data(), H->tyz.size() * 8);
    if (coef) std::memcpy(coef, H->tcoef.data(), H->tcoef.size() * 8);
    return NNQS_OK;
}

void nnqs_ham_free(nnqs_ham *H) {
    if (!H) return;
    cudaFree(H->d_gxy);
    cudaFree(H->d_goff);
    cudaFree(H->d_gspin);
    cudaFree(H->d_tyz);
    cudaFree(H->d_tcoef);
    cudaFree(H->d_ghkeys);
    cudaFree(H->d_ghvals);
    cudaFree(H->d_txy);
    delete H;
}

nnqs_status nnqs_ham_build_ungrouped(nnqs_ham *H) {
    if (!H) return set_error(NNQS_E_INVAL, "null handle");
    if (!H->d_gxy) return set_error(NNQS_E_INVAL, "Hamiltonian has no device tables");
    if (H->d_txy) return NNQS_OK;
    const int W = H->W;
    std::vector<uint64_t> txy(size_t(std::max<int64_t>(H->n_terms, 1)) * W, 0);
    for (int64_t g = 0; g < H->n_groups; ++g)
        for (int64_t t = H->goff[g]; t < H->goff[g + 1]; ++t)
            for (int w = 0; w < W; ++w) txy[size_t(t) * W + w] = H->gxy[size_t(g) * W + w];
    const size_t bytes = txy.size() * 8;
    cudaError_t e = cudaMalloc(&H->d_txy, bytes);
    if (e != cudaSuccess) {
        H->d_txy = nullptr;
        return cuda_error(e, "cudaMalloc (ungrouped X/Y masks)");
    }
    e = cudaMemcpy(H->d_txy, txy.data(), bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_error(e, "cudaMemcpy (ungrouped X/Y masks)");
    H->ungrouped_bytes = bytes;
    return NNQS_OK;
}

nnqs_status nnqs_ham_layout_bytes(const nnqs_ham *H, int64_t bytes[4]) {
    if (!H || !bytes) return set_error(NNQS_E_INVAL, "null argument");
    const int64_t W = H->W, T = H->n_terms, G = H->n_groups, N = H->n_qubits;
    bytes[0] = G * (8 * W + 4 + 1) + T * (8 * W + 8);  // grouped: masks, offsets, spin codes; terms: Y/Z, coef
    bytes[1] = T * (16 * W + 8);                       // ungrouped: X/Y, Y/Z, coef per term
    bytes[2] = G * (N + 4) + T * (N + 8);              // grouped, one byte per qubit
    bytes[3] = T * (2 * N + 4 + 8);                    // ungrouped, one byte per qubit (+ 4-byte Y count)
    return NNQS_OK;
}

nnqs_status nnqs_coupled_host(const nnqs_ham *H, const uint64_t *x, int n_alpha, int n_beta, uint64_t *xp,
                              double *hxx, int64_t cap, int64_t *count) {
    if (!H || !x || !count) return set_error(NNQS_E_INVAL, "null argument");
    const int W = H->W;
    int64_t k = 0;
    for (int64_t g = 0; g < H->n_groups; ++g) {
        uint64_t y[2] = {0, 0};
        int na = 0, nb = 0;
        for (int w = 0; w < W; ++w) {
            y[w] = x[w] ^ H->gxy[g * W + w];
            na += __builtin_popcountll(y[w] & kEven);
            nb += __builtin_popcountll(y[w] & ~kEven);
        }
        if (na != n_alpha || nb != n_beta) continue;
        double c = 0.0;
        for (int64_t t = H->goff[g]; t < H->goff[g + 1]; ++t) {
            int par = 0;
            for (int w = 0; w < W; ++w) par += __builtin_popcountll(x[w] & H->tyz[t * W + w]);
            c += (par & 1) ? -H->tcoef[t] : H->tcoef[t];
        }
        if (k < cap) {
            if (xp)
                for (int w = 0; w < W; ++w) xp[k * W + w] = y[w];
            if (hxx) hxx[k] = c;
        }
        ++k;
    }
    *count = k;
    if (k > cap) return set_error(NNQS_E_INVAL, "cap smaller than the coupled set");
    return NNQS_OK;
}

// ---------------------------------------------------------------- local energy
size_t nnqs_eloc_workspace_size(const nnqs_ham *H, const nnqs_model *M, int64_t n_lut, int64_t n_rows, int mode,
                                int prec) {
    if (!H || n_lut < 0 || n_rows < 0) return 0;
    if (mode == NNQS_SA) return eloc_sa_workspace(H, n_lut, n_rows, NNQS_SWEEP_AUTO) + 4096;
    return eloc_exact_workspace(H, M, n_lut, n_rows, prec);
}

nnqs_status nnqs_eloc(const nnqs_ham *H, const nnqs_model *M, const float *params, const uint64_t *lut,
                      const double *lut_logpsi, int64_t n_lut, int64_t row_begin, int64_t n_rows, int n_alpha,
                      int n_beta, int mode, int prec, int flags, double *eloc_out, void *workspace,
                      size_t workspace_bytes, nnqs_stream stream) {
    NNQS_TRY(eloc_args(H, n_lut, row_begin, n_rows, n_alpha, n_beta, mode));
    NNQS_TRY(eloc_flags(H, flags, mode));
    if (n_rows > 0 && (!lut || !eloc_out)) return set_error(NNQS_E_INVAL, "null device pointer");
    cudaStream_t s = (cudaStream_t)stream;
    if (mode == NNQS_SA) {
        if (n_lut > 0 && !lut_logpsi) return set_error(NNQS_E_INVAL, "lut_logpsi required in NNQS_SA mode");
        NNQS_TRY(check_ws(workspace, workspace_bytes, eloc_sa_workspace(H, n_lut, n_rows, flags)));
        NNQS_TRY(reset_status(workspace, s));
        Arena a(workspace);
        DevStatus *st = a.take<DevStatus>(kStatusBytes / sizeof(DevStatus));
        return eloc_sa(H, lut, lut_logpsi, n_lut, row_begin, n_rows, n_alpha, n_beta, flags, eloc_out, a, st, s);
    }
    if (!M || !params) return set_error(NNQS_E_INVAL, "NNQS_EXACT needs the model and its parameters");
    if (!prec_valid(prec)) return set_error(NNQS_E_INVAL, "bad precision");
    NNQS_TRY(check_ws(workspace, workspace_bytes, eloc_exact_workspace(H, M, n_lut, n_rows, prec)));
    NNQS_TRY(reset_status(workspace, s));
    Arena a(workspace);
    DevStatus *st = a.take<DevStatus>(kStatusBytes / sizeof(DevStatus));
    return eloc_exact(H, M, params, lut, n_lut, row_begin, n_rows, n_alpha, n_beta, prec, eloc_out, a, st, s);
}

size_t nnqs_exact_coupled_workspace_size(const nnqs_ham *H, int64_t n_rows) {
    if (!H || n_rows < 0) return 0;
    return exact_coupled_workspace(H, n_rows);
}

nnqs_status nnqs_exact_coupled(const nnqs_ham *H, const uint64_t *lut, int64_t n_lut, int64_t row_begin,
                               int64_t n_rows, int n_alpha, int n_beta, uint64_t *unique_out, int64_t cap_unique,
                               int64_t *n_unique_out, int32_t *row_count, int32_t *row_idx, double *row_hxx,
                               int64_t row_cap, void *workspace, size_t workspace_bytes, nnqs_stream stream) {
    NNQS_TRY(eloc_args(H, n_lut, row_begin, n_rows, n_alpha, n_beta, NNQS_EXACT));
    if (!n_unique_out) return set_error(NNQS_E_INVAL, "null n_unique_out");
    *n_unique_out = 0;
    if (cap_unique < 0 || row_cap < 0) return set_error(NNQS_E_INVAL, "negative capacity");
    if (n_rows > 0 && (!lut || !unique_out || !row_count || (row_cap > 0 && (!row_idx || !row_hxx))))
        return set_error(NNQS_E_INVAL, "null device pointer");
    cudaStream_t s = (cudaStream_t)stream;
    NNQS_TRY(check_ws(workspace, workspace_bytes, exact_coupled_workspace(H, n_rows)));
    NNQS_TRY(reset_status(workspace, s));
    Arena a(workspace);
    DevStatus *st = a.take<DevStatus>(kStatusBytes / sizeof(DevStatus));
    return exact_coupled(H, lut, row_begin, n_rows, n_alpha, n_beta, unique_out, cap_unique, n_unique_out, row_count,
                         row_idx, row_hxx, row_cap, a, st, s);
}

// ---------------------------------------------------------------- statistics
size_t nnqs_energy_stats_workspace_size(int64_t n) { return stats_workspace(n); }

nnqs_status nnqs_energy_stats(const double *eloc, const uint64_t *weights, int64_t n, double *stats, void *workspace,
                              size_t workspace_bytes, nnqs_stream stream) {
    if (n <= 0 || !eloc || !weights || !stats) return set_error(NNQS_E_INVAL, "bad arguments");
    NNQS_TRY(check_ws(workspace, workspace_bytes, stats_workspace(n)));
    cudaStream_t s = (cudaStream_t)stream;
    NNQS_TRY(reset_status(workspace, s));
    Arena a(workspace);
    a.take<char>(kStatusBytes);
    return energy_stats(eloc, weights, n, stats, a, s);
}

}  // extern "C"
