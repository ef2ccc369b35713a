// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/nnqs.h"

namespace nnqs {

// ---- error reporting ------------------------------------------------------
nnqs_status set_error(nnqs_status st, const std::string &msg);
nnqs_status cuda_error(cudaError_t e, const char *where);

#define NNQS_CUDA_TRY(expr)                                      \
    do {                                                         \
        cudaError_t _e = (expr);                                 \
        if (_e != cudaSuccess) return nnqs::cuda_error(_e, #expr); \
    } while (0)

#define NNQS_TRY(expr)                       \
    do {                                     \
        nnqs_status _s = (expr);             \
        if (_s != NNQS_OK) return _s;        \
    } while (0)

// ---- launches: counting and optional CUDA-event timing (prof.cpp) ---------
cudaError_t note_launch();  // counts one launch, returns cudaGetLastError()
void note_replay(uint64_t launches);  // a CUDA-graph replay of that many kernel launches
bool profiling_on();
// algorithmic work (flops, bytes) of a launch, for roofline accounting
void note_work(const char *name, double flops, double bytes);
class ProfScope {
   public:
    ProfScope(const char *name, cudaStream_t s);
    ~ProfScope();

   private:
    const char *name_;
    cudaStream_t s_;
    cudaEvent_t e0_{}, e1_{};
    bool on_ = false;
};

// every kernel launch of the library goes through this macro
#define NNQS_LAUNCH(name, stream, ...)                   \
    do {                                                 \
        nnqs::ProfScope _nnqs_ps((name), (stream));      \
        __VA_ARGS__;                                     \
        NNQS_CUDA_TRY(nnqs::note_launch());              \
    } while (0)

// ---- device status word (first 256 bytes of every workspace) --------------
// code: first error recorded (atomicCAS from 0); index: offending row.
struct DevStatus {
    int32_t code;
    int32_t pad;
    long long index;
};
constexpr size_t kStatusBytes = 256;

// ---- bump allocator over a caller workspace --------------------------------
struct Arena {
    char *base;      // may be null when only sizing
    size_t used = 0;
    explicit Arena(void *b) : base(static_cast<char *>(b)) {}
    template <class T>
    T *take(size_t count) {
        size_t off = (used + 255) & ~size_t(255);
        used = off + count * sizeof(T);
        return base ? reinterpret_cast<T *>(base + off) : nullptr;
    }
};

// ---- Hamiltonian handle -----------------------------------------------------
constexpr uint64_t kEven = 0x5555555555555555ull;  // alpha qubits (even bits)

}  // namespace nnqs

struct nnqs_ham {
    int n_spatial = 0, n_qubits = 0, W = 1;
    int64_t n_terms = 0, n_groups = 0, max_group = 0;
    int max_xy_weight = 0;  // largest popcount of a group X/Y mask
    // host tables (Alg. 1 output)
    std::vector<uint64_t> gxy;   // [G][W]
    std::vector<int64_t> goff;   // [G+1]
    std::vector<uint64_t> tyz;   // [T][W]
    std::vector<double> tcoef;   // [T]
    // device tables
    uint64_t *d_gxy = nullptr;     // [G][W]
    uint32_t *d_goff = nullptr;    // [G+1]
    uint8_t *d_gspin = nullptr;    // [G] (popc(m&A)/2) | (popc(m&B)/2) << 4, 0xFF = never conserving
    uint64_t *d_tyz = nullptr;     // [T][W]
    double *d_tcoef = nullptr;     // [T]
    // X/Y mask -> group index, open addressing (for the pair sweep)
    uint64_t *d_ghkeys = nullptr;  // [cap][W], all-ones = empty
    int32_t *d_ghvals = nullptr;   // [cap]
    int64_t ghcap = 0;
    size_t device_bytes = 0;
    // ungrouped layout (every term with its own X/Y mask), built on request
    // for the layout comparison of Sec. 3.4 (nnqs_ham_build_ungrouped)
    uint64_t *d_txy = nullptr;     // [T][W]
    size_t ungrouped_bytes = 0;
};

namespace nnqs {
// ham_build.cpp
nnqs_status build_pauli_host(int n_spatial, const double *h, const double *eri, double e_core,
                             double drop_tol, nnqs_ham *H);
nnqs_status upload_ham(nnqs_ham *H);
uint64_t hash_words(const uint64_t *k, int W);  // same mix as the device hash

// abi.cpp: argument checks shared by the local-energy entry points
nnqs_status eloc_args(const nnqs_ham *H, int64_t n_lut, int64_t row_begin, int64_t n_rows, int n_alpha, int n_beta,
                      int mode);
nnqs_status eloc_flags(const nnqs_ham *H, int flags, int mode);

// eloc.cu
int num_sms();  // SMs of the current device (152 if the query fails)
// bytes for any sweep (the size query takes no flags)
size_t eloc_sa_workspace(const nnqs_ham *H, int64_t n_lut, int64_t n_rows, int flags);
// bytes for the sweep a call with `flags` runs (AUTO resolved)
size_t eloc_sa_workspace_for(const nnqs_ham *H, int64_t n_lut, int64_t n_rows, int flags);
nnqs_status eloc_sa(const nnqs_ham *H, const uint64_t *lut, const double *lut_lp, int64_t n_lut,
                    int64_t row_begin, int64_t n_rows, int n_alpha, int n_beta, int flags,
                    double *out, Arena &ws, DevStatus *status, cudaStream_t s);
size_t stats_workspace(int64_t n);
nnqs_status energy_stats(const double *eloc, const uint64_t *w, int64_t n, double *stats,
                         Arena &ws, cudaStream_t s);
}  // namespace nnqs
