// nnqs_energy_grad: one energy and gradient evaluation on the unique
// samples of a VMC step (Sec. 2.1):
//   log psi(S)                       ansatz forward
//   E_loc(S) restricted to S         Alg. 2 (sample-aware)
//   E, Var                           Eq. (energy) with sample counts
//   seeds 2 w (E_loc - E)/sum w      gradient estimator, E_loc held fixed
//   grad                             ansatz reverse mode
// When the samples fit in one activation chunk the forward's activations are
// kept for the reverse mode (one forward per call); otherwise the reverse
// mode recomputes them chunk by chunk.  Every stage is enqueued on the
// caller's stream; no host synchronisation.
#include <cuda_runtime.h>

#include <algorithm>

#include "dev_common.cuh"
#include "internal.h"
#include "model.h"

namespace nnqs {
namespace {

// seed_i = 2 w_i (E_loc,i - E) / sum w as (Re -> d log|psi|, Im -> d phase):
// 2 Re[(E_loc - E) d ln psi*] = 2 Re(E_loc - E) d log|psi| + 2 Im(E_loc - E) d phase
__global__ void k_seeds(const double2 *__restrict__ eloc, const uint64_t *__restrict__ w,
                        const double *__restrict__ stats, int64_t n, double2 *__restrict__ seed) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double f = 2.0 * (double)w[i] / stats[3];
    seed[i] = make_double2(f * (eloc[i].x - stats[0]), f * (eloc[i].y - stats[1]));
}

// fused: the ansatz keeps its activations in `region` while E_loc and the
// statistics run in `region2`; otherwise every stage reuses `region`
struct Layout {
    double *lp, *eloc, *seed;
    bool fused;
    char *region, *region2;
};

Layout layout(const nnqs_ham *H, const nnqs_model *M, int64_t n, int prec, Arena &a) {
    Layout L{};
    L.lp = a.take<double>(size_t(2 * std::max<int64_t>(n, 1)));
    L.eloc = a.take<double>(size_t(2 * std::max<int64_t>(n, 1)));
    L.seed = a.take<double>(size_t(2 * std::max<int64_t>(n, 1)));
    const size_t ew = std::max(eloc_sa_workspace(H, n, n, NNQS_SWEEP_AUTO), stats_workspace(n));
    L.fused = logpsi_single_chunk(M, n, prec);
    if (L.fused) {
        L.region = a.take<char>(logpsi_workspace(M, n, prec, true));
        L.region2 = a.take<char>(ew);
    } else {
        L.region = a.take<char>(std::max({ew, logpsi_workspace(M, n, prec, false), logpsi_workspace(M, n, prec, true)}));
        L.region2 = L.region;
    }
    return L;
}

}  // namespace
}  // namespace nnqs

using namespace nnqs;

extern "C" size_t nnqs_energy_grad_workspace_size(const nnqs_ham *H, const nnqs_model *M, int64_t n_u, int prec) {
    if (!H || !M || n_u < 0) return 0;
    Arena a(nullptr);
    a.take<char>(kStatusBytes);
    layout(H, M, n_u, prec, a);
    return a.used + 1024;
}

extern "C" nnqs_status nnqs_energy_grad(const nnqs_ham *H, const nnqs_model *M, const float *params,
                                        const uint64_t *samples, const uint64_t *weights, int64_t n_u, int prec,
                                        double *stats, double *eloc_out, double *grad_f64, float *grad_f32,
                                        void *workspace, size_t workspace_bytes, nnqs_stream stream) {
    if (!H || !M || n_u <= 0) return set_error(NNQS_E_INVAL, "null handle or empty sample set");
    if (!H->d_gxy) return set_error(NNQS_E_INVAL, "Hamiltonian has no device tables");
    if (!params || !samples || !weights || !stats || (!grad_f64 && !grad_f32))
        return set_error(NNQS_E_INVAL, "null device pointer");
    if (M->N != H->n_qubits) return set_error(NNQS_E_INVAL, "model and Hamiltonian disagree on the qubit count");
    if (!prec_valid(prec)) return set_error(NNQS_E_INVAL, "bad precision");
    if (n_u >= (int64_t(1) << 31)) return set_error(NNQS_E_INVAL, "more than 2^31 samples");
    const size_t need = nnqs_energy_grad_workspace_size(H, M, n_u, prec);
    if (!workspace || reinterpret_cast<uintptr_t>(workspace) % 256 || workspace_bytes < need)
        return set_error(NNQS_E_WORKSPACE, "workspace null, misaligned or smaller than " + std::to_string(need));
    cudaStream_t s = (cudaStream_t)stream;
    NNQS_CUDA_TRY(cudaMemsetAsync(workspace, 0, sizeof(DevStatus), s));
    Arena a(workspace);
    DevStatus *st = a.take<DevStatus>(kStatusBytes / sizeof(DevStatus));
    const Layout L = layout(H, M, n_u, prec, a);
    double *eloc = eloc_out ? eloc_out : L.eloc;
    // E_loc over S with the table log psi(S), statistics, seeds
    auto middle = [&]() -> nnqs_status {
        {
            Arena sub(L.region2);
            NNQS_TRY(eloc_sa(H, samples, L.lp, n_u, 0, n_u, M->cfg.n_alpha, M->cfg.n_beta, NNQS_SWEEP_AUTO, eloc,
                             sub, st, s));
        }
        {
            Arena sub(L.region2);
            NNQS_TRY(energy_stats(eloc, weights, n_u, stats, sub, s));
        }
        NNQS_LAUNCH("k_seeds", s, k_seeds<<<grid_for(n_u, 256), 256, 0, s>>>(reinterpret_cast<const double2 *>(eloc),
                                                                           weights, stats, n_u,
                                                                           reinterpret_cast<double2 *>(L.seed)));
        return NNQS_OK;
    };
    if (L.fused) {
        Arena sub(L.region);
        return logpsi_forward_backward(M, params, samples, n_u, prec, L.lp, L.seed, grad_f64, grad_f32, sub, st, s,
                                       middle);
    }
    {
        Arena sub(L.region);
        NNQS_TRY(logpsi_forward(M, params, samples, n_u, prec, L.lp, sub, st, s));
    }
    NNQS_TRY(middle());
    {
        Arena sub(L.region);
        NNQS_TRY(logpsi_backward(M, params, samples, n_u, prec, L.seed, grad_f64, grad_f32, sub, st, s));
    }
    return NNQS_OK;
}

extern "C" int nnqs_energy_grad_sampled_supported(const nnqs_model *M, int prec, int64_t max_unique) {
    const int tcm = tc_mode(prec);
    return M && (tcm == 1 || tcm == 2) && sample_keep_ok(M, prec, max_unique) && reverse_lite_ok(M, tcm) ? 1 : 0;
}

extern "C" size_t nnqs_energy_grad_sampled_workspace_size(const nnqs_ham *H, const nnqs_model *M, int64_t n_u,
                                                          int prec) {
    return nnqs_energy_grad_workspace_size(H, M, n_u, prec);
}

extern "C" nnqs_status nnqs_energy_grad_sampled(const nnqs_ham *H, const nnqs_model *M, const float *params,
                                                const void *sample_workspace, size_t sample_workspace_bytes,
                                                int64_t max_unique, const uint64_t *samples, const uint64_t *weights,
                                                int64_t n_u, int prec, double *stats, double *eloc_out,
                                                double *grad_f64, float *grad_f32, void *workspace,
                                                size_t workspace_bytes, nnqs_stream stream) {
    if (!H || !M || n_u <= 0) return set_error(NNQS_E_INVAL, "null handle or empty sample set");
    if (!H->d_gxy) return set_error(NNQS_E_INVAL, "Hamiltonian has no device tables");
    if (!params || !samples || !weights || !stats || (!grad_f64 && !grad_f32))
        return set_error(NNQS_E_INVAL, "null device pointer");
    if (M->N != H->n_qubits) return set_error(NNQS_E_INVAL, "model and Hamiltonian disagree on the qubit count");
    if (!prec_valid(prec)) return set_error(NNQS_E_INVAL, "bad precision");
    if (n_u > max_unique) return set_error(NNQS_E_INVAL, "more samples than the sampler call's max_unique");
    SampleKept kept{};
    NNQS_TRY(sample_kept(M, prec, max_unique, sample_workspace, sample_workspace_bytes, &kept));
    const size_t need = nnqs_energy_grad_sampled_workspace_size(H, M, n_u, prec);
    if (!workspace || reinterpret_cast<uintptr_t>(workspace) % 256 || workspace_bytes < need)
        return set_error(NNQS_E_WORKSPACE, "workspace null, misaligned or smaller than " + std::to_string(need));
    cudaStream_t s = (cudaStream_t)stream;
    NNQS_CUDA_TRY(cudaMemsetAsync(workspace, 0, sizeof(DevStatus), s));
    Arena a(workspace);
    DevStatus *st = a.take<DevStatus>(kStatusBytes / sizeof(DevStatus));
    const Layout L = layout(H, M, n_u, prec, a);
    if (!L.fused) return set_error(NNQS_E_INVAL, "more samples than one activation chunk");
    double *eloc = eloc_out ? eloc_out : L.eloc;
    auto middle = [&]() -> nnqs_status {
        {
            Arena sub(L.region2);
            NNQS_TRY(eloc_sa(H, samples, L.lp, n_u, 0, n_u, M->cfg.n_alpha, M->cfg.n_beta, NNQS_SWEEP_AUTO, eloc,
                             sub, st, s));
        }
        {
            Arena sub(L.region2);
            NNQS_TRY(energy_stats(eloc, weights, n_u, stats, sub, s));
        }
        NNQS_LAUNCH("k_seeds", s, k_seeds<<<grid_for(n_u, 256), 256, 0, s>>>(reinterpret_cast<const double2 *>(eloc),
                                                                           weights, stats, n_u,
                                                                           reinterpret_cast<double2 *>(L.seed)));
        return NNQS_OK;
    };
    Arena sub(L.region);
    return logpsi_forward_backward_rows(M, params, samples, n_u, prec, L.lp, L.seed, grad_f64, grad_f32, sub, st, s,
                                        middle, kept);
}

