// Placeholder until the tcgen05 kernel lands: NNQS_MIXED reports
// NNQS_E_UNSUPPORTED.
#include "tc_gemm.h"

namespace nnqs {
void tc_weights_take(const nnqs_model *, Arena &, TcWeights *) {}
nnqs_status tc_weights_prepare(const nnqs_model *, const float *, TcWeights &, cudaStream_t) {
    return set_error(NNQS_E_UNSUPPORTED, "tensor-core path not built yet");
}
template <class R>
nnqs_status tc_linear_fwd(cudaStream_t, const TcWeights &, int, int, const R *, int64_t, int64_t, const R *, R *, R *,
                          const R *) {
    return set_error(NNQS_E_UNSUPPORTED, "tensor-core path not built yet");
}
template nnqs_status tc_linear_fwd<float>(cudaStream_t, const TcWeights &, int, int, const float *, int64_t, int64_t,
                                          const float *, float *, float *, const float *);
template nnqs_status tc_linear_fwd<double>(cudaStream_t, const TcWeights &, int, int, const double *, int64_t, int64_t,
                                           const double *, double *, double *, const double *);
template <class R>
nnqs_status tc_linear_fwd_ld(cudaStream_t, const TcWeights &, int, int, const R *, int64_t, int64_t, const R *, R *,
                             int64_t, R *, const R *) {
    return set_error(NNQS_E_UNSUPPORTED, "tensor-core path not built yet");
}
template nnqs_status tc_linear_fwd_ld<float>(cudaStream_t, const TcWeights &, int, int, const float *, int64_t,
                                             int64_t, const float *, float *, int64_t, float *, const float *);
template nnqs_status tc_linear_fwd_ld<double>(cudaStream_t, const TcWeights &, int, int, const double *, int64_t,
                                              int64_t, const double *, double *, int64_t, double *, const double *);
}  // namespace nnqs
