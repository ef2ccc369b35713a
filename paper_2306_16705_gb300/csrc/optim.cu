// Adam update (Kingma & Ba, 2015) and AdamW (Adam with decoupled weight
// decay, Loshchilov & Hutter, 2019: theta <- theta (1 - lr lambda) before the
// Adam step), in place, FP32 state with FP64 bias corrections computed once
// on the host.  The paper trains with AdamW under the warm-up schedule of
// Sec. 4.1 (nnqs_lr_warmup); the learning rate of a step is the caller's.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "internal.h"

namespace nnqs {
namespace {
__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, int64_t n, float lr_t, float b1, float b2, float eps_t,
                       float decay) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = decay == 1.0f ? p[i] : p[i] * decay;
        p[i] = pi - lr_t * mi / (sqrtf(vi) + eps_t);
    }
}
}  // namespace
}  // namespace nnqs

using namespace nnqs;

namespace {
nnqs_status adam_impl(float *params, const float *grad, float *m, float *v, int64_t n, int64_t step, double lr,
                      double beta1, double beta2, double eps, double weight_decay, nnqs_stream stream) {
    if (!params || !grad || !m || !v || n < 0 || step < 1) return set_error(NNQS_E_INVAL, "bad Adam arguments");
    if (!(beta1 >= 0 && beta1 < 1 && beta2 >= 0 && beta2 < 1 && eps > 0 && lr >= 0 && weight_decay >= 0 &&
          lr * weight_decay < 1))
        return set_error(NNQS_E_INVAL, "bad Adam hyperparameters");
    if (n == 0) return NNQS_OK;
    // theta -= lr * mhat / (sqrt(vhat) + eps) with mhat = m / c1, vhat = v / c2
    //       == theta -= (lr * sqrt(c2) / c1) * m / (sqrt(v) + eps * sqrt(c2))
    const double c1 = 1.0 - std::pow(beta1, (double)step), c2 = 1.0 - std::pow(beta2, (double)step);
    const float lr_t = (float)(lr * std::sqrt(c2) / c1), eps_t = (float)(eps * std::sqrt(c2));
    const float decay = (float)(1.0 - lr * weight_decay);
    const int block = 256;
    const int64_t blocks = std::min<int64_t>((n + block - 1) / block, 152 * 16);
    NNQS_LAUNCH("k_adam", (cudaStream_t)stream,
                k_adam<<<(unsigned)blocks, block, 0, (cudaStream_t)stream>>>(params, grad, m, v, n, lr_t, (float)beta1,
                                                                             (float)beta2, eps_t, decay));
    return NNQS_OK;
}
}  // namespace

extern "C" nnqs_status nnqs_adam_step(float *params, const float *grad, float *m, float *v, int64_t n, int64_t step,
                                      double lr, double beta1, double beta2, double eps, nnqs_stream stream) {
    return adam_impl(params, grad, m, v, n, step, lr, beta1, beta2, eps, 0.0, stream);
}

extern "C" nnqs_status nnqs_adamw_step(float *params, const float *grad, float *m, float *v, int64_t n, int64_t step,
                                       double lr, double beta1, double beta2, double eps, double weight_decay,
                                       nnqs_stream stream) {
    return adam_impl(params, grad, m, v, n, step, lr, beta1, beta2, eps, weight_decay, stream);
}

extern "C" double nnqs_lr_warmup(int64_t step, int d_model, int64_t warmup) {
    if (step < 1 || d_model < 1 || warmup < 1) return 0.0;
    const double i = (double)step;
    return std::pow((double)d_model, -0.5) * std::min(std::pow(i, -0.5), i * std::pow((double)warmup, -1.5));
}
