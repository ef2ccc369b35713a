// Ansatz handle: configuration and the flat FP32 parameter layout of
// include/nnqs.h.
#pragma once
#include <functional>
#include <string>
#include <vector>

#include "internal.h"

namespace nnqs {

struct LayerOff {
    int64_t ln1_g, ln1_b, wqkv, bqkv, wo, bo, ln2_g, ln2_b, w1, b1, w2, b2;
};

struct ParamLayout {
    int64_t tok_emb, pos_emb;
    std::vector<LayerOff> layer;
    int64_t lnf_g, lnf_b, head_w, head_b;
    int64_t ph_w1, ph_b1, ph_w2, ph_b2, ph_w3, ph_b3;
    int64_t total;
    std::vector<std::pair<std::string, std::pair<int64_t, int64_t>>> named;  // name -> (offset, numel)
};

}  // namespace nnqs

struct nnqs_model {
    nnqs_model_cfg cfg;
    int N, T, W, d, L, H, dh, F, P;  // qubits, tokens, words, width, layers, heads, head dim, FFN width, phase hidden
    nnqs::ParamLayout lay;
};

namespace nnqs {

ParamLayout make_layout(const nnqs_model_cfg &c);

inline bool prec_valid(int p) {
    return p == NNQS_FP64 || p == NNQS_MIXED || p == NNQS_FP32 || p == NNQS_BF16X3 || p == NNQS_FP8;
}
// tensor-core use of a precision: 0 none, 1 BF16 operands, 2 split BF16
// operands in the forward layers, 3 E4M3 operands in the forward layers
inline int tc_mode(int p) { return p == NNQS_MIXED ? 1 : p == NNQS_BF16X3 ? 2 : p == NNQS_FP8 ? 3 : 0; }

// ansatz.cu
size_t logpsi_workspace(const nnqs_model *M, int64_t n, int prec, bool backward);
nnqs_status logpsi_forward(const nnqs_model *M, const float *params, const uint64_t *x, int64_t n, int prec,
                           double *out, Arena &ws, DevStatus *st, cudaStream_t s);
nnqs_status logpsi_backward(const nnqs_model *M, const float *params, const uint64_t *x, int64_t n, int prec,
                            const double *seed, double *grad64, float *grad32, Arena &ws, DevStatus *st,
                            cudaStream_t s);
// true when n samples fit in one backward chunk (then the fused form below applies)
bool logpsi_single_chunk(const nnqs_model *M, int64_t n, int prec);
// log psi of n samples (activations kept) -> between() -> reverse mode with the
// seeds `between` wrote, without a second forward; n must fit in one chunk.
// Workspace: logpsi_workspace(M, n, prec, true).
nnqs_status logpsi_forward_backward(const nnqs_model *M, const float *params, const uint64_t *x, int64_t n, int prec,
                                    double *lp_out, const double *seed, double *grad64, float *grad32, Arena &ws,
                                    DevStatus *st, cudaStream_t s, const std::function<nnqs_status()> &between);

// conditionals pi~(. | prefix) for the sampler (ansatz.cu)
struct CondCtx;
// kv_nodes: capacity of the key/value cache in tree nodes (0 = no cache)
size_t cond_workspace(const nnqs_model *M, int64_t max_prefixes, int prec, int64_t kv_nodes);
nnqs_status cond_create(const nnqs_model *M, const float *params, int prec, int64_t max_prefixes, int64_t kv_nodes,
                        Arena &ws, CondCtx **out, cudaStream_t s);
// full recomputation over the S = t+1 positions of every prefix
nnqs_status cond_step(const nnqs_model *M, CondCtx *ctx, const uint64_t *prefixes, int64_t n, int S, double *cond,
                      DevStatus *st, cudaStream_t s);
// cached: only position t; prefixes are tree nodes g0..g0+n-1 and anc[i][0..t-1]
// (row stride T) the nodes of prefix i's ancestors at depths 0..t-1
nnqs_status cond_step_cached(const nnqs_model *M, CondCtx *ctx, const uint64_t *prefixes, int64_t n, int t,
                             int64_t g0, const int32_t *anc, double *cond, DevStatus *st, cudaStream_t s);
// the cached step with the counts on the device (no host round trip):
// prefixes g0 .. g0 + n - 1 with n = *n_dev <= cap and g0 = *g0_dev; only for
// the fused decode layer (BF16 / split BF16, d = 64) and cap within one chunk
bool cond_cached_dev_ok(const nnqs_model *M, const CondCtx *ctx, int64_t cap);
// the same test from the model and the precision alone (before any context)
bool cond_dev_walk_ok(const nnqs_model *M, int prec, int64_t cap);
nnqs_status cond_step_cached_dev(const nnqs_model *M, CondCtx *ctx, const uint64_t *prefixes, const int64_t *n_dev,
                                 const int64_t *g0_dev, int64_t cap, int t, const int32_t *anc, double *cond,
                                 DevStatus *st, cudaStream_t s, float *act = nullptr,
                                 float *fin = nullptr);
void cond_destroy(CondCtx *c);

// sampler.cu: what an NNQS_SAMPLE_KEEP call left in its workspace -- per tree
// node the layers' input and mid residual rows act[node][L][2][d] and the
// final residual fin[node][d], the last level's depth-major ancestor table
// anc[t * stride + i] (the node of sample i's row t) and its prefixes pref
// [stride][W] (the samples, in the order returned)
struct SampleKept {
    const float *act, *fin;
    const int32_t *anc;
    const uint64_t *pref;
    int64_t stride;
};
bool sample_keep_ok(const nnqs_model *M, int prec, int64_t max_unique);
bool reverse_lite_ok(const nnqs_model *M, int tcm);  // ansatz.cu: the fused reverse mode and its lite workspace apply
nnqs_status sample_kept(const nnqs_model *M, int prec, int64_t max_unique, const void *ws, size_t ws_bytes,
                        SampleKept *out);
// logpsi_forward_backward with the forward's quantities taken from the tree an
// NNQS_SAMPLE_KEEP sampler call kept (x: that call's samples, in its order)
nnqs_status logpsi_forward_backward_rows(const nnqs_model *M, const float *params, const uint64_t *x, int64_t n,
                                         int prec, double *lp_out, const double *seed, double *g64, float *g32,
                                         Arena &ws, DevStatus *st, cudaStream_t s,
                                         const std::function<nnqs_status()> &between, const SampleKept &kept);

// eloc_exact.cu
size_t eloc_exact_workspace(const nnqs_ham *H, const nnqs_model *M, int64_t n_lut, int64_t n_rows, int prec);
nnqs_status eloc_exact(const nnqs_ham *H, const nnqs_model *M, const float *params, const uint64_t *lut,
                       int64_t n_lut, int64_t row_begin, int64_t n_rows, int n_alpha, int n_beta, int prec,
                       double *out, Arena &ws, DevStatus *st, cudaStream_t s);
// the coupled set exact mode builds, exported (nnqs_exact_coupled)
size_t exact_coupled_workspace(const nnqs_ham *H, int64_t n_rows);
nnqs_status exact_coupled(const nnqs_ham *H, const uint64_t *lut, int64_t row_begin, int64_t n_rows, int n_alpha,
                          int n_beta, uint64_t *unique_out, int64_t cap_unique, int64_t *n_unique_out,
                          int32_t *row_count, int32_t *row_idx, double *row_hxx, int64_t row_cap, Arena &ws,
                          DevStatus *st, cudaStream_t s);

}  // namespace nnqs
