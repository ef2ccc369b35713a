// Ansatz handle, parameter layout and the entry points that run the ansatz
// (nnqs_logpsi, nnqs_logpsi_backward, nnqs_energy_grad).
#include <cstring>
#include <new>

#include "model.h"

namespace nnqs {

ParamLayout make_layout(const nnqs_model_cfg &c) {
    ParamLayout L{};
    const int64_t d = c.d_model, N = c.n_qubits, T = N / 2, Hh = c.phase_hidden;
    int64_t off = 0;
    auto put = [&](const std::string &name, int64_t numel) {
        int64_t o = off;
        L.named.push_back({name, {o, numel}});
        off += numel;
        return o;
    };
    L.tok_emb = put("tok_emb", 5 * d);
    L.pos_emb = put("pos_emb", T * d);
    for (int l = 0; l < c.n_layers; ++l) {
        const std::string p = "l" + std::to_string(l) + ".";
        LayerOff lo{};
        lo.ln1_g = put(p + "ln1.g", d);
        lo.ln1_b = put(p + "ln1.b", d);
        lo.wqkv = put(p + "attn.wqkv", 3 * d * d);
        lo.bqkv = put(p + "attn.bqkv", 3 * d);
        lo.wo = put(p + "attn.wo", d * d);
        lo.bo = put(p + "attn.bo", d);
        lo.ln2_g = put(p + "ln2.g", d);
        lo.ln2_b = put(p + "ln2.b", d);
        lo.w1 = put(p + "ffn.w1", 4 * d * d);
        lo.b1 = put(p + "ffn.b1", 4 * d);
        lo.w2 = put(p + "ffn.w2", 4 * d * d);
        lo.b2 = put(p + "ffn.b2", d);
        L.layer.push_back(lo);
    }
    L.lnf_g = put("lnf.g", d);
    L.lnf_b = put("lnf.b", d);
    L.head_w = put("head.w", 4 * d);
    L.head_b = put("head.b", 4);
    L.ph_w1 = put("phase.w1", Hh * N);
    L.ph_b1 = put("phase.b1", Hh);
    L.ph_w2 = put("phase.w2", Hh * Hh);
    L.ph_b2 = put("phase.b2", Hh);
    L.ph_w3 = put("phase.w3", Hh);
    L.ph_b3 = put("phase.b3", 1);
    L.total = off;
    return L;
}

}  // namespace nnqs

using namespace nnqs;

static nnqs_status check_ws2(void *ws, size_t have, size_t need) {
    if (ws == nullptr) return set_error(NNQS_E_WORKSPACE, "workspace is null");
    if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return set_error(NNQS_E_WORKSPACE, "workspace not 256-byte aligned");
    if (have < need) return set_error(NNQS_E_WORKSPACE, "workspace too small: need " + std::to_string(need));
    return NNQS_OK;
}

static bool prec_ok(int p) { return prec_valid(p); }

extern "C" {

nnqs_status nnqs_model_create(const nnqs_model_cfg *cfg, nnqs_model **out) {
    if (!cfg || !out) return set_error(NNQS_E_INVAL, "null argument");
    *out = nullptr;
    const nnqs_model_cfg &c = *cfg;
    if (c.n_qubits < 2 || c.n_qubits > 128 || c.n_qubits % 2) return set_error(NNQS_E_INVAL, "n_qubits must be even, 2..128");
    const int n = c.n_qubits / 2;
    if (c.n_alpha < 0 || c.n_beta < 0 || c.n_alpha > n || c.n_beta > n) return set_error(NNQS_E_INVAL, "bad electron counts");
    if (c.d_model < 1 || c.n_heads < 1 || c.d_model % c.n_heads) return set_error(NNQS_E_INVAL, "d_model must be a multiple of n_heads");
    if (c.d_model > 256 || c.d_model / c.n_heads > 64) return set_error(NNQS_E_UNSUPPORTED, "d_model <= 256 and head dim <= 64 supported");
    if (c.n_layers < 0 || c.n_layers > 64 || c.phase_hidden < 1 || c.phase_hidden > 4096 || c.reserved != 0)
        return set_error(NNQS_E_INVAL, "bad layer count, phase width or reserved field");
    nnqs_model *M = new (std::nothrow) nnqs_model();
    if (!M) return set_error(NNQS_E_NOMEM, "host allocation failed");
    M->cfg = c;
    M->N = c.n_qubits;
    M->T = n;
    M->W = (c.n_qubits + 63) / 64;
    M->d = c.d_model;
    M->L = c.n_layers;
    M->H = c.n_heads;
    M->dh = c.d_model / c.n_heads;
    M->F = 4 * c.d_model;
    M->P = c.phase_hidden;
    M->lay = make_layout(c);
    *out = M;
    return NNQS_OK;
}

void nnqs_model_free(nnqs_model *M) { delete M; }

int64_t nnqs_model_param_count(const nnqs_model *M) { return M ? M->lay.total : -1; }

nnqs_status nnqs_model_param_offset(const nnqs_model *M, const char *name, int64_t *offset, int64_t *numel) {
    if (!M || !name) return set_error(NNQS_E_INVAL, "null argument");
    for (auto &e : M->lay.named)
        if (e.first == name) {
            if (offset) *offset = e.second.first;
            if (numel) *numel = e.second.second;
            return NNQS_OK;
        }
    return set_error(NNQS_E_INVAL, std::string("no parameter named ") + name);
}

size_t nnqs_logpsi_workspace_size(const nnqs_model *M, int64_t n, int prec) {
    if (!M || n < 0 || !prec_ok(prec)) return 0;
    return logpsi_workspace(M, n, prec, false);
}

nnqs_status nnqs_logpsi(const nnqs_model *M, const float *params, const uint64_t *x, int64_t n, int prec, double *out,
                        void *workspace, size_t workspace_bytes, nnqs_stream stream) {
    if (!M || n < 0 || !prec_ok(prec)) return set_error(NNQS_E_INVAL, "bad model, count or precision");
    if (n > 0 && (!params || !x || !out)) return set_error(NNQS_E_INVAL, "null device pointer");
    NNQS_TRY(check_ws2(workspace, workspace_bytes, logpsi_workspace(M, n, prec, false)));
    cudaStream_t s = (cudaStream_t)stream;
    NNQS_CUDA_TRY(cudaMemsetAsync(workspace, 0, sizeof(DevStatus), s));
    Arena a(workspace);
    DevStatus *st = a.take<DevStatus>(kStatusBytes / sizeof(DevStatus));
    if (n == 0) return NNQS_OK;
    return logpsi_forward(M, params, x, n, prec, out, a, st, s);
}

size_t nnqs_logpsi_backward_workspace_size(const nnqs_model *M, int64_t n, int prec) {
    if (!M || n < 0 || !prec_ok(prec)) return 0;
    return logpsi_workspace(M, n, prec, true);
}

nnqs_status nnqs_logpsi_backward(const nnqs_model *M, const float *params, const uint64_t *x, int64_t n, int prec,
                                 const double *seed, double *grad_f64, float *grad_f32, void *workspace,
                                 size_t workspace_bytes, nnqs_stream stream) {
    if (!M || n < 0 || !prec_ok(prec)) return set_error(NNQS_E_INVAL, "bad model, count or precision");
    if (!params || (!grad_f64 && !grad_f32) || (n > 0 && (!x || !seed)))
        return set_error(NNQS_E_INVAL, "null device pointer");
    NNQS_TRY(check_ws2(workspace, workspace_bytes, logpsi_workspace(M, n, prec, true)));
    cudaStream_t s = (cudaStream_t)stream;
    NNQS_CUDA_TRY(cudaMemsetAsync(workspace, 0, sizeof(DevStatus), s));
    Arena a(workspace);
    DevStatus *st = a.take<DevStatus>(kStatusBytes / sizeof(DevStatus));
    return logpsi_backward(M, params, x, n, prec, seed, grad_f64, grad_f32, a, st, s);
}

}  // extern "C"
