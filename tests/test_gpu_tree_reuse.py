"""The energy gradient from the sampler's tree (nnqs_sample with
NNQS_SAMPLE_KEEP, then nnqs_energy_grad_sampled): the decode step keeps each
tree node's layer inputs and mid residuals, and the reverse mode reads each
token row's from its node instead of running the forward again (Sec. 2.1
gradient estimator, Sec. 3.3 sampler).  Checked against the separate-forward
path on the same samples and against the FP64 oracle."""
import numpy as np
import pytest
import torch

from oracle import ansatz as OA
from oracle import hamiltonian as OH
from paper_2306_16705_gb300 import binding as B
from paper_2306_16705_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    B.lib()


@pytest.fixture(scope="module")
def n40():
    wl = I.WORKLOADS["n40"]
    h, eri = I.workload_integrals(wl)
    ham = B.build_pauli(h, eri)
    model = B.Model(wl.n_qubits, wl.n_alpha, wl.n_beta, wl.d_model, wl.n_layers, wl.n_heads)
    params = I.workload_params(wl)
    return wl, h, eri, ham, model, params, model.pack(params)


def keep_sample(model, flat, n, seed, max_unique, prec):
    nb = B.lib().nnqs_sample_workspace_size(model.handle, max_unique, prec, B.SAMPLE_KEEP)
    ws = B.workspace(nb)
    x, w = B.sample(model, flat, n, seed, max_unique, prec, ws=ws, flags=B.SAMPLE_KEEP)
    return x, w, ws


@pytest.mark.parametrize("prec", [B.MIXED, B.BF16X3])
def test_keep_draws_the_same_samples(n40, prec):
    wl, h, eri, ham, model, params, flat = n40
    x0, w0 = B.sample(model, flat, 4096, 5, 1 << 13, prec)
    x1, w1, _ = keep_sample(model, flat, 4096, 5, 1 << 13, prec)
    assert torch.equal(x0, x1) and torch.equal(w0, w1)


@pytest.mark.parametrize("prec", [B.MIXED, B.BF16X3])
def test_sampled_gradient_matches_separate_forward(n40, prec):
    """Same samples and weights: the energies agree within 1e-7 Ha (both
    paths' log psi carry the precision's operand rounding; the decode and the
    fused forward sum in different orders) and every gradient tensor within
    the BF16 reverse-mode bound of its largest entry (the reverse mode is the
    same; its inputs differ by that rounding)."""
    wl, h, eri, ham, model, params, flat = n40
    x, w, ws = keep_sample(model, flat, 4096, 7, 1 << 13, prec)
    st0, el0, g0 = B.energy_grad(ham, model, flat, x, w, prec)
    st1, el1, g1 = B.energy_grad_sampled(ham, model, flat, ws, 1 << 13, x, w, prec)
    assert abs(st0[0].item() - st1[0].item()) <= 1e-7, (st0[0].item(), st1[0].item())
    G0, G1 = model.unpack(g0, params), model.unpack(g1, params)
    tol = 1e-1 if prec == B.MIXED else 4e-2
    for k in params:
        err = np.abs(G0[k] - G1[k]).max()
        assert err <= tol * max(1e-3, np.abs(G0[k]).max()), (k, err)


def test_sampled_gradient_n40_bench_config_against_oracle(n40):
    """The benchmark's configuration through the tree path (N_s = 16,384,
    split BF16): the energy within the 1e-6 Ha gate of the FP64 oracle on the
    same samples and weights (its own log psi and Alg. 2 local energy), every
    gradient tensor within 4e-2 of its largest entry of the oracle's reverse
    mode."""
    from oracle import vmc as OV

    wl, h, eri, ham, model, params, flat = n40
    x, w, ws = keep_sample(model, flat, 16384, 1000, 1 << 15, B.BF16X3)
    stats, _, g = B.energy_grad_sampled(ham, model, flat, ws, 1 << 15, x, w, B.BF16X3)
    strings = OH.build(h, eri)
    S = B.from_device_bits(x)
    wn = w.cpu().numpy().astype(np.uint64)
    la, ph, cache = OA.forward(params, I.unpack_bits(S, wl.n_qubits), wl.n_alpha, wl.n_beta, wl.n_heads,
                               want_cache=True)
    lp_ref = np.stack([la, ph], 1)
    ref_el = OH.eloc_lut(*strings, S, lp_ref, S, wl.n_alpha, wl.n_beta)
    E_ref, _ = OV.energy_stats(ref_el, wn)
    assert abs(float(stats[0].item()) - E_ref.real) <= 1e-6, (float(stats[0].item()), E_ref.real)
    s_la, s_ph = OV.grad_seeds(ref_el, wn)
    R = OA.backward(cache, s_la, s_ph)
    G = model.unpack(g, params)
    for k in params:
        err = np.abs(G[k] - R[k]).max()
        assert err <= 4e-2 * max(1e-3, np.abs(R[k]).max()), (k, err, np.abs(R[k]).max())


def test_sampled_gradient_rejects_other_samples(n40):
    """Samples that are not the kept call's (a changed row) are reported."""
    wl, h, eri, ham, model, params, flat = n40
    x, w, ws = keep_sample(model, flat, 2048, 9, 1 << 12, B.BF16X3)
    y = x.clone()
    y[3, 0] ^= 1 << 20
    with pytest.raises(B.NNQSError) as e:
        B.energy_grad_sampled(ham, model, flat, ws, 1 << 12, y, w, B.BF16X3)
    assert e.value.status == B.E_INVAL


def test_tree_reuse_unsupported_cases():
    """FP32 arithmetic or d_model != 64: no kept tree, the calls say so."""
    wl = I.WORKLOADS["n12"]  # d_model 32
    model = B.Model(wl.n_qubits, wl.n_alpha, wl.n_beta, wl.d_model, wl.n_layers, wl.n_heads)
    assert B.lib().nnqs_energy_grad_sampled_supported(model.handle, B.BF16X3, 512) == 0
    m64 = B.Model(40, 10, 10, 64, 4, 8)
    assert B.lib().nnqs_energy_grad_sampled_supported(m64.handle, B.FP32, 512) == 0
    assert B.lib().nnqs_energy_grad_sampled_supported(m64.handle, B.BF16X3, 512) == 1
    flat = model.pack(I.workload_params(wl))
    with pytest.raises(B.NNQSError) as e:
        B.sample(model, flat, 100, 1, 512, B.BF16X3, flags=B.SAMPLE_KEEP)
    assert e.value.status == B.E_UNSUPPORTED
