"""Parity at the workloads' full sizes, on outputs the oracle computes one by
one: the 76-qubit (N_u = 65,536) and 120-qubit (N_u = 131,072, 19.2 M Pauli
strings) sample-aware local energy against the Slater-Condon path of the
oracle (matrix elements from the integrals, no Pauli strings), the
120-qubit ansatz on sampled rows against the FP64 oracle forward, and one
complete 120-qubit VMC step (sampling, E_loc, reverse mode with activation
recomputation over several chunks, Zipf-weighted statistics)."""
import numpy as np
import pytest
import torch

from oracle import ansatz as OA
from oracle import hamiltonian as OH
from paper_2306_16705_gb300 import binding as B
from paper_2306_16705_gb300 import inputs as I

pytestmark = pytest.mark.gpu

N_U = {"n76": 65536, "n120": 131072}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    B.lib()


@pytest.fixture(scope="module", params=["n76", "n120"])
def big(request):
    wl = I.WORKLOADS[request.param]
    h, eri = I.workload_integrals(wl)
    ham = B.build_pauli(h, eri)
    S = I.clustered_sector_samples(wl.n_spatial, wl.n_alpha, wl.n_beta, N_U[request.param], seed=wl.seed,
                                   n_centers=16)
    lp = I.random_logpsi(len(S), seed=wl.seed + 1, amp_std=0.5)
    return wl, h, eri, ham, S, lp


@pytest.mark.parametrize("flags", [B.SWEEP_GROUPS, B.SWEEP_PAIRS])
def test_eloc_full_size_sampled_rows(big, flags):
    """Three 8-row windows (first, middle, ragged last rows) of E_loc over the
    full table; FP64 within 1e-10 of sum |H psi'/psi| per row."""
    wl, h, eri, ham, S, lp = big
    n = len(S)
    assert ham.info()["n_terms"] == {"n76": 3076443, "n120": 19233001}[wl.name]
    xs = B.to_device_bits(S)
    lpd = torch.from_numpy(lp).cuda()
    for rb in (0, n // 2 - 3, n - 8):
        o = B.eloc(ham, xs, lpd, wl.n_alpha, wl.n_beta, flags=flags, row_begin=rb, n_rows=8).cpu().numpy()
        got = o[:, 0] + 1j * o[:, 1]
        ref, sc = OH.eloc_slater_condon(h, eri, S, lp, np.arange(rb, rb + 8))
        assert np.all(np.abs(got - ref) <= 1e-10 * sc), (rb, np.abs(got - ref).max())


def test_logpsi_full_size_n120_sampled_rows():
    """log psi of all 131,072 samples (d=128, 6 layers, 60 tokens) on the GPU;
    eight rows checked against the FP64 oracle: FP32 within 2e-4, split BF16
    within 1e-3 of the scale."""
    wl = I.WORKLOADS["n120"]
    params = I.ansatz_params(wl.n_qubits, wl.d_model, wl.n_layers, 5, std=0.05, bias_std=0.05, phase_std=0.05)
    m = B.Model(wl.n_qubits, wl.n_alpha, wl.n_beta, wl.d_model, wl.n_layers, wl.n_heads)
    flat = m.pack(params)
    S = I.random_sector_samples(wl.n_spatial, wl.n_alpha, wl.n_beta, N_U["n120"], seed=6)
    xs = B.to_device_bits(S)
    rows = np.array([0, 1, 4095, 65536, 99999, 131069, 131070, 131071])
    la, ph = OA.forward(params, I.unpack_bits(S[rows], wl.n_qubits), wl.n_alpha, wl.n_beta, wl.n_heads)
    ref = np.stack([la, ph], 1)
    scale = max(1.0, np.abs(ref).max())
    for prec, tol in ((B.FP32, 2e-4), (B.BF16X3, 1e-3)):
        got = B.logpsi(m, flat, xs, prec).cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.abs(got[rows] - ref).max() <= tol * scale, prec


def test_vmc_step_full_size_n120():
    """Sampling (N_s = 131,072 from the random-init ansatz), Zipf(1.2)
    weights on the unique samples, E_loc over the 19.2 M strings, statistics
    and the reverse mode over several recomputed activation chunks: split
    BF16 and FP32 energies agree within 1e-6 Ha and their gradients within
    2e-2 of the norm."""
    wl = I.WORKLOADS["n120"]
    h, eri = I.workload_integrals(wl)
    ham = B.build_pauli(h, eri)
    m = B.Model(wl.n_qubits, wl.n_alpha, wl.n_beta, wl.d_model, wl.n_layers, wl.n_heads)
    flat = m.pack(I.workload_params(wl))
    xs, w = B.sample(m, flat, N_U["n120"], seed=7, max_unique=1 << 18, prec=B.BF16X3)
    assert int(w.sum().item()) == N_U["n120"]
    bits = B.from_device_bits(xs)
    assert np.all(np.diff([OH.words_to_int(r) for r in bits[:2000]]) > 0)  # sorted, unique
    z = torch.from_numpy(I.zipf_counts(xs.shape[0], 1.2, seed=3).astype(np.int64)).cuda()
    s3, _, g3 = B.energy_grad(ham, m, flat, xs, z, B.BF16X3)
    s32, _, g32 = B.energy_grad(ham, m, flat, xs, z, B.FP32)
    e3, e32 = float(s3[0].item()), float(s32[0].item())
    assert np.isfinite(e3) and abs(e3 - e32) <= 1e-6, (e3, e32)
    g3, g32 = g3.double().cpu().numpy(), g32.double().cpu().numpy()
    assert np.all(np.isfinite(g3))
    assert np.linalg.norm(g3 - g32) <= 2e-2 * np.linalg.norm(g32)
