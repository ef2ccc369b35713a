"""Pins of the oracle's energy statistics, gradient estimator and Adam step:
numpy's weighted average, finite differences of the exact variational energy
E(theta) of Eq. (energy3) under full enumeration, and torch.optim.Adam."""
import numpy as np
import pytest
import torch

from oracle import ansatz as OA
from oracle import hamiltonian as OH
from oracle import vmc as OV
from paper_2306_16705_gb300 import inputs as I


def test_energy_stats_match_numpy_average():
    rng = np.random.default_rng(0)
    e = rng.normal(size=100) + 1j * rng.normal(size=100)
    w = rng.integers(1, 50, size=100)
    E, var = OV.energy_stats(e, w)
    assert abs(E - np.average(e, weights=w)) < 1e-14
    assert abs(var - np.average(np.abs(e - np.average(e, weights=w)) ** 2, weights=w)) < 1e-13


def test_gradient_estimator_equals_fd_of_exact_energy():
    """With weights = p_theta over the whole sector and E_loc exact, the
    estimator of Sec. 2.1 is the exact gradient of E(theta) (Eq. energy3)."""
    wl = I.WORKLOADS["n12"]
    h, eri = I.workload_integrals(wl)
    xy, yz, coef = OH.build(h, eri)
    lut = I.sector_states(wl.n_spatial, wl.n_alpha, wl.n_beta)
    bits = I.unpack_bits(lut, wl.n_qubits)
    M = OH.determinant_matrix(h, eri, lut[:, 0].astype(np.int64))
    params = I.ansatz_params(wl.n_qubits, 16, 1, 4, std=0.3, bias_std=0.1, phase_std=0.3)
    nh = 2

    def energy(pp):
        la, ph = OA.forward(pp, bits, wl.n_alpha, wl.n_beta, nh)
        psi = np.exp(la + 1j * ph)
        return (np.vdot(psi, M @ psi) / np.vdot(psi, psi)).real

    la, ph = OA.forward(params, bits, wl.n_alpha, wl.n_beta, nh)
    el = OH.eloc_lut(xy, yz, coef, lut, np.stack([la, ph], 1), lut, wl.n_alpha, wl.n_beta)
    p = np.exp(2 * la)
    G = OV.energy_grad(params, bits, el, p, wl.n_alpha, wl.n_beta, nh)
    rng = np.random.default_rng(2)
    for k in ["l0.attn.wqkv", "head.w", "phase.w2", "phase.b1", "tok_emb", "l0.ffn.w2"]:
        for idx in rng.choice(params[k].size, size=3, replace=False):
            pp = {kk: vv.astype(np.float64).copy() for kk, vv in params.items()}
            step = 1e-6  # small enough to stay off the ReLU kinks of the phase MLP
            pp[k].reshape(-1)[idx] += step
            ep = energy(pp)
            pp[k].reshape(-1)[idx] -= 2 * step
            em = energy(pp)
            fd = (ep - em) / (2 * step)
            assert abs(fd - G[k].reshape(-1)[idx]) < 1e-8 + 1e-6 * abs(fd), (k, idx)


def test_adam_matches_torch():
    rng = np.random.default_rng(3)
    theta = rng.normal(size=50)
    t = torch.tensor(theta.copy(), requires_grad=True)
    opt = torch.optim.Adam([t], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    m = np.zeros(50)
    v = np.zeros(50)
    for step in range(1, 6):
        g = rng.normal(size=50)
        t.grad = torch.tensor(g)
        opt.step()
        theta, m, v = OV.adam_step(theta, g, m, v, step)
    assert np.abs(theta - t.detach().numpy()).max() < 1e-14


def test_adamw_matches_torch():
    """Decoupled weight decay (Sec. 4.1 trains with AdamW) against the library
    routine torch.optim.AdamW; a sign or order slip in the decay term fails."""
    rng = np.random.default_rng(4)
    theta = rng.normal(size=50)
    t = torch.tensor(theta.copy(), requires_grad=True)
    opt = torch.optim.AdamW([t], lr=3e-3, betas=(0.9, 0.999), eps=1e-8, weight_decay=0.05)
    m = np.zeros(50)
    v = np.zeros(50)
    for step in range(1, 6):
        g = rng.normal(size=50)
        t.grad = torch.tensor(g)
        opt.step()
        theta, m, v = OV.adamw_step(theta, g, m, v, step, lr=3e-3, weight_decay=0.05)
    assert np.abs(theta - t.detach().numpy()).max() < 1e-14
    # weight_decay = 0 is plain Adam
    th0 = rng.normal(size=8)
    g = rng.normal(size=8)
    a = OV.adamw_step(th0, g, np.zeros(8), np.zeros(8), 1, weight_decay=0.0)
    b = OV.adam_step(th0, g, np.zeros(8), np.zeros(8), 1)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))


def test_lr_warmup_schedule():
    """Sec. 4.1: d^-1/2 min(i^-1/2, i S_w^-3/2): linear rise to the peak
    (d S_w)^-1/2 at i = S_w, then i^-1/2 decay; values worked by hand for
    d = 64, S_w = 4000."""
    d, sw = 64, 4000
    assert OV.lr_warmup(1, d, sw) == pytest.approx(0.125 * 4000 ** -1.5, rel=1e-15)
    assert OV.lr_warmup(1, d, sw) == pytest.approx(4.941058844013093e-07, rel=1e-12)
    assert OV.lr_warmup(sw, d, sw) == pytest.approx(1 / np.sqrt(256000.0), rel=1e-15)
    assert OV.lr_warmup(sw, d, sw) == pytest.approx(0.0019764235376052372, rel=1e-12)
    for i in (2, 17, 1000, 3999):
        assert OV.lr_warmup(i, d, sw) == pytest.approx(i * OV.lr_warmup(1, d, sw), rel=1e-13)
    for i in (4001, 10 ** 4, 10 ** 5):
        assert OV.lr_warmup(i, d, sw) == pytest.approx(OV.lr_warmup(sw, d, sw) * np.sqrt(sw / i), rel=1e-13)
    lrs = [OV.lr_warmup(i, d, sw) for i in range(1, 3 * sw)]
    assert int(np.argmax(lrs)) + 1 == sw
