"""The learned part, trained on the GPU by the library's own kernels (BAS
sampling, sample-aware local energy, hand-written reverse mode, Adam) and
judged by exact FP64 quantities: the variational energy by full enumeration
against exact diagonalisation (12 qubits), and the gain over the method
without learning -- the random-init ansatz and the best single determinant --
on the 30-qubit, 14-electron workload.  Also: checkpoint/resume is
bit-identical to an uninterrupted run."""
import numpy as np
import pytest
import torch

from oracle import hamiltonian as OH
from paper_2306_16705_gb300 import binding as B
from paper_2306_16705_gb300 import inputs as I
from paper_2306_16705_gb300.vmc import VMC

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    B.lib()


def exact_energy(model, flat, S, M):
    """E(theta) = <psi|H|psi>/<psi|psi> over the whole sector (FP64 path)."""
    lp = B.logpsi(model, flat, B.to_device_bits(S), B.FP64).cpu().numpy()
    psi = np.exp(lp[:, 0] + 1j * lp[:, 1])
    return float((np.vdot(psi, M @ psi) / np.vdot(psi, psi)).real)


def test_training_n12_approaches_exact_ground_state():
    wl = I.WORKLOADS["n12"]
    h, eri = I.workload_integrals(wl)
    ham = B.build_pauli(h, eri)
    E0, st, _ = OH.ed_ground(h, eri, wl.n_alpha, wl.n_beta)
    M = OH.determinant_matrix(h, eri, st)
    S = I.sector_states(wl.n_spatial, wl.n_alpha, wl.n_beta)
    model = B.Model(wl.n_qubits, wl.n_alpha, wl.n_beta, wl.d_model, wl.n_layers, wl.n_heads)
    flat = model.pack(I.workload_params(wl, std=0.05, phase_std=0.05))
    e_init = exact_energy(model, flat, S, M)
    e_det = float(np.min(np.diag(M)))  # best single determinant
    vmc = VMC(ham, model, flat.clone(), prec=B.FP32, n_samples=100_000, max_unique=512, lr=5e-3, seed=3)
    for _ in range(400):
        vmc.step(check=False)
    e_fin = exact_energy(model, vmc.params, S, M)
    print(f"n12: E0 {E0:.6f}  best determinant {e_det:.6f}  init {e_init:.6f}  trained {e_fin:.6f}")
    assert e_fin >= E0 - 1e-9  # variational
    assert e_fin < e_det  # beats every single determinant
    # at least half of the gap closed (about 69 % after 300-800 steps here:
    # training then plateaus near -15.21 Ha against E0 = -16.52 Ha)
    assert (e_fin - E0) < 0.5 * (e_init - E0)


def test_training_n30_gains_over_no_learning():
    """30 spin orbitals, 14 electrons (d=64, 4 layers, Adam lr 1e-3): after
    training, the sampled energy lies below the random-init ansatz's and below
    the best single determinant met in any sample."""
    wl = I.WORKLOADS["n30"]
    h, eri = I.workload_integrals(wl)
    ham = B.build_pauli(h, eri)
    model = B.Model(wl.n_qubits, wl.n_alpha, wl.n_beta, wl.d_model, wl.n_layers, wl.n_heads)
    flat = model.pack(I.workload_params(wl))
    vmc = VMC(ham, model, flat.clone(), prec=B.MIXED, n_samples=8192, max_unique=8192, lr=1e-3, seed=4)
    energies = []
    best_det = np.inf
    for it in range(200):
        st = vmc.step(check=(it % 50 == 0)).cpu().numpy()
        energies.append(st[0])
        if it % 20 == 0 or it == 199:
            xs = B.from_device_bits(vmc.last_samples)
            for x in xs[:64]:
                xp, hx = ham.coupled(x, wl.n_alpha, wl.n_beta)
                diag = hx[np.all(xp == x[None, :], axis=1)]
                best_det = min(best_det, float(diag[0]))
    e_init = float(np.mean(energies[:5]))
    e_fin = float(np.mean(energies[-10:]))
    print(f"n30: init {e_init:.4f}  trained {e_fin:.4f}  best determinant seen {best_det:.4f}")
    assert e_fin < e_init - 1.0
    assert e_fin < best_det


def test_checkpoint_resume_is_bit_identical():
    wl = I.WORKLOADS["n12"]
    h, eri = I.workload_integrals(wl)
    ham = B.build_pauli(h, eri)
    model = B.Model(wl.n_qubits, wl.n_alpha, wl.n_beta, wl.d_model, wl.n_layers, wl.n_heads)
    flat = model.pack(I.workload_params(wl, std=0.05))
    for prec in (B.FP32, B.MIXED):
        a = VMC(ham, model, flat.clone(), prec=prec, n_samples=50_000, max_unique=512, lr=5e-3, seed=9)
        for _ in range(6):
            a.step(check=True)
        b = VMC(ham, model, flat.clone(), prec=prec, n_samples=50_000, max_unique=512, lr=5e-3, seed=9)
        for _ in range(3):
            b.step(check=True)
        sd = b.state_dict()
        c = VMC(ham, model, torch.zeros_like(flat), prec=prec, n_samples=50_000, max_unique=512, lr=5e-3, seed=0)
        c.load_state_dict(sd)
        for _ in range(3):
            c.step(check=True)
        assert torch.equal(a.params, c.params)
        assert torch.equal(a.m, c.m) and torch.equal(a.v, c.v)


def test_paper_recipe_adamw_warmup_and_sample_schedule():
    """The Sec. 4.1 recipe through the driver: each update is the oracle's
    AdamW step with the warm-up learning rate of that step, the sampler runs
    N_s = 10^5 in the first iterations, and a table overflow holds N_s."""
    from oracle import vmc as OV
    wl = I.WORKLOADS["n12"]
    h, eri = I.workload_integrals(wl)
    ham = B.build_pauli(h, eri)
    model = B.Model(wl.n_qubits, wl.n_alpha, wl.n_beta, wl.d_model, wl.n_layers, wl.n_heads)
    flat = model.pack(I.workload_params(wl, std=0.05, phase_std=0.05))
    vmc = VMC(ham, model, flat.clone(), prec=B.FP32, max_unique=512, seed=2, optimizer="adamw",
              weight_decay=0.01, schedule="paper", warmup=50)
    th = flat.double().cpu().numpy()
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    for step in range(1, 4):
        assert vmc.current_n_samples() == 10 ** 5
        lr = vmc.current_lr()
        assert lr == pytest.approx(OV.lr_warmup(step, wl.d_model, 50), rel=1e-15)
        vmc.step()
        assert int(vmc.last_weights.sum().item()) == 10 ** 5
        g = vmc.grad.double().cpu().numpy()
        th, m, v = OV.adamw_step(th, g, m, v, step, lr=lr, weight_decay=0.01)
        assert np.abs(vmc.params.double().cpu().numpy() - th).max() < 1e-6
    # a sample count whose unique prefixes overflow the table is divided by ten
    small = VMC(ham, model, flat.clone(), prec=B.FP32, max_unique=64, seed=2, schedule="paper")
    small.sample()
    assert small.ns_hold is not None and small.ns_hold < 10 ** 5
