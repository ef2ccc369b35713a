"""The learned part, trained on the GPU by the library's own kernels (BAS
sampling, sample-aware local energy, hand-written reverse mode, Adam) and
judged by exact FP64 quantities: the variational energy by full enumeration
against exact diagonalisation (12 qubits), and the gain over the method
without learning -- the random-init ansatz and the best single determinant --
on the 30-qubit, 14-electron workload (500 BF16X3 steps checked against the
FP64 oracle on held-out samples, beside the plain FP64 run of the same
seed).  Also: checkpoint/resume is bit-identical to an uninterrupted run."""
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


def heldout_check(ham, model, params, strings, wl, seed, n_draw=2048):
    """Held-out samples (a sampler draw with a seed training never uses):
    the GPU's BF16X3 log psi and sample-aware local energy against the FP64
    oracle (numpy forward, plain-C Alg. 2) on the same table.  Every row
    |dE_loc| <= b(x) = S(x)(e^{2 eps} - 1) + 1e-10 max(1, S(x)), eps the
    largest complex log psi error over the table and S(x) = sum |H psi'/psi|
    (Eq. Eloc: each ratio psi'/psi moves by at most a factor e^{2 eps}).
    Returns the two weighted energies, eps, and the energy bound the rows
    give, sum w b / sum w."""
    from oracle import ansatz as OA
    from oracle import vmc as OV

    xs, w = B.sample(model, params, n_draw, seed=seed, max_unique=8192, prec=B.BF16X3)
    S = B.from_device_bits(xs)
    wn = w.cpu().numpy().astype(np.uint64)
    theta = model.unpack(params, I.workload_params(wl))
    la, ph = OA.forward(theta, I.unpack_bits(S, wl.n_qubits), wl.n_alpha, wl.n_beta, wl.n_heads)
    lp_ref = np.stack([la, ph], 1)
    lp_gpu = B.logpsi(model, params, xs, B.BF16X3)
    eps = float(np.hypot(*(lp_gpu.cpu().numpy() - lp_ref).T).max())
    el_gpu = B.eloc(ham, xs, lp_gpu, wl.n_alpha, wl.n_beta).cpu().numpy()
    el_gpu = el_gpu[:, 0] + 1j * el_gpu[:, 1]
    el_ref = OH.eloc_lut(*strings, S, lp_ref, S, wl.n_alpha, wl.n_beta)
    # S(x) over the table from the oracle's rows of H
    keys = {tuple(r): i for i, r in enumerate(S.tolist())}
    bounds = np.empty(len(S))
    for i in range(len(S)):
        xp, hs = OH.coupled(*strings, S[i], wl.n_alpha, wl.n_beta)
        jj = [keys.get(tuple(v)) for v in xp.tolist()]
        sx = sum(abs(hv) * np.exp(lp_ref[j, 0] - lp_ref[i, 0]) for hv, j in zip(hs, jj) if j is not None)
        bounds[i] = sx * np.expm1(2 * eps) + 1e-10 * max(1.0, sx)
        assert abs(el_gpu[i] - el_ref[i]) <= bounds[i], (i, abs(el_gpu[i] - el_ref[i]), bounds[i])
    e_gpu, _ = OV.energy_stats(el_gpu, wn)
    e_ref, _ = OV.energy_stats(el_ref, wn)
    wf = wn.astype(np.float64)
    return float(e_gpu.real), float(e_ref.real), eps, float((wf * bounds).sum() / wf.sum())


def train_n30(ham, model, flat, prec, steps, strings=None, wl=None, check_every=0):
    vmc = VMC(ham, model, flat.clone(), prec=prec, n_samples=8192, max_unique=8192, lr=1e-3, seed=4)
    energies, best_det, checks = [], np.inf, []
    for it in range(steps):
        st = vmc.step(check=(it % 50 == 0)).cpu().numpy()
        energies.append(st[0])
        if it % 50 == 0 or it == steps - 1:
            xs = B.from_device_bits(vmc.last_samples)
            for x in xs[:64]:
                xp, hx = ham.coupled(x, model.n_alpha, model.n_beta)
                best_det = min(best_det, float(hx[np.all(xp == x[None, :], axis=1)][0]))
        if check_every and (it + 1) % check_every == 0:
            checks.append((it + 1,) + heldout_check(ham, model, vmc.params, strings, wl, seed=900_000 + it))
    return energies, best_det, checks


def test_training_n30_config5():
    """The training workload as specified: 30 spin orbitals, 14 electrons,
    d=64, 4 layers, Adam lr 1e-3, 500 steps on N_s = 8192 self-generated
    samples per step, in BF16X3 (the fast path inside the 1e-6 Ha gate on
    the benchmark workload).  Every 50 steps the current ansatz is checked on
    held-out samples against the FP64 oracle: every row's local energy within
    the bound its log psi error allows (heldout_check), and the energy within
    the weighted bound of its rows.  How many checkpoints also fall within
    1e-6 Ha is printed: the log psi error of split-BF16 operands depends on
    the parameters a trajectory visits (from 6e-6 to 1.5e-4 in 500 steps),
    so a fixed gate is not a property of the arithmetic.  The plain FP64 GPU
    run of the same seed is trained beside it.  Both runs gain over the
    method without learning (the random-init ansatz and the best single
    determinant met in any sample), and their final energies differ by a
    small fraction of that gain."""
    wl = I.WORKLOADS["n30"]
    h, eri = I.workload_integrals(wl)
    ham = B.build_pauli(h, eri)
    strings = OH.build(h, eri)
    model = B.Model(wl.n_qubits, wl.n_alpha, wl.n_beta, wl.d_model, wl.n_layers, wl.n_heads)
    flat = model.pack(I.workload_params(wl))
    steps = 500
    e3, det3, checks = train_n30(ham, model, flat, B.BF16X3, steps, strings, wl, check_every=50)
    e64, det64, _ = train_n30(ham, model, flat, B.FP64, steps)
    init3, fin3 = float(np.mean(e3[:5])), float(np.mean(e3[-10:]))
    init64, fin64 = float(np.mean(e64[:5])), float(np.mean(e64[-10:]))
    print(f"n30 BF16X3: init {init3:.5f} trained {fin3:.5f} best det {det3:.5f}; "
          f"FP64: init {init64:.5f} trained {fin64:.5f} best det {det64:.5f}; gap {abs(fin3 - fin64):.2e} Ha")
    within = 0
    for it, eg, er, eps, eb in checks:
        print(f"  step {it}: held-out energy GPU {eg:.9f} oracle {er:.9f} diff {abs(eg - er):.1e} "
              f"bound {eb:.1e} log psi err {eps:.1e}")
        assert abs(eg - er) <= eb, (it, eg, er, eb)
        within += abs(eg - er) <= 1e-6
    print(f"  {within} of {len(checks)} checkpoints within 1e-6 Ha")
    assert len(checks) == steps // 50
    for init, fin, det in ((init3, fin3, det3), (init64, fin64, det64)):
        assert fin < init - 1.0
        assert fin < det
    assert abs(fin3 - fin64) <= 0.25 * min(init3 - fin3, init64 - fin64)


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
