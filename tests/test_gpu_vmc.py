"""GPU parity of the rest of the VMC step against the oracle: exact-mode
local energy (every coupled x', Eq. Eloc), the composite energy/gradient call
(Sec. 2.1 estimator), finite differences of its surrogate, the batch
autoregressive sampler (Sec. 3.1 BAS, mask of Sec. 3.3) and Adam."""
import numpy as np
import pytest
import torch

from oracle import ansatz as OA
from oracle import hamiltonian as OH
from oracle import vmc as OV
from paper_2306_16705_gb300 import binding as B
from paper_2306_16705_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    B.lib()


def model_for(wl, seed=7, std=0.3, hidden=512):
    params = I.ansatz_params(wl.n_qubits, wl.d_model, wl.n_layers, seed, std=std, bias_std=0.1,
                             phase_std=0.1)
    m = B.Model(wl.n_qubits, wl.n_alpha, wl.n_beta, wl.d_model, wl.n_layers, wl.n_heads, hidden)
    return m, params, m.pack(params)


def c(a):
    a = a.cpu().numpy()
    return a[:, 0] + 1j * a[:, 1]


@pytest.fixture(scope="module")
def n12():
    wl = I.WORKLOADS["n12"]
    h, eri = I.workload_integrals(wl)
    return wl, B.build_pauli(h, eri), OH.build(h, eri), h, eri


def test_exact_mode_n12(n12):
    wl, ham, strings, h, eri = n12
    m, params, flat = model_for(wl)
    S = I.sector_states(wl.n_spatial, wl.n_alpha, wl.n_beta)
    rows = S[::7].copy()

    def fn(packed):
        return OA.forward(params, I.unpack_bits(packed, wl.n_qubits), wl.n_alpha, wl.n_beta, wl.n_heads)

    ref = OH.eloc_exact(*strings, rows, wl.n_alpha, wl.n_beta, fn)
    got = c(B.eloc(ham, B.to_device_bits(rows), None, wl.n_alpha, wl.n_beta, mode=B.EXACT, model=m,
                   params=flat, prec=B.FP64))
    assert np.abs(got - ref).max() <= 1e-10 * max(1.0, np.abs(ref).max())
    # exact over the whole sector == sample-aware with S = whole sector
    la, ph = fn(S)
    sa = c(B.eloc(ham, B.to_device_bits(S), torch.from_numpy(np.stack([la, ph], 1)).cuda(),
                  wl.n_alpha, wl.n_beta))
    ex = c(B.eloc(ham, B.to_device_bits(S), None, wl.n_alpha, wl.n_beta, mode=B.EXACT, model=m,
                  params=flat, prec=B.FP64))
    assert np.abs(sa - ex).max() <= 1e-10 * max(1.0, np.abs(ex).max())


def test_exact_mode_n40_two_rows():
    wl = I.WORKLOADS["n40"]
    h, eri = I.workload_integrals(wl)
    ham = B.build_pauli(h, eri)
    strings = OH.build(h, eri)
    m, params, flat = model_for(wl, std=0.2)
    rows = I.random_sector_samples(wl.n_spatial, wl.n_alpha, wl.n_beta, 2, seed=12)

    def fn(packed):
        return OA.forward(params, I.unpack_bits(packed, wl.n_qubits), wl.n_alpha, wl.n_beta, wl.n_heads)

    ref = OH.eloc_exact(*strings, rows, wl.n_alpha, wl.n_beta, fn)
    got = c(B.eloc(ham, B.to_device_bits(rows), None, wl.n_alpha, wl.n_beta, mode=B.EXACT, model=m,
                   params=flat, prec=B.FP64))
    assert np.abs(got - ref).max() <= 1e-10 * max(1.0, np.abs(ref).max())


def test_energy_grad_matches_oracle(n12):
    wl, ham, strings, h, eri = n12
    m, params, flat = model_for(wl, seed=8)
    S = I.sector_states(wl.n_spatial, wl.n_alpha, wl.n_beta)
    w = I.uniform_counts(len(S), 1024, seed=0)
    keep = w > 0
    S, w = S[keep], w[keep]
    stats, el, g = B.energy_grad(ham, m, flat, B.to_device_bits(S),
                                 torch.from_numpy(w.view(np.int64)).cuda(), B.FP64)
    bits = I.unpack_bits(S, wl.n_qubits)
    la, ph = OA.forward(params, bits, wl.n_alpha, wl.n_beta, wl.n_heads)
    ref_el = OH.eloc_lut(*strings, S, np.stack([la, ph], 1), S, wl.n_alpha, wl.n_beta)
    assert np.abs(c(el) - ref_el).max() <= 1e-10 * max(1.0, np.abs(ref_el).max())
    E, var = OV.energy_stats(ref_el, w)
    st = stats.cpu().numpy()
    assert abs(st[0] - E.real) < 1e-10 and abs(st[1] - E.imag) < 1e-10
    assert abs(st[2] - var) < 1e-9 * max(1, var) and st[3] == w.sum()
    G = m.unpack(g, params)
    R = OV.energy_grad(params, bits, ref_el, w, wl.n_alpha, wl.n_beta, wl.n_heads)
    for k in params:
        assert np.abs(G[k] - R[k]).max() <= 1e-8 * max(1e-3, np.abs(R[k]).max()), k


def test_energy_grad_finite_differences_n76():
    """76 qubits (two words), d=64, 4 layers: the FP64 gradient against central
    differences (h = 1e-4) of the surrogate 2 sum w [Re(E_loc-E) log|psi| +
    Im(E_loc-E) phase] / sum w with E_loc, E frozen, on 16 random parameters."""
    wl = I.WORKLOADS["n76"]
    h, eri = I.workload_integrals(wl)
    ham = B.build_pauli(h, eri)
    m, params, flat = model_for(wl, seed=21, std=0.1)
    S = I.clustered_sector_samples(wl.n_spatial, wl.n_alpha, wl.n_beta, 256, seed=5, n_centers=4)
    w = np.random.default_rng(1).integers(1, 100, size=len(S)).astype(np.uint64)
    xs = B.to_device_bits(S)
    wt = torch.from_numpy(w.view(np.int64)).cuda()
    stats, el, g = B.energy_grad(ham, m, flat, xs, wt, B.FP64)
    st = stats.cpu().numpy()
    e = c(el)
    seed = np.stack([2 * w * (e.real - st[0]) / st[3], 2 * w * (e.imag - st[1]) / st[3]], 1)

    def surrogate(fl):
        lp = B.logpsi(m, fl, xs, B.FP64).cpu().numpy()
        return float((seed[:, 0] * lp[:, 0]).sum() + (seed[:, 1] * lp[:, 1]).sum())

    g = g.cpu().numpy()
    rng = np.random.default_rng(3)
    idx = rng.choice(m.n_params, size=16, replace=False)
    for k in idx:
        fp = flat.clone()
        fm = flat.clone()
        fp[k] += 1e-4
        fm[k] -= 1e-4
        step = float(fp[k].item()) - float(fm[k].item())  # exact FP32 step
        fd = (surrogate(fp) - surrogate(fm)) / step
        assert abs(fd - g[k]) <= 1e-5 * max(1.0, abs(fd)) + 1e-7, (k, fd, g[k])


def test_sampler_statistics_n12():
    """Sum of counts = N_s, samples unique, sorted and in the sector, and a
    chi-square test of the counts against the exact |psi|^2."""
    wl = I.WORKLOADS["n12"]
    m, params, flat = model_for(wl, seed=9, std=0.5)
    S = I.sector_states(wl.n_spatial, wl.n_alpha, wl.n_beta)
    p = OV.exact_distribution(params, I.unpack_bits(S, wl.n_qubits), wl.n_alpha, wl.n_beta,
                              wl.n_heads)
    for prec in (B.FP64, B.FP32):
        Ns = 1_000_000
        xs, ws = B.sample(m, flat, Ns, seed=123, max_unique=4096, prec=prec)
        x = B.from_device_bits(xs)
        wc = ws.cpu().numpy().astype(np.uint64)
        assert wc.sum() == Ns and np.all(wc > 0)
        assert np.array_equal(I.sort_keys(x), x)
        assert len({int(v) for v in x[:, 0]}) == len(x)
        pos = np.searchsorted(S[:, 0], x[:, 0])
        assert np.all(S[pos, 0] == x[:, 0])  # every sample is a sector state
        counts = np.zeros(len(S))
        counts[pos] = wc
        expct = Ns * p
        big = expct > 20
        chi2 = (((counts - expct) ** 2)[big] / expct[big]).sum()
        dof = big.sum() - 1
        # 5-sigma bound of the chi-square distribution
        assert chi2 < dof + 5 * np.sqrt(2 * dof), (chi2, dof)


def test_sampler_large_counts_and_determinism():
    """N_s = 10^12 exercises the large-mean binomial; frequencies agree with
    |psi|^2 within 6 standard deviations; the same seed repeats exactly."""
    wl = I.WORKLOADS["n12"]
    m, params, flat = model_for(wl, seed=10, std=0.5)
    S = I.sector_states(wl.n_spatial, wl.n_alpha, wl.n_beta)
    p = OV.exact_distribution(params, I.unpack_bits(S, wl.n_qubits), wl.n_alpha, wl.n_beta,
                              wl.n_heads)
    Ns = 10 ** 12
    xs, ws = B.sample(m, flat, Ns, seed=7, max_unique=4096, prec=B.FP64)
    x = B.from_device_bits(xs)
    wc = ws.cpu().numpy().astype(np.uint64)
    assert int(wc.sum()) == Ns
    pos = np.searchsorted(S[:, 0], x[:, 0])
    counts = np.zeros(len(S))
    counts[pos] = wc.astype(np.float64)
    sd = np.sqrt(Ns * p * (1 - p))
    ok = p > 1e-9
    assert np.all(np.abs(counts - Ns * p)[ok] <= 6 * sd[ok] + 1)
    xs2, ws2 = B.sample(m, flat, Ns, seed=7, max_unique=4096, prec=B.FP64)
    assert torch.equal(xs, xs2) and torch.equal(ws, ws2)
    xs3, ws3 = B.sample(m, flat, Ns, seed=8, max_unique=4096, prec=B.FP64)
    assert not torch.equal(ws, ws3)
    with pytest.raises(B.NNQSError) as e:
        B.sample(m, flat, Ns, seed=7, max_unique=100, prec=B.FP64)
    assert e.value.status == B.E_TABLE_FULL


def test_adam_matches_oracle():
    rng = np.random.default_rng(0)
    n = 100003
    theta = rng.normal(size=n).astype(np.float32)
    pt = torch.from_numpy(theta.copy()).cuda()
    m = torch.zeros(n, device="cuda")
    v = torch.zeros(n, device="cuda")
    th, mm, vv = theta.astype(np.float64), np.zeros(n), np.zeros(n)
    for step in range(1, 4):
        g = rng.normal(size=n).astype(np.float32)
        B.adam_step(pt, torch.from_numpy(g).cuda(), m, v, step, lr=1e-3)
        th, mm, vv = OV.adam_step(th, g.astype(np.float64), mm, vv, step)
    assert np.abs(pt.cpu().numpy() - th).max() < 1e-6


@pytest.mark.parametrize("prec", [B.FP64, B.FP32, B.MIXED, B.BF16X3])
@pytest.mark.parametrize("wl_name,ns", [("n12", 100_000), ("n40", 4096)])
def test_sampler_kv_cache_equals_recompute(wl_name, ns, prec):
    """The key/value-cached sampler (one new token per prefix per step) draws
    exactly the samples of the full recomputation with the same seed."""
    wl = I.WORKLOADS[wl_name]
    m, params, flat = model_for(wl, seed=12, std=0.3)
    xa, wa = B.sample(m, flat, ns, seed=5, max_unique=8192, prec=prec)
    xb, wb = B.sample(m, flat, ns, seed=5, max_unique=8192, prec=prec, flags=B.SAMPLE_RECOMPUTE)
    assert torch.equal(xa, xb) and torch.equal(wa, wb)
    assert int(wa.sum().item()) == ns


def test_energy_grad_mixed_and_fp32_against_fp64(n12):
    """Energies of the three arithmetic paths on the same samples and
    parameters.  With these deliberately large weights (std 0.3) FP32 lands
    a few 1e-6 Ha from FP64 and BF16 a few 1e-3; the benchmark reports the
    differences on its own workload.  Bounded loosely here: 1e-5 and 1e-1
    relative."""
    wl, ham, strings, h, eri = n12
    m, params, flat = model_for(wl, seed=8)
    S = I.sector_states(wl.n_spatial, wl.n_alpha, wl.n_beta)
    w = torch.from_numpy(np.ones(len(S), dtype=np.int64)).cuda()
    xs = B.to_device_bits(S)
    precs = (B.FP64, B.FP32, B.MIXED, B.BF16X3)
    e = {p: B.energy_grad(ham, m, flat, xs, w, p)[0].cpu().numpy()[0] for p in precs}
    assert abs(e[B.FP32] - e[B.FP64]) < 1e-5 * abs(e[B.FP64])
    assert abs(e[B.MIXED] - e[B.FP64]) < 1e-1 * abs(e[B.FP64])
    assert abs(e[B.BF16X3] - e[B.FP64]) < 1e-4 * abs(e[B.FP64])
    assert abs(e[B.BF16X3] - e[B.FP64]) < 0.05 * abs(e[B.MIXED] - e[B.FP64])


@pytest.mark.parametrize("prec", [B.FP32, B.BF16X3])
def test_energy_gate_n40_against_plain_fp64(prec):
    """The 40-qubit, 20-electron step at full size (N_s = 16384 samples drawn
    by the sampler from the random-init ansatz): the energy of the fast
    arithmetic path and of the plain FP64 path on the same samples and
    parameters differ by at most 1e-6 Ha, and the fused single-chunk
    gradient of the fast path stays within 2e-2 of the FP64 gradient's norm."""
    wl = I.WORKLOADS["n40"]
    h, eri = I.workload_integrals(wl)
    ham = B.build_pauli(h, eri)
    m = B.Model(wl.n_qubits, wl.n_alpha, wl.n_beta, wl.d_model, wl.n_layers, wl.n_heads)
    flat = m.pack(I.workload_params(wl))
    xs, w = B.sample(m, flat, 16384, seed=21, max_unique=1 << 15, prec=prec)
    st64, _, g64 = B.energy_grad(ham, m, flat, xs, w, B.FP64)
    stp, _, gp = B.energy_grad(ham, m, flat, xs, w, prec)
    e64, ep = float(st64[0].item()), float(stp[0].item())
    assert abs(ep - e64) <= 1e-6, (ep, e64)
    g64, gp = g64.double().cpu().numpy(), gp.double().cpu().numpy()
    assert np.linalg.norm(gp - g64) <= 2e-2 * np.linalg.norm(g64)


def test_adamw_matches_oracle():
    rng = np.random.default_rng(1)
    n = 100003
    theta = rng.normal(size=n).astype(np.float32)
    pt = torch.from_numpy(theta.copy()).cuda()
    m = torch.zeros(n, device="cuda")
    v = torch.zeros(n, device="cuda")
    th, mm, vv = theta.astype(np.float64), np.zeros(n), np.zeros(n)
    for step in range(1, 4):
        g = rng.normal(size=n).astype(np.float32)
        B.adamw_step(pt, torch.from_numpy(g).cuda(), m, v, step, lr=3e-3, weight_decay=0.05)
        th, mm, vv = OV.adamw_step(th, g.astype(np.float64), mm, vv, step, lr=3e-3, weight_decay=0.05)
    assert np.abs(pt.cpu().numpy() - th).max() < 1e-6
    with pytest.raises(B.NNQSError):
        B.adamw_step(pt, pt, m, v, 1, lr=1.0, weight_decay=1.0)


def test_energy_function_autograd(n12):
    """vmc.EnergyFunction, the torch.autograd.Function over nnqs_energy_grad:
    its forward returns Re E and .backward() leaves in params.grad the
    estimator 2 Re sum w (E_loc - E) d ln psi* / sum w (Sec. 2.1).  Checked
    against the oracle gradient (FP32 storage of an FP64 accumulation:
    2^-24 relative per entry plus 1e-8 of the tensor's scale) and against
    central differences (h = 1e-4) of the surrogate with E_loc and E frozen
    on 8 random parameters; a torch.optim.Adam step consumes the gradient."""
    from paper_2306_16705_gb300.vmc import EnergyFunction

    wl, ham, strings, h, eri = n12
    m, params, flat = model_for(wl, seed=18)
    S = I.sector_states(wl.n_spatial, wl.n_alpha, wl.n_beta)
    w = I.uniform_counts(len(S), 1024, seed=3)
    keep = w > 0
    S, w = S[keep], w[keep]
    xs = B.to_device_bits(S)
    wt = torch.from_numpy(w.view(np.int64)).cuda()
    p = flat.clone().requires_grad_(True)
    E = EnergyFunction.apply(p, ham, m, xs, wt, B.FP64)
    E.backward()
    assert p.grad is not None and p.grad.dtype == torch.float32
    bits = I.unpack_bits(S, wl.n_qubits)
    la, ph = OA.forward(params, bits, wl.n_alpha, wl.n_beta, wl.n_heads)
    ref_el = OH.eloc_lut(*strings, S, np.stack([la, ph], 1), S, wl.n_alpha, wl.n_beta)
    E_ref, _ = OV.energy_stats(ref_el, w)
    assert abs(E.item() - E_ref.real) <= 1e-6 * max(1.0, abs(E_ref.real))  # FP32 output
    G = m.unpack(p.grad, params)
    R = OV.energy_grad(params, bits, ref_el, w, wl.n_alpha, wl.n_beta, wl.n_heads)
    for k in params:
        scale = np.abs(R[k]).max()
        assert np.all(np.abs(G[k] - R[k]) <= 2.0 ** -24 * np.abs(R[k]) + 1e-8 * max(1e-3, scale)), k
    # central differences of the surrogate, E_loc and E frozen at the forward
    el = ref_el
    seed_la = 2 * w * (el.real - E_ref.real) / w.sum()
    seed_ph = 2 * w * (el.imag - E_ref.imag) / w.sum()

    def surrogate(fl):
        lp = B.logpsi(m, fl, xs, B.FP64).cpu().numpy()
        return float((seed_la * lp[:, 0]).sum() + (seed_ph * lp[:, 1]).sum())

    g = p.grad.detach().cpu().numpy()
    rng = np.random.default_rng(4)
    # transformer parameters only: a ReLU of the phase MLP can change sign
    # within +-h and break the central difference
    n_tf = m.offset("phase.w1")[0]
    for k in rng.choice(n_tf, size=8, replace=False):
        fp, fm = flat.clone(), flat.clone()
        fp[k] += 1e-4
        fm[k] -= 1e-4
        step = float(fp[k].item()) - float(fm[k].item())
        fd = (surrogate(fp) - surrogate(fm)) / step
        assert abs(fd - g[k]) <= 1e-5 * max(1.0, abs(fd)) + 1e-7, (k, fd, g[k])
    # torch.optim consumes the gradient: Adam's first step moves every
    # parameter whose gradient is well above eps by lr
    opt = torch.optim.Adam([p], lr=1e-3)
    before = p.detach().clone()
    opt.step()
    moved = (p.detach() - before).abs()
    big = p.grad.abs() > 1e-5
    assert big.sum() > 1000
    assert torch.allclose(moved[big], torch.full_like(moved[big], 1e-3), rtol=1e-2)


def test_replica_samples_differ():
    """The first sampler seeds of bench replicas 0 and 1 draw different
    sample sets from the same ansatz."""
    import bench
    from paper_2306_16705_gb300.vmc import sample_seed

    wl = I.WORKLOADS["n12"]
    m, params, flat = model_for(wl, seed=9, std=0.5)
    draws = [B.sample(m, flat, 4096, seed=sample_seed(bench.replica_seed(r), 0), max_unique=4096, prec=B.FP64)
             for r in (0, 1)]
    (x0, w0), (x1, w1) = draws
    assert int(w0.sum().item()) == int(w1.sum().item()) == 4096
    assert not (x0.shape == x1.shape and torch.equal(x0, x1) and torch.equal(w0, w1))


def test_sampler_device_counts_table_full_n40():
    """The cached sampler with the fused decode layer (40 qubits, split BF16)
    keeps the level sizes on the device and synchronises once: a table that
    overflows still reports NNQS_E_TABLE_FULL, and a sufficient one gives
    the same draws as the recomputation."""
    wl = I.WORKLOADS["n40"]
    m, params, flat = model_for(wl, seed=31, std=0.3)
    with pytest.raises(B.NNQSError) as e:
        B.sample(m, flat, 20000, seed=3, max_unique=64, prec=B.BF16X3)
    assert e.value.status == B.E_TABLE_FULL
    xa, wa = B.sample(m, flat, 20000, seed=3, max_unique=32768, prec=B.BF16X3)
    xb, wb = B.sample(m, flat, 20000, seed=3, max_unique=32768, prec=B.BF16X3, flags=B.SAMPLE_RECOMPUTE)
    assert torch.equal(xa, xb) and torch.equal(wa, wb)
    assert int(wa.sum().item()) == 20000


def test_sampler_graph_replays_n40():
    """Repeated calls with the same model, parameters and workspace replay the
    device-count walk as a CUDA graph (captured on the second call): the
    draws of every call equal the direct walk's, the seed and N_s of each
    call are honoured, and parameter updates between calls are seen."""
    wl = I.WORKLOADS["n40"]
    m, params, flat = model_for(wl, seed=32, std=0.3)
    nb = B.lib().nnqs_sample_workspace_size(m.handle, 1 << 15, B.BF16X3, 0)
    ws = B.workspace(nb)
    ref = {sd: B.sample(m, flat, 12000, seed=sd, max_unique=1 << 15, prec=B.BF16X3, flags=B.SAMPLE_RECOMPUTE)
           for sd in (11, 12)}
    for k in range(4):  # direct, capture + launch, replay, replay
        sd = 11 if k % 2 == 0 else 12
        x, w = B.sample(m, flat, 12000, seed=sd, max_unique=1 << 15, prec=B.BF16X3, ws=ws)
        assert torch.equal(x, ref[sd][0]) and torch.equal(w, ref[sd][1]), k
    x, w = B.sample(m, flat, 5000, seed=11, max_unique=1 << 15, prec=B.BF16X3, ws=ws)
    assert int(w.sum().item()) == 5000
    flat.mul_(1.5)  # new parameter values at the same address
    x2, w2 = B.sample(m, flat, 12000, seed=11, max_unique=1 << 15, prec=B.BF16X3, ws=ws)
    xr, wr = B.sample(m, flat, 12000, seed=11, max_unique=1 << 15, prec=B.BF16X3, flags=B.SAMPLE_RECOMPUTE)
    assert torch.equal(x2, xr) and torch.equal(w2, wr)
