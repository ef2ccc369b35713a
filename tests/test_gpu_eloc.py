"""GPU parity of the sample-aware local energy (Eq. Eloc restricted to S,
Sec. 3.4 (4), Alg. 2) and the energy statistics against the FP64 oracle,
through the C ABI.

Tolerance (FP64 path): |E_gpu - E_oracle| <= 1e-10 * max(1, sum_x' |H_xx'
psi(x')/psi(x)|) per row -- relative to the sum of absolute contributions so
that cancellation inside E_loc does not make the bound meaningless."""
import numpy as np
import pytest
import torch

from oracle import hamiltonian as OH
from oracle import vmc as OV
from paper_2306_16705_gb300 import binding as B
from paper_2306_16705_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    B.lib()


def abs_scale(strings, lut, lp, rows, na, nb):
    """sum_x' |H_xx' psi(x')/psi(x)| over x' in the table, per row."""
    xy, yz, coef = strings
    keys = {tuple(int(v) for v in r): i for i, r in enumerate(lut)}
    out = []
    for x in rows:
        xs, hs = OH.coupled(xy, yz, coef, x, na, nb)
        i = keys[tuple(int(v) for v in x)]
        s = 0.0
        for xr, hv in zip(xs, hs):
            j = keys.get(tuple(int(v) for v in xr))
            if j is not None:
                s += abs(hv) * np.exp(lp[j, 0] - lp[i, 0])
        out.append(max(1.0, s))
    return np.array(out)


def run_gpu(ham, lut, lp, na, nb, flags, row_begin=0, n_rows=None):
    out = B.eloc(ham, B.to_device_bits(lut), torch.from_numpy(lp).cuda(), na, nb, flags=flags,
                 row_begin=row_begin, n_rows=n_rows)
    o = out.cpu().numpy()
    return o[:, 0] + 1j * o[:, 1]


@pytest.fixture(scope="module")
def n12():
    wl = I.WORKLOADS["n12"]
    h, eri = I.workload_integrals(wl)
    return wl, h, eri, B.build_pauli(h, eri), OH.build(h, eri)


@pytest.mark.parametrize("flags", [B.SWEEP_GROUPS, B.SWEEP_PAIRS, B.SWEEP_AUTO])
def test_ed_invariant_on_gpu(n12, flags):
    wl, h, eri, ham, strings = n12
    E0, st, vec = OH.ed_ground(h, eri, wl.n_alpha, wl.n_beta)
    lut = I.sector_states(wl.n_spatial, wl.n_alpha, wl.n_beta)
    lp = np.stack([np.log(np.abs(vec)), np.where(vec < 0, np.pi, 0.0)], axis=1)
    got = run_gpu(ham, lut, lp, wl.n_alpha, wl.n_beta, flags)
    ref = OH.eloc_lut(*strings, lut, lp, lut, wl.n_alpha, wl.n_beta)
    M = OH.determinant_matrix(h, eri, st)
    scale = np.maximum(1.0, (np.abs(M) @ np.abs(vec)) / np.abs(vec))
    assert np.all(np.abs(got - ref) <= TOL * scale)
    assert np.all(np.abs(got - E0) <= TOL * scale)


@pytest.mark.parametrize("flags", [B.SWEEP_GROUPS, B.SWEEP_PAIRS])
def test_n12_random_table_and_subsets(n12, flags):
    wl, h, eri, ham, strings = n12
    lut = I.sector_states(wl.n_spatial, wl.n_alpha, wl.n_beta)
    # shuffle the table: the library must not rely on sorted input
    perm = np.random.default_rng(1).permutation(len(lut))
    lut = lut[perm]
    lp = I.random_logpsi(len(lut), seed=2, amp_std=0.7)
    for rb, nr in [(0, 400), (0, 1), (37, 129), (399, 1), (5, 0)]:
        got = run_gpu(ham, lut, lp, wl.n_alpha, wl.n_beta, flags, rb, nr)
        if nr == 0:
            assert got.shape == (0,)
            continue
        srt = np.lexsort([lut[:, 0]])
        ref = OH.eloc_lut(*strings, lut[srt], lp[srt], lut[rb:rb + nr], wl.n_alpha, wl.n_beta)
        sc = abs_scale(strings, lut, lp, lut[rb:rb + nr], wl.n_alpha, wl.n_beta)
        assert np.all(np.abs(got - ref) <= TOL * sc), (rb, nr)


@pytest.fixture(scope="module")
def n40():
    wl = I.WORKLOADS["n40"]
    h, eri = I.workload_integrals(wl)
    return wl, B.build_pauli(h, eri), OH.build(h, eri)


@pytest.mark.parametrize("flags", [B.SWEEP_GROUPS, B.SWEEP_PAIRS])
def test_n40_clustered_samples(n40, flags):
    """40 qubits, 3000 clustered samples (many coupled pairs), ragged row
    window spanning several CTA tiles."""
    wl, ham, strings = n40
    lut = I.clustered_sector_samples(wl.n_spatial, wl.n_alpha, wl.n_beta, 3000, seed=7, n_centers=6)
    lp = I.random_logpsi(len(lut), seed=8, amp_std=0.5)
    rb, nr = 211, 389
    got = run_gpu(ham, lut, lp, wl.n_alpha, wl.n_beta, flags, rb, nr)
    ref = OH.eloc_lut(*strings, lut, lp, lut[rb:rb + nr], wl.n_alpha, wl.n_beta)
    sc = abs_scale(strings, lut, lp, lut[rb:rb + nr], wl.n_alpha, wl.n_beta)
    assert np.all(np.abs(got - ref) <= TOL * sc)
    # the sample set really exercises off-diagonal hits
    diag_only = np.array([OH.coupled(*strings, x, wl.n_alpha, wl.n_beta)[0].shape[0] for x in lut[rb:rb + 3]])
    assert np.all(diag_only > 1)


def test_n40_sweeps_agree_and_are_deterministic(n40):
    wl, ham, strings = n40
    lut = I.clustered_sector_samples(wl.n_spatial, wl.n_alpha, wl.n_beta, 5000, seed=9, n_centers=4)
    lp = I.random_logpsi(len(lut), seed=10, amp_std=0.5)
    a = run_gpu(ham, lut, lp, wl.n_alpha, wl.n_beta, B.SWEEP_GROUPS)
    b = run_gpu(ham, lut, lp, wl.n_alpha, wl.n_beta, B.SWEEP_PAIRS)
    a2 = run_gpu(ham, lut, lp, wl.n_alpha, wl.n_beta, B.SWEEP_GROUPS)
    assert np.array_equal(a, a2)
    assert np.abs(a - b).max() <= 1e-12 * max(1.0, np.abs(a).max())


def test_two_word_bitstrings():
    """70 qubits (two words), interacting orbitals on both sides of qubit 64."""
    n = 35
    act = [0, 9, 30, 31, 32, 34]
    h0, eri0 = I.integrals(len(act), 5, 4)
    h = np.zeros((n, n))
    eri = np.zeros((n, n, n, n))
    h[np.ix_(act, act)] = h0
    eri[np.ix_(act, act, act, act)] = eri0
    ham = B.build_pauli(h, eri)
    strings = OH.build(h, eri)
    lut = I.clustered_sector_samples(n, 3, 2, 150, seed=3, n_centers=3, orbitals=act)
    lp = I.random_logpsi(len(lut), seed=4)
    for flags in (B.SWEEP_GROUPS, B.SWEEP_PAIRS):
        got = run_gpu(ham, lut, lp, 3, 2, flags)
        ref = OH.eloc_lut(*strings, lut, lp, lut, 3, 2)
        sc = abs_scale(strings, lut, lp, lut, 3, 2)
        assert np.all(np.abs(got - ref) <= TOL * sc)


def test_device_detected_errors(n12):
    wl, h, eri, ham, strings = n12
    lut = I.sector_states(wl.n_spatial, wl.n_alpha, wl.n_beta)[:50].copy()
    lp = np.zeros((50, 2))
    bad = lut.copy()
    bad[7, 0] ^= np.uint64(1)  # one electron more or less
    with pytest.raises(B.NNQSError) as e:
        run_gpu(ham, bad, lp, wl.n_alpha, wl.n_beta, B.SWEEP_AUTO)
    assert e.value.status == B.E_SECTOR
    dup = lut.copy()
    dup[9] = dup[3]
    with pytest.raises(B.NNQSError) as e:
        run_gpu(ham, dup, lp, wl.n_alpha, wl.n_beta, B.SWEEP_AUTO)
    assert e.value.status == B.E_DUPLICATE
    high = lut.copy()
    high[2, 0] |= np.uint64(1) << np.uint64(40)
    with pytest.raises(B.NNQSError) as e:
        run_gpu(ham, high, lp, wl.n_alpha, wl.n_beta, B.SWEEP_AUTO)
    assert e.value.status == B.E_INVAL
    lutd = B.to_device_bits(lut)
    lpd = torch.from_numpy(lp).cuda()
    out = torch.empty((50, 2), dtype=torch.float64, device="cuda")
    small = B.workspace(256)
    st = B.lib().nnqs_eloc(ham.handle, None, None, B._ptr(lutd), B._ptr(lpd), 50, 0, 50, 3, 3, B.SA,
                           B.FP64, 0, B._ptr(out), B._ptr(small), 256, B._stream())
    assert st == B.E_WORKSPACE
    st = B.lib().nnqs_eloc(ham.handle, None, None, B._ptr(lutd), None, 50, 0, 50, 3, 3, B.SA,
                           B.FP64, 0, B._ptr(out), B._ptr(small), 256, B._stream())
    assert st == B.E_INVAL  # no log-psi table in sample-aware mode
    # the context is still usable afterwards
    got = run_gpu(ham, lut, lp, wl.n_alpha, wl.n_beta, B.SWEEP_AUTO)
    assert np.all(np.isfinite(got))


def test_energy_stats_match_oracle():
    rng = np.random.default_rng(0)
    for n in (1, 7, 1000, 70001):
        e = rng.normal(size=n) + 1j * rng.normal(size=n)
        w = rng.integers(1, 1000, size=n).astype(np.uint64)
        et = torch.from_numpy(np.stack([e.real, e.imag], 1)).cuda()
        wt = torch.from_numpy(w.view(np.int64)).cuda()
        s = B.energy_stats(et, wt).cpu().numpy()
        E, var = OV.energy_stats(e, w)
        assert abs(s[0] - E.real) < 1e-12 and abs(s[1] - E.imag) < 1e-12
        assert abs(s[2] - var) < 1e-12 * max(1, var) and s[3] == w.astype(np.float64).sum()


def test_ungrouped_terms_sweep_equals_grouped(n40):
    """The ungrouped layout (every string probes its own coupled x') gives the
    sample-aware E_loc of the grouped sweeps (Alg. 2) up to the order of the
    FP64 additions, on clustered 40-qubit samples and on the 70-qubit
    two-word case."""
    wl, ham, strings = n40
    lut = I.clustered_sector_samples(wl.n_spatial, wl.n_alpha, wl.n_beta, 3000, seed=11, n_centers=5)
    lp = I.random_logpsi(len(lut), seed=12, amp_std=0.5)
    ham.build_ungrouped()
    a = run_gpu(ham, lut, lp, wl.n_alpha, wl.n_beta, B.SWEEP_TERMS)
    b = run_gpu(ham, lut, lp, wl.n_alpha, wl.n_beta, B.SWEEP_GROUPS)
    c = run_gpu(ham, lut, lp, wl.n_alpha, wl.n_beta, B.SWEEP_PAIRS)
    sc = abs_scale(strings, lut, lp, lut, wl.n_alpha, wl.n_beta)
    assert np.all(np.abs(a - b) <= 1e-12 * sc)
    assert np.all(np.abs(a - c) <= 1e-12 * sc)
    rb, nr = 101, 257
    d = run_gpu(ham, lut, lp, wl.n_alpha, wl.n_beta, B.SWEEP_TERMS, rb, nr)
    assert np.all(np.abs(d - a[rb:rb + nr]) <= 1e-12 * sc[rb:rb + nr])
    # two words per bitstring
    n = 35
    act = [0, 9, 30, 31, 32, 34]
    h0, eri0 = I.integrals(len(act), 5, 4)
    h = np.zeros((n, n))
    eri = np.zeros((n, n, n, n))
    h[np.ix_(act, act)] = h0
    eri[np.ix_(act, act, act, act)] = eri0
    ham2 = B.build_pauli(h, eri)
    ham2.build_ungrouped()
    lut2 = I.clustered_sector_samples(n, 3, 2, 150, seed=3, n_centers=3, orbitals=act)
    lp2 = I.random_logpsi(len(lut2), seed=4)
    ref = OH.eloc_lut(*OH.build(h, eri), lut2, lp2, lut2, 3, 2)
    got = run_gpu(ham2, lut2, lp2, 3, 2, B.SWEEP_TERMS)
    assert np.all(np.abs(got - ref) <= TOL * abs_scale(OH.build(h, eri), lut2, lp2, lut2, 3, 2))


@pytest.mark.parametrize("flags", [B.SWEEP_GROUPS, B.SWEEP_PAIRS, B.SWEEP_TERMS])
def test_ratio_table_and_direct_rows(n12, flags):
    """Every coupled sample is a hit on the whole 12-qubit sector.  The ratio
    psi(x')/psi(x) comes from the per-sample table psi = exp(log|psi| - max)
    e^{i phase} for ordinary rows, and from the direct FP64 exp / sincos for
    rows more than 600 below the table's largest log|psi| (every 7th row
    here, 650 below): both against the oracle's direct exp."""
    wl, h, eri, ham, strings = n12
    if flags == B.SWEEP_TERMS:
        ham.build_ungrouped()
    lut = I.sector_states(wl.n_spatial, wl.n_alpha, wl.n_beta)
    lp = I.random_logpsi(len(lut), seed=21, amp_std=0.3)
    lp[::7, 0] -= 650.0
    got = run_gpu(ham, lut, lp, wl.n_alpha, wl.n_beta, flags)
    ref = OH.eloc_lut(*strings, lut, lp, lut, wl.n_alpha, wl.n_beta)
    sc = abs_scale(strings, lut, lp, lut, wl.n_alpha, wl.n_beta)
    assert np.all(np.isfinite(got))
    assert np.all(np.abs(got - ref) <= TOL * sc)
