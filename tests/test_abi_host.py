"""CPU-only checks of the C ABI: the library loads, exports every function
include/nnqs.h declares, and its host-side Hamiltonian builder (Eq. eham ->
Eq. sham, Alg. 1) reproduces the oracle's tables: masks, offsets and the
coupled sets bit for bit, coefficients to rounding."""
import os
import re

import numpy as np
import pytest

from oracle import hamiltonian as OH
from paper_2306_16705_gb300 import _build
from paper_2306_16705_gb300 import binding as B
from paper_2306_16705_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    B.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "nnqs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nnqs_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported():
    import ctypes
    L = ctypes.CDLL(B.lib_path())
    names = declared_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    # and the binding declares the same set
    assert set(names) == set(B._SIGS), set(names) ^ set(B._SIGS)


def _compare(n, seed, rank, e_core=0.0):
    h, eri = I.integrals(n, seed, rank)
    ham = B.build_pauli(h, eri, e_core, device=False)
    gxy, off, yz, coef = ham.export()
    oxy, oyz, ocoef = OH.build(h, eri, e_core)
    ogxy, ooff, _, _ = OH.group(oxy, oyz, ocoef)
    assert np.array_equal(gxy, ogxy)
    assert np.array_equal(off, ooff)
    assert np.array_equal(yz, oyz)
    assert np.abs(coef - ocoef).max() <= 1e-13 * max(1.0, np.abs(ocoef).max())
    return ham, (oxy, oyz, ocoef)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 6])
def test_host_builder_matches_oracle_small(n):
    _compare(n, 40 + n, 3, e_core=0.7)


def test_host_builder_matches_oracle_n40_and_coupled_sets():
    wl = I.WORKLOADS["n40"]
    ham, (oxy, oyz, ocoef) = _compare(wl.n_spatial, wl.seed, wl.rank)
    info = ham.info()
    assert (info["n_terms"], info["n_groups"]) == (233001, 46171)
    S = I.random_sector_samples(wl.n_spatial, wl.n_alpha, wl.n_beta, 3, seed=5)
    for x in S:
        xs, hs = ham.coupled(x, wl.n_alpha, wl.n_beta)
        oxs, ohs = OH.coupled(oxy, oyz, ocoef, x, wl.n_alpha, wl.n_beta)
        o = np.lexsort([xs[:, w] for w in range(xs.shape[1])])
        assert np.array_equal(xs[o], oxs)  # same set, bit-exact
        assert np.abs(hs[o] - ohs).max() < 1e-12


def test_host_builder_two_words():
    """A 70-qubit molecule (two words per bitstring) with a sparse active set
    so the oracle stays fast: orbitals straddling qubit 64."""
    n = 35
    h0, eri0 = I.integrals(5, 77, 3)
    act = [0, 16, 31, 32, 34]
    h = np.zeros((n, n))
    eri = np.zeros((n, n, n, n))
    h[np.ix_(act, act)] = h0
    eri[np.ix_(act, act, act, act)] = eri0
    ham, (oxy, oyz, ocoef) = _compare_arrays(h, eri)
    assert ham.info()["n_words"] == 2
    rng = np.random.default_rng(0)
    for _ in range(4):
        occ = np.zeros(70, dtype=np.uint8)
        for p in rng.choice(act, 2, replace=False):
            occ[2 * p] = 1
        for p in rng.choice(act, 3, replace=False):
            occ[2 * p + 1] = 1
        x = I.pack_occupations(occ[None])[0]
        xs, hs = ham.coupled(x, 2, 3)
        oxs, ohs = OH.coupled(oxy, oyz, ocoef, x, 2, 3)
        o = np.lexsort([xs[:, w] for w in range(2)])
        assert np.array_equal(xs[o], oxs)
        assert np.abs(hs[o] - ohs).max() < 1e-12


def _compare_arrays(h, eri):
    ham = B.build_pauli(h, eri, device=False)
    gxy, off, yz, coef = ham.export()
    oxy, oyz, ocoef = OH.build(h, eri)
    ogxy, ooff, _, _ = OH.group(oxy, oyz, ocoef)
    assert np.array_equal(gxy, ogxy) and np.array_equal(off, ooff) and np.array_equal(yz, oyz)
    assert np.abs(coef - ocoef).max() <= 1e-13 * max(1.0, np.abs(ocoef).max())
    return ham, (oxy, oyz, ocoef)


def test_argument_errors_are_status_codes():
    h, eri = I.integrals(2, 0, 1)
    with pytest.raises(B.NNQSError) as e:
        B.build_pauli(np.zeros((65, 65)), np.zeros((1,)), device=False)
    assert e.value.status == B.E_INVAL
    bad = h.copy()
    bad[0, 0] = np.nan
    with pytest.raises(B.NNQSError) as e:
        B.build_pauli(bad, eri, device=False)
    assert e.value.status == B.E_NONFINITE


def test_entry_points_reject_bad_arguments_before_any_device_work():
    """Null handles, negative counts and empty sample sets come back as
    NNQS_E_INVAL with a message, from the host-side checks alone (these calls
    touch no device)."""
    L = B.lib()
    assert L.nnqs_energy_stats(None, None, 0, None, None, 0, None) == B.E_INVAL
    assert L.nnqs_last_error()
    assert L.nnqs_energy_grad(None, None, None, None, None, 0, 0, None, None, None, None, None, 0,
                              None) == B.E_INVAL
    assert L.nnqs_logpsi(None, None, None, 4, 0, None, None, 0, None) == B.E_INVAL
    assert L.nnqs_logpsi_backward(None, None, None, -1, 0, None, None, None, None, 0, None) == B.E_INVAL
    assert L.nnqs_sample(None, None, 16, 1, 0, 0, 8, None, None, None, None, 0, None) == B.E_INVAL
    assert L.nnqs_eloc(None, None, None, None, None, 0, 0, 0, 1, 1, 0, 0, 0, None, None, 0,
                       None) == B.E_INVAL


def test_model_layout_matches_named_shapes():
    wl = I.WORKLOADS["n40"]
    m = B.Model(wl.n_qubits, wl.n_alpha, wl.n_beta, wl.d_model, wl.n_layers, wl.n_heads)
    shapes = I.ansatz_shapes(wl.n_qubits, wl.d_model, wl.n_layers)
    off = 0
    for name, shape in shapes:
        o, n = m.offset(name)
        assert (o, n) == (off, int(np.prod(shape))), name
        off += n
    assert m.n_params == off


def test_layout_bytes_grouped_vs_ungrouped():
    """Byte counts of the grouped layout (Alg. 1) and the ungrouped one it
    replaces (Sec. 3.4): per-group and per-string sizes applied to the built
    40-qubit Hamiltonian, and at 120 qubits (closed-form string and group
    counts of dense integrals) the one-byte-per-qubit forms give 2.97 GB
    against 4.85 GB, a 39 % reduction."""
    from math import comb

    wl = I.WORKLOADS["n40"]
    h, eri = I.workload_integrals(wl)
    ham = B.build_pauli(h, eri, device=False)
    i = ham.info()
    T, G, N, W = i["n_terms"], i["n_groups"], i["n_qubits"], i["n_words"]
    b = ham.layout_bytes()
    assert b["grouped"] == G * (8 * W + 5) + T * (8 * W + 8)
    assert b["ungrouped"] == T * (16 * W + 8)
    assert b["grouped_bytewise"] == G * (N + 4) + T * (N + 8)
    assert b["ungrouped_bytewise"] == T * (2 * N + 12)
    assert b["grouped"] < b["ungrouped"]
    n, N = 60, 120
    T120 = 1 + N + comb(N, 2) + 4 * (N - 1) * comb(n, 2) + 12 * comb(n, 4) + 4 * comb(n, 2) ** 2
    G120 = 1 + 2 * comb(n, 2) + 2 * comb(n, 4) + comb(n, 2) ** 2
    d2 = G120 * (N + 4) + T120 * (N + 8)
    d1 = T120 * (2 * N + 12)
    assert abs(d2 / 1e9 - 2.97) < 0.01 and abs(d1 / 1e9 - 4.85) < 0.01
    assert abs((1 - d2 / d1) - 0.39) < 0.01


def test_lr_warmup_host_call_matches_oracle():
    """nnqs_lr_warmup is host-only: it runs without a GPU and follows the
    oracle's Sec. 4.1 schedule; invalid arguments give 0."""
    from oracle import vmc as OV
    for d in (32, 64, 128):
        for i in (1, 2, 100, 3999, 4000, 4001, 12345, 10 ** 5):
            assert B.lr_warmup(i, d, 4000) == pytest.approx(OV.lr_warmup(i, d, 4000), rel=1e-15)
    assert B.lr_warmup(0, 64, 4000) == 0.0 and B.lr_warmup(5, 0, 4000) == 0.0 and B.lr_warmup(5, 64, 0) == 0.0


def test_paper_sample_schedule():
    """N_s of Sec. 4.1: 10^5 for the first 100 iterations, then tenfold per
    100 iterations (the reading of 'gradually') up to 10^12."""
    from paper_2306_16705_gb300.vmc import paper_n_samples
    assert [paper_n_samples(i) for i in (0, 99)] == [10 ** 5] * 2
    assert [paper_n_samples(i) for i in (100, 199, 200, 700)] == [10 ** 6, 10 ** 6, 10 ** 7, 10 ** 12]
    assert paper_n_samples(10 ** 5) == 10 ** 12


def test_tree_reuse_host_logic():
    """The host-side rules of the energy gradient from the sampler's tree
    (nnqs_energy_grad_sampled): it applies to d_model = 64 with BF16 or split
    BF16 arithmetic and at most 65,536 unique samples, and the keep-mode
    sampler workspace holds the kept rows on top of the plain one (2 L + 1
    rows of 64 floats per tree node, at least T max_unique nodes)."""
    lib = B.lib()
    m = B.Model(40, 10, 10, 64, 4, 8)
    assert lib.nnqs_energy_grad_sampled_supported(m.handle, B.BF16X3, 1 << 15) == 1
    assert lib.nnqs_energy_grad_sampled_supported(m.handle, B.MIXED, 1 << 15) == 1
    assert lib.nnqs_energy_grad_sampled_supported(m.handle, B.FP32, 1 << 15) == 0
    assert lib.nnqs_energy_grad_sampled_supported(m.handle, B.FP64, 1 << 15) == 0
    assert lib.nnqs_energy_grad_sampled_supported(m.handle, B.BF16X3, 1 << 17) == 0
    small = B.Model(12, 3, 3, 32, 2, 4)
    assert lib.nnqs_energy_grad_sampled_supported(small.handle, B.BF16X3, 512) == 0
    mu = 1 << 12
    plain = lib.nnqs_sample_workspace_size(m.handle, mu, B.BF16X3, 0)
    keep = lib.nnqs_sample_workspace_size(m.handle, mu, B.BF16X3, B.SAMPLE_KEEP)
    assert keep - plain >= 20 * mu * (2 * 4 + 1) * 64 * 4
