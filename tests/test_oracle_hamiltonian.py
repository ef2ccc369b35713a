"""Pins of the oracle's Hamiltonian and local energy against what the
mathematics fixes: the determinant (Slater-Condon) rule, explicit Kronecker-
product Jordan-Wigner matrices, closed-form counts, Hermiticity, number
conservation and the exact-eigenstate invariant of Eq. (Eloc)."""
import math
from functools import reduce

import numpy as np
import pytest

from oracle import ansatz as OA
from oracle import hamiltonian as OH
from paper_2306_16705_gb300 import inputs as I


def closed_counts(N, n_occ):
    """N_h, N_XY and C_x for dense generic integrals: counted by string class
    (identity, Z, ZZ, one-body hops with Z/ZZ dressings, the X/Y patterns of
    four distinct spatial-orbital excitations, and pair excitations) and by
    single/double excitations within the (n_occ, n_occ) sector."""
    n = N // 2
    C = math.comb
    nh = 1 + N + C(N, 2) + 4 * (N - 1) * C(n, 2) + 12 * C(n, 4) + 4 * C(n, 2) ** 2
    nxy = 1 + 2 * C(n, 2) + 2 * C(n, 4) + C(n, 2) ** 2
    nv = n - n_occ
    cx = 1 + 2 * n_occ * nv + 2 * C(n_occ, 2) * C(nv, 2) + (n_occ * nv) ** 2
    return nh, nxy, cx


def kron_jw_matrix(h, eri, e_core=0.0):
    """Dense 2^N matrix of Eq. (eham) with every a+_j written as the explicit
    Kronecker product Z x ... x Z x (X - iY)/2 x I x ... (qubit 0 = least
    significant bit of the basis index)."""
    n = h.shape[0]
    N = 2 * n
    I2 = np.eye(2)
    Z = np.diag([1.0, -1.0])
    X = np.array([[0, 1], [1, 0]], dtype=complex)
    Y = np.array([[0, -1j], [1j, 0]])
    cr = (X - 1j * Y) / 2

    def op(j, dag):
        mats = []
        for q in range(N):  # index bit q = qubit q -> kron order reversed
            mats.append(Z if q < j else ((cr if dag else cr.conj().T) if q == j else I2))
        return reduce(np.kron, mats[::-1])

    A = [op(j, True) for j in range(N)]
    Aa = [op(j, False) for j in range(N)]
    H = e_core * np.eye(2 ** N, dtype=complex)
    for s in range(2):
        for p in range(n):
            for q in range(n):
                H += h[p, q] * A[2 * p + s] @ Aa[2 * q + s]
    for s in range(2):
        for t in range(2):
            for p in range(n):
                for q in range(n):
                    for r in range(n):
                        for u in range(n):
                            H += 0.5 * eri[p, q, r, u] * (A[2 * p + s] @ A[2 * r + t]
                                                          @ Aa[2 * u + t] @ Aa[2 * q + s])
    return H


@pytest.mark.parametrize("n", [2, 3, 4])
def test_jw_matches_determinant_rule_full_space(n):
    h, eri = I.integrals(n, 11 + n, 3)
    xy, yz, coef = OH.build(h, eri, 0.25)
    st = np.arange(2 ** (2 * n), dtype=np.int64)
    M_det = OH.determinant_matrix(h, eri, st, 0.25)
    M_pauli = OH.pauli_matrix(xy, yz, coef, 2 * n, st)
    assert np.abs(M_det - M_pauli).max() < 1e-12


def test_jw_matches_kronecker_operators():
    n = 2
    h, eri = I.integrals(n, 5, 2)
    xy, yz, coef = OH.build(h, eri, -0.5)
    st = np.arange(2 ** (2 * n), dtype=np.int64)
    Hk = kron_jw_matrix(h, eri, -0.5)
    assert np.abs(Hk.imag).max() < 1e-13
    assert np.abs(Hk.real - OH.pauli_matrix(xy, yz, coef, 2 * n, st)).max() < 1e-12


def test_jw_matches_determinant_rule_n12_sector():
    wl = I.WORKLOADS["n12"]
    h, eri = I.workload_integrals(wl)
    xy, yz, coef = OH.build(h, eri)
    st = OH.sector_ints(wl.n_spatial, wl.n_alpha, wl.n_beta)
    M_det = OH.determinant_matrix(h, eri, st)
    M_pauli = OH.pauli_matrix(xy, yz, coef, wl.n_qubits, st)
    assert np.abs(M_det - M_pauli).max() < 1e-12


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6])
def test_counts_closed_form(n):
    h, eri = I.integrals(n, n, 4)
    xy, yz, coef = OH.build(h, eri)
    gxy, off, _, _ = OH.group(xy, yz, coef)
    nh, nxy, _ = closed_counts(2 * n, max(1, n // 2))
    assert len(coef) == nh
    assert len(gxy) == nxy
    assert off[0] == 0 and off[-1] == len(coef) and np.all(np.diff(off) > 0)


def test_counts_closed_form_n40():
    wl = I.WORKLOADS["n40"]
    h, eri = I.workload_integrals(wl)
    xy, yz, coef = OH.build(h, eri)
    gxy, off, _, _ = OH.group(xy, yz, coef)
    nh, nxy, _ = closed_counts(40, 10)
    assert (len(coef), len(gxy)) == (nh, nxy) == (233001, 46171)


def test_strings_real_and_even_y():
    """Hermitian H has real Pauli coefficients; a real symmetric H has none on
    strings with an odd number of Y (those matrices are imaginary)."""
    h, eri = I.integrals(5, 3, 4)
    xy, yz, c = OH.jw_strings(h, eri)
    ny = OH.popcount(xy & yz).sum(axis=1)
    assert np.abs(c.imag).max() < 1e-12
    assert np.abs(c[ny % 2 == 1]).max() < 1e-12
    X, Y, coef = OH.fold_and_drop(xy, yz, c)
    assert np.all(OH.popcount(X & Y).sum(axis=1) % 2 == 0)


def test_hermitian_term_by_term():
    wl = I.WORKLOADS["n12"]
    h, eri = I.workload_integrals(wl)
    xy, yz, coef = OH.build(h, eri)
    st = OH.sector_ints(wl.n_spatial, wl.n_alpha, wl.n_beta)
    M = OH.pauli_matrix(xy, yz, coef, wl.n_qubits, st)
    assert np.array_equal(M, M.T)


def test_number_conservation():
    n = 3
    h, eri = I.integrals(n, 9, 3)
    xy, yz, coef = OH.build(h, eri)
    st = np.arange(2 ** (2 * n), dtype=np.int64)
    M = OH.pauli_matrix(xy, yz, coef, 2 * n, st)
    na = OH.popcount((st & 0x555).astype(np.uint64))
    nb = OH.popcount((st & 0xAAA).astype(np.uint64))
    cross = (na[:, None] != na[None, :]) | (nb[:, None] != nb[None, :])
    assert np.abs(M[cross]).max() < 1e-13 * np.abs(h).max()


def test_diagonal_slater_condon():
    wl = I.WORKLOADS["n12"]
    h, eri = I.workload_integrals(wl)
    xy, yz, coef = OH.build(h, eri)
    st = OH.sector_ints(wl.n_spatial, wl.n_alpha, wl.n_beta)
    M = OH.pauli_matrix(xy, yz, coef, wl.n_qubits, st[:40])
    for i, s in enumerate(st[:40]):
        bits = [(int(s) >> j) & 1 for j in range(wl.n_qubits)]
        assert abs(M[i, i] - OH.diag_energy_slater_condon(h, eri, bits)) < 1e-12


@pytest.mark.parametrize("n,nocc", [(6, 3), (10, 4)])
def test_coupled_set_size_closed_form(n, nocc):
    h, eri = I.integrals(n, 21, 5)
    xy, yz, coef = OH.build(h, eri)
    S = I.random_sector_samples(n, nocc, nocc, 6, seed=3)
    _, _, cx = closed_counts(2 * n, nocc)
    for x in S:
        xs, hs = OH.coupled(xy, yz, coef, x, nocc, nocc)
        assert len(xs) == cx
        assert len({tuple(r) for r in xs}) == cx
        # every coupled state differs from x in at most 4 qubits
        assert np.all(OH.popcount(xs ^ x[None, :]).sum(axis=1) <= 4)


def test_ed_invariant_eloc_equals_ground_energy():
    """With psi the exact ground state, E_loc(x) = E0 for every x (Eq. Eloc
    with H psi = E0 psi), using the sample table = whole sector."""
    wl = I.WORKLOADS["n12"]
    h, eri = I.workload_integrals(wl)
    xy, yz, coef = OH.build(h, eri)
    E0, st, vec = OH.ed_ground(h, eri, wl.n_alpha, wl.n_beta)
    lut = I.sector_states(wl.n_spatial, wl.n_alpha, wl.n_beta)
    assert np.array_equal(lut[:, 0].astype(np.int64), st)
    lp = np.stack([np.log(np.abs(vec)), np.where(vec < 0, np.pi, 0.0)], axis=1)
    el = OH.eloc_lut(xy, yz, coef, lut, lp, lut, wl.n_alpha, wl.n_beta)
    # tolerance scale per x: sum_x' |H_xx' psi(x')/psi(x)| (cancellation guard;
    # a few sector states have |psi| ~ 1e-13 and amplify rounding)
    M = OH.determinant_matrix(h, eri, st)
    scale = np.maximum(1.0, (np.abs(M) @ np.abs(vec)) / np.abs(vec))
    assert np.all(np.abs(el - E0) <= 1e-10 * scale)
    assert np.median(np.abs(el - E0)) < 1e-12 * abs(E0)


def test_eloc_matches_dense_matvec_and_exact_mode():
    """E_loc over the whole sector equals (H psi)(x)/psi(x) with H from the
    determinant rule, and the exact-mode sum with psi from the ansatz."""
    wl = I.WORKLOADS["n12"]
    h, eri = I.workload_integrals(wl)
    xy, yz, coef = OH.build(h, eri)
    params = I.workload_params(wl, std=0.3, phase_std=0.3)
    lut = I.sector_states(wl.n_spatial, wl.n_alpha, wl.n_beta)
    bits = I.unpack_bits(lut, wl.n_qubits)
    la, ph = OA.forward(params, bits, wl.n_alpha, wl.n_beta, wl.n_heads)
    psi = np.exp(la + 1j * ph)
    M = OH.determinant_matrix(h, eri, lut[:, 0].astype(np.int64))
    ref = (M @ psi) / psi
    el = OH.eloc_lut(xy, yz, coef, lut, np.stack([la, ph], 1), lut, wl.n_alpha, wl.n_beta)
    assert np.abs(el - ref).max() < 1e-11 * np.abs(ref).max()

    def fn(packed):
        return OA.forward(params, I.unpack_bits(packed, wl.n_qubits), wl.n_alpha, wl.n_beta,
                          wl.n_heads)

    ex = OH.eloc_exact(xy, yz, coef, lut[:25], wl.n_alpha, wl.n_beta, fn)
    assert np.abs(ex - ref[:25]).max() < 1e-11 * np.abs(ref).max()


def test_variational_bound():
    wl = I.WORKLOADS["n12"]
    h, eri = I.workload_integrals(wl)
    E0, st, _ = OH.ed_ground(h, eri, wl.n_alpha, wl.n_beta)
    M = OH.determinant_matrix(h, eri, st)
    for seed in range(3):
        params = I.ansatz_params(wl.n_qubits, wl.d_model, wl.n_layers, seed, std=0.5,
                                 phase_std=0.5)
        lut = I.sector_states(wl.n_spatial, wl.n_alpha, wl.n_beta)
        la, ph = OA.forward(params, I.unpack_bits(lut, wl.n_qubits), wl.n_alpha, wl.n_beta,
                            wl.n_heads)
        psi = np.exp(la + 1j * ph)
        E = np.vdot(psi, M @ psi).real / np.vdot(psi, psi).real
        assert E >= E0 - 1e-12


def test_w2_bitstrings_match_w1_subset():
    """Two-word keys: a 66-qubit molecule's row, restricted to states that only
    move electrons among the low 64 qubits, equals the same computation with
    the key split across words (checks the word indexing of the oracle)."""
    n = 33
    rng = np.random.default_rng(0)
    h = np.zeros((n, n))
    eri = np.zeros((n, n, n, n))
    # only orbitals 0, 1, 31, 32 interact: crosses the word boundary at qubit 64
    act = [0, 1, 31, 32]
    for p in act:
        for q in act:
            h[p, q] = h[q, p] = rng.normal() if p != q else -1.0
    xy, yz, coef = OH.build(h, eri)
    assert xy.shape[1] == 2
    # compare with the same active space relabelled onto orbitals 0..3
    h4 = h[np.ix_(act, act)]
    xy4, yz4, coef4 = OH.build(h4, np.zeros((4, 4, 4, 4)))
    st4 = OH.sector_ints(4, 1, 1)
    M4 = OH.pauli_matrix(xy4, yz4, coef4, 8, st4)
    # build the 66-qubit row for each state of the relabelled sector
    def embed(s):
        bits = np.zeros(66, dtype=np.uint8)
        for k, p in enumerate(act):
            bits[2 * p] = (s >> (2 * k)) & 1
            bits[2 * p + 1] = (s >> (2 * k + 1)) & 1
        return I.pack_occupations(bits[None, :])[0]
    keys = {tuple(int(v) for v in embed(int(s))): i for i, s in enumerate(st4)}
    for j, s in enumerate(st4):
        xs, hs = OH.coupled(xy, yz, coef, embed(int(s)), 1, 1)
        for xr, hv in zip(xs, hs):
            i = keys[tuple(int(v) for v in xr)]
            # Z strings between orbitals 1 and 31 are empty here, so the
            # matrix elements agree exactly with the compact relabelling
            assert abs(M4[j, i] - hv) < 1e-13


@pytest.mark.parametrize("n,na,nb,seed", [(6, 3, 3, 0), (5, 2, 3, 7), (4, 1, 2, 2)])
def test_slater_condon_matches_determinant_rule(n, na, nb, seed):
    """The closed-form Slater-Condon elements (integrals only) equal the
    matrix built by applying the second-quantised operators of Eq. (eham) to
    determinants, over a whole sector (every 0-, 1- and 2-orbital pair)."""
    h, eri = I.integrals(n, seed, 4)
    st = OH.sector_ints(n, na, nb)
    M = OH.determinant_matrix(h, eri, st, 0.3)
    S = np.array([[OH.slater_condon(h, eri, int(a), int(b), 0.3) for b in st] for a in st])
    assert np.abs(S - M).max() < 1e-12 * max(1.0, np.abs(M).max())


def test_eloc_slater_condon_matches_pauli_strings():
    """The second sample-aware E_loc path (Slater-Condon elements, no strings)
    equals the Pauli-string E_loc of Alg. 2 on clustered 40-qubit samples."""
    wl = I.WORKLOADS["n40"]
    h, eri = I.workload_integrals(wl)
    xy, yz, coef = OH.build(h, eri)
    lut = I.clustered_sector_samples(wl.n_spatial, wl.n_alpha, wl.n_beta, 800, seed=3, n_centers=3)
    lp = I.random_logpsi(len(lut), seed=4, amp_std=0.5)
    rows = np.array([0, 17, 401, 799])
    a = OH.eloc_lut(xy, yz, coef, lut, lp, lut[rows], wl.n_alpha, wl.n_beta)
    b, sc = OH.eloc_slater_condon(h, eri, lut, lp, rows)
    assert np.all(np.abs(a - b) <= 1e-11 * sc)
    diag = np.array([OH.slater_condon(h, eri, OH.words_to_int(lut[i]), OH.words_to_int(lut[i])) for i in rows])
    assert np.all(np.abs(b - diag) > 1e-3)  # off-diagonal pairs contribute
