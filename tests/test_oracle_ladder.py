"""The CPU rungs of the local-energy speed-up ladder (Sec. 4.3, Fig.
speedup-eloc) compute the same sample-aware sum as the oracle's definitional
E_loc (ungrouped strings, hash-merged rows, binary search): on the whole
12-qubit sector, on clustered 40-qubit samples (many coupled pairs inside S),
and on two-word 70-qubit strings."""
import numpy as np
import pytest

from oracle import hamiltonian as OH
from oracle import ladder as OL
from paper_2306_16705_gb300 import inputs as I


def grouped(h, eri):
    xy, yz, coef = OH.build(h, eri)
    return OH.group(xy, yz, coef), (xy, yz, coef)


def check(n_qubits, na, nb, h, eri, lut, lp, rows):
    (gxy, goff, gyz, gcoef), (xy, yz, coef) = grouped(h, eri)
    ref = OH.eloc_lut(xy, yz, coef, lut, lp, lut[rows], na, nb)
    scale = max(1.0, float(np.abs(ref).max()))
    for rung in OL.RUNGS:
        got = OL.eloc(rung, n_qubits, gxy, goff, gyz, gcoef, lut, lp, lut[rows])
        assert np.abs(got - ref).max() <= 1e-12 * scale, rung
    return ref


def test_ladder_rungs_n12_sector():
    wl = I.WORKLOADS["n12"]
    h, eri = I.workload_integrals(wl)
    S = I.sector_states(wl.n_spatial, wl.n_alpha, wl.n_beta)
    lp = I.random_logpsi(len(S), seed=3, amp_std=0.3)
    ref = check(wl.n_qubits, wl.n_alpha, wl.n_beta, h, eri, S, lp, np.arange(len(S)))
    assert np.count_nonzero(np.abs(ref) > 1e-8) > 100


def test_ladder_rungs_n40_clustered():
    wl = I.WORKLOADS["n40"]
    h, eri = I.workload_integrals(wl)
    S = I.clustered_sector_samples(wl.n_spatial, wl.n_alpha, wl.n_beta, 600, seed=4, n_centers=3)
    lp = I.random_logpsi(len(S), seed=5, amp_std=0.2)
    check(wl.n_qubits, wl.n_alpha, wl.n_beta, h, eri, S, lp, np.array([0, 1, 77, 298, 599]))


def test_ladder_rungs_two_words():
    """70 qubits (two words) with integrals on a 6-orbital active space."""
    n = 35
    act = [0, 9, 30, 31, 32, 34]
    h0, eri0 = I.integrals(len(act), 5, 4)
    h = np.zeros((n, n))
    eri = np.zeros((n, n, n, n))
    h[np.ix_(act, act)] = h0
    eri[np.ix_(act, act, act, act)] = eri0
    S = I.clustered_sector_samples(n, 3, 2, 150, seed=3, n_centers=3, orbitals=act)
    lp = I.random_logpsi(len(S), seed=6, amp_std=0.2)
    check(2 * n, 3, 2, h, eri, S, lp, np.arange(len(S)))


def test_ladder_row_not_in_table_is_an_error():
    wl = I.WORKLOADS["n12"]
    h, eri = I.workload_integrals(wl)
    S = I.sector_states(wl.n_spatial, wl.n_alpha, wl.n_beta)
    (gxy, goff, gyz, gcoef), _ = grouped(h, eri)
    lp = I.random_logpsi(len(S), seed=3)
    for rung in OL.RUNGS:
        with pytest.raises(RuntimeError):
            OL.eloc(rung, wl.n_qubits, gxy, goff, gyz, gcoef, S[1:], lp[1:], S[:1])
