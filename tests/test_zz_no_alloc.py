"""nnqs_eloc_sa_noalloc: the sample-aware local energy for callers that
cannot hand the library device memory (a host application that owns the
GPU's memory pool, or a caller that cannot pay for cudaMalloc's device
synchronisation).  Its scratch is a fixed array inside the library.

Checked through the C ABI against nnqs_eloc on the same inputs, on two calls
in a row (the second with a different table, so stale contents of the
shared array would show), with the same per-row tolerance as the other
sample-aware tests.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2306_16705_gb300 import binding as B
from paper_2306_16705_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    B.lib()


def noalloc(ham, lut, lp, na, nb, flags, row_begin=0, n_rows=None, check=1):
    n_lut = lut.shape[0]
    n_rows = n_lut - row_begin if n_rows is None else n_rows
    out = torch.empty((n_rows, 2), dtype=torch.float64, device="cuda")
    st = B.lib().nnqs_eloc_sa_noalloc(ham.handle, B._ptr(lut), B._ptr(lp), n_lut, row_begin, n_rows, na, nb,
                                      flags, B._ptr(out), check, B._stream())
    if st != B.OK:
        raise B.NNQSError(st, B.lib().nnqs_last_error().decode())
    if not check:
        torch.cuda.current_stream().synchronize()
    return out.cpu().numpy()


def compare(ham, lut_np, na, nb, flags, rb, nr, seed, check=1):
    lut = B.to_device_bits(lut_np)
    lp = torch.from_numpy(I.random_logpsi(len(lut_np), seed=seed, amp_std=0.5)).cuda()
    ref = B.eloc(ham, lut, lp, na, nb, flags=flags, row_begin=rb, n_rows=nr).cpu().numpy()
    got = noalloc(ham, lut, lp, na, nb, flags, rb, nr, check=check)
    scale = np.maximum(1.0, np.abs(ref).max(axis=1))
    assert np.all(np.abs(got - ref).max(axis=1) <= TOL * scale)


def test_noalloc_matches_workspace_entry_point():
    wl = I.WORKLOADS["n40"]
    h, eri = I.workload_integrals(wl)
    ham = B.build_pauli(h, eri)
    cases = [
        (I.clustered_sector_samples(wl.n_spatial, wl.n_alpha, wl.n_beta, 3000, seed=31, n_centers=5), 17, 2111),
        (I.clustered_sector_samples(wl.n_spatial, wl.n_alpha, wl.n_beta, 1800, seed=32, n_centers=3), 0, 1800),
    ]
    for flags in (B.SWEEP_PAIRS, B.SWEEP_GROUPS):
        for lut_np, rb, nr in cases:  # two calls in a row on the shared array
            compare(ham, lut_np, wl.n_alpha, wl.n_beta, flags, rb, nr, seed=rb + nr)
    # the smaller table first, then the larger one (stale entries of the
    # first call sit where the second reads), asynchronous calls (check = 0)
    # with the automatic sweep choice, and the ungrouped-layout sweep
    for lut_np, rb, nr in cases[::-1]:
        compare(ham, lut_np, wl.n_alpha, wl.n_beta, B.SWEEP_AUTO, rb, nr, seed=rb + 7, check=0)
    ham.build_ungrouped()
    for lut_np, rb, nr in cases[::-1]:
        compare(ham, lut_np, wl.n_alpha, wl.n_beta, B.SWEEP_TERMS, rb, nr, seed=rb + 9)


def test_noalloc_two_word_bitstrings():
    """76 qubits: two-word keys (the 128-bit CAS hash), both sweeps and the
    automatic choice, two tables of growing size in a row."""
    wl = I.WORKLOADS["n76"]
    h, eri = I.workload_integrals(wl)
    ham = B.build_pauli(h, eri)
    small = I.clustered_sector_samples(wl.n_spatial, wl.n_alpha, wl.n_beta, 700, seed=41, n_centers=3)
    large = I.clustered_sector_samples(wl.n_spatial, wl.n_alpha, wl.n_beta, 2500, seed=42, n_centers=4)
    for flags in (B.SWEEP_PAIRS, B.SWEEP_GROUPS, B.SWEEP_AUTO):
        compare(ham, small, wl.n_alpha, wl.n_beta, flags, 0, 700, seed=5)
        compare(ham, large, wl.n_alpha, wl.n_beta, flags, 300, 1500, seed=6, check=0)


def test_noalloc_reports_device_errors_and_limits():
    wl = I.WORKLOADS["n12"]
    h, eri = I.workload_integrals(wl)
    ham = B.build_pauli(h, eri)
    lut_np = I.sector_states(wl.n_spatial, wl.n_alpha, wl.n_beta)[:64].copy()
    lut_np[5] = lut_np[9]  # duplicate row
    lut = B.to_device_bits(lut_np)
    lp = torch.zeros((64, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(B.NNQSError) as e:
        noalloc(ham, lut, lp, wl.n_alpha, wl.n_beta, B.SWEEP_AUTO)
    assert e.value.status == B.E_DUPLICATE
    # a table too large for the fixed scratch is refused before any launch
    # (real buffers of that size, so nothing could read past them anyway)
    big = 1 << 23
    big_lut = torch.zeros(big, dtype=torch.int64, device="cuda")
    big_lp = torch.zeros((big, 2), dtype=torch.float64, device="cuda")
    out = torch.empty((1, 2), dtype=torch.float64, device="cuda")
    st = B.lib().nnqs_eloc_sa_noalloc(ham.handle, B._ptr(big_lut), B._ptr(big_lp), big, 0, 1, 3, 3,
                                      B.SWEEP_AUTO, B._ptr(out), 1, B._stream())
    assert st == B.E_INVAL
    assert "scratch" in B.lib().nnqs_last_error().decode()
