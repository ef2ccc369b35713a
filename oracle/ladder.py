"""The CPU rungs of the local-energy speed-up ladder (Sec. 4.3, Fig.
speedup-eloc): bare, SA+FUSE and +LUT, each the sample-aware sum of Eq.
(Eloc) over the grouped Hamiltonian of Alg. 1 (ladder.c says what each rung
does).  TEST INFRASTRUCTURE, timed by the benchmark's CPU baseline.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import lib

RUNGS = ("bare", "sa_fuse", "lut")


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def tuples_of(keys: np.ndarray, n_qubits: int) -> np.ndarray:
    """[n][W] uint64 bitstrings -> [n][N] uint8 boolean tuples (qubit q =
    bit q % 64 of word q // 64)."""
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    q = np.arange(n_qubits)
    return np.ascontiguousarray(((keys[:, q // 64] >> (q % 64).astype(np.uint64)) & np.uint64(1)).astype(np.uint8))


def tuple_table(keys, logpsi, n_qubits):
    """S as boolean tuples sorted in byte-wise (memcmp) order, with log psi
    permuted alike: the table of the first two rungs."""
    t = tuples_of(keys, n_qubits)
    order = np.lexsort(t.T[::-1])  # column 0 is the primary key
    return np.ascontiguousarray(t[order]), np.ascontiguousarray(np.asarray(logpsi, dtype=np.float64)[order])


def eloc(rung: str, n_qubits: int, gxy, goff, yz, coef, keys, logpsi, x, table=None) -> np.ndarray:
    """E_loc of the rows x by one rung; keys sorted ascending with logpsi in
    the same order (``table``: tuple_table's result, reused across calls);
    returns complex [len(x)]."""
    W = keys.shape[1]
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    tuples, tlp = tuple_table(keys, logpsi, n_qubits) if table is None else table
    gxy = np.ascontiguousarray(gxy, dtype=np.uint64)
    goff = np.ascontiguousarray(goff, dtype=np.int64)
    yz = np.ascontiguousarray(yz, dtype=np.uint64)
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    lp = np.ascontiguousarray(logpsi, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.uint64)
    out = np.zeros(2 * len(x))
    rc = lib().ladder_eloc(RUNGS.index(rung), n_qubits, W, len(goff) - 1, _ptr(gxy), _ptr(goff), _ptr(yz),
                           _ptr(coef), len(keys), _ptr(keys), _ptr(lp), _ptr(tuples), _ptr(tlp), len(x), _ptr(x),
                           _ptr(out))
    if rc != 0:
        raise RuntimeError("ladder_eloc failed (a row not in S, or no memory)")
    return out[0::2] + 1j * out[1::2]
