"""Oracle: the qubit Hamiltonian, its pins, and the local energy.

TEST INFRASTRUCTURE (see the package docstring).

Readings of the paper used here:
* spin orbital P = 2p + s (s = 0 alpha, 1 beta), qubit P (Sec. 3.3);
* H = e_core + sum h_pq a+_{ps} a_{qs}
      + 1/2 sum (pq|rs) a+_{ps} a+_{rt} a_{st} a_{qs}        (Eq. eham with
  the physicist integral g^{PQ}_{RS} = (PS|QR) and spin deltas);
* Jordan-Wigner a+_j = Z_{<j}(X_j - iY_j)/2 with |1> occupied (Sec. 2.3);
* folded coefficient coef = Re(c) Re((-i)^{nY}) (Alg. 1), strings with
  |coef| < 1e-12 dropped;
* groups and terms in ascending key order (Alg. 1 keeps dictionary order,
  which only changes the order of a sum).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import lib

EVEN = np.uint64(0x5555555555555555)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def popcount(a):
    a = np.asarray(a, dtype=np.uint64)
    if hasattr(np, "bitwise_count"):
        return np.bitwise_count(a).astype(np.int64)
    out = np.zeros(a.shape, dtype=np.int64)
    v = a.copy()
    while np.any(v):
        out += (v & np.uint64(1)).astype(np.int64)
        v >>= np.uint64(1)
    return out


def jw_strings(h, eri, e_core: float = 0.0):
    """All merged Pauli strings of Eq. (sham), unfolded and undropped.

    Returns (xy[n,W] uint64, yz[n,W] uint64, c[n] complex128) in arbitrary
    order.  Built in C by expanding every ladder-operator product (Sec. 2.3).
    """
    h = np.ascontiguousarray(h, dtype=np.float64)
    eri = np.ascontiguousarray(eri, dtype=np.float64)
    n = h.shape[0]
    W = (2 * n + 63) // 64
    L = lib()
    cnt = L.oracle_jw_build(n, _ptr(h), _ptr(eri), float(e_core))
    if cnt < 0:
        raise MemoryError("oracle_jw_build failed")
    xy = np.zeros((cnt, W), dtype=np.uint64)
    yz = np.zeros((cnt, W), dtype=np.uint64)
    re = np.zeros(cnt)
    im = np.zeros(cnt)
    if L.oracle_jw_fetch(_ptr(xy), _ptr(yz), _ptr(re), _ptr(im)) != 0:
        raise RuntimeError("oracle_jw_fetch failed")
    return xy, yz, re + 1j * im


def _key_order(*cols):
    """lexsort order with the first array's top word most significant."""
    keys = []
    for c in reversed(cols):
        for w in range(c.shape[1]):
            keys.append(c[:, w])
    return np.lexsort(keys)


def fold_and_drop(xy, yz, c, tol: float = 1e-12):
    """Alg. 1 coefficient folding coef = Re(c) * Re((-i)^{nY}) and the drop of
    |coef| < tol; result sorted by (xy, yz)."""
    ny = popcount(xy & yz).sum(axis=1)
    re_phase = np.array([1.0, 0.0, -1.0, 0.0])[ny % 4]
    coef = c.real * re_phase
    keep = np.abs(coef) >= tol
    xy, yz, coef = xy[keep], yz[keep], coef[keep]
    o = _key_order(xy, yz)
    return np.ascontiguousarray(xy[o]), np.ascontiguousarray(yz[o]), np.ascontiguousarray(coef[o])


def build(h, eri, e_core: float = 0.0, tol: float = 1e-12):
    """The folded, dropped, sorted Pauli-string Hamiltonian (xy, yz, coef)."""
    return fold_and_drop(*jw_strings(h, eri, e_core), tol=tol)


def group(xy, yz, coef):
    """Alg. 1 compaction: unique X/Y masks, CSR offsets, per-term YZ masks and
    folded coefficients.  Input sorted by (xy, yz)."""
    if len(xy) == 0:
        W = xy.shape[1]
        return np.zeros((0, W), np.uint64), np.zeros(1, np.int64), yz, coef
    change = np.any(xy[1:] != xy[:-1], axis=1)
    starts = np.concatenate([[0], np.nonzero(change)[0] + 1])
    off = np.concatenate([starts, [len(xy)]]).astype(np.int64)
    return np.ascontiguousarray(xy[starts]), off, yz, coef


def diag_energy_slater_condon(h, eri, x_bits):
    """Closed-form diagonal <x|H|x> for a determinant (Slater-Condon):
    sum_{P occ} h_PP + 1/2 sum_{P != Q occ} [(PP|QQ) - delta_{sP sQ} (PQ|QP)]."""
    occ = [P for P in range(len(x_bits)) if x_bits[P]]
    e = 0.0
    for P in occ:
        e += h[P // 2, P // 2]
    for P in occ:
        for Q in occ:
            if P == Q:
                continue
            p, q = P // 2, Q // 2
            e += 0.5 * eri[p, p, q, q]
            if P % 2 == Q % 2:
                e -= 0.5 * eri[p, q, q, p]
    return e


def _apply_ladder_string(ops, states):
    """Apply a product of ladder operators (rightmost first) to every basis
    state in ``states`` (int64 occupation integers).  The sign of a_j or a+_j
    on a determinant is (-1)^{number of occupied orbitals with index < j}.
    Returns (new_states, sign, alive)."""
    cur = states.copy()
    sign = np.ones(len(states))
    alive = np.ones(len(states), dtype=bool)
    for j, dag in reversed(ops):
        bit = (cur >> j) & 1
        alive &= (bit == 0) if dag else (bit == 1)
        below = popcount((cur & ((1 << j) - 1)).astype(np.uint64))
        sign *= np.where(below % 2 == 1, -1.0, 1.0)
        cur = cur ^ (1 << j)
    return cur, sign, alive


def determinant_matrix(h, eri, states, e_core: float = 0.0):
    """Dense <s_i|H|s_j> over a basis of occupation integers closed under H
    (the full space, or one (n_alpha, n_beta) sector), from the action of the
    second-quantised operators of Eq. (eham) on determinants."""
    states = np.asarray(states, dtype=np.int64)
    order = np.argsort(states)
    srt = states[order]
    M = np.zeros((len(states), len(states)))
    M[np.arange(len(states)), np.arange(len(states))] += e_core
    n = h.shape[0]
    cols = np.arange(len(states))

    def add(coef, ops):
        new, sign, alive = _apply_ladder_string(ops, states)
        if not np.any(alive):
            return
        pos = np.searchsorted(srt, new[alive])
        pos = np.minimum(pos, len(srt) - 1)
        ok = srt[pos] == new[alive]
        if not np.all(ok):
            raise ValueError("basis not closed under H")
        rows = order[pos]
        np.add.at(M, (rows, cols[alive]), coef * sign[alive])

    for s in range(2):
        for p in range(n):
            for q in range(n):
                if h[p, q] != 0.0:
                    add(h[p, q], [(2 * p + s, True), (2 * q + s, False)])
    for s in range(2):
        for t in range(2):
            for p in range(n):
                for q in range(n):
                    for r in range(n):
                        for u in range(n):
                            v = eri[p, q, r, u]
                            if v != 0.0:
                                add(0.5 * v, [(2 * p + s, True), (2 * r + t, True),
                                              (2 * u + t, False), (2 * q + s, False)])
    return M


def _ladder(state: int, ops):
    """Apply ladder operators (j, dagger), rightmost first, to the
    determinant ``state`` (Python int, bit P = spin orbital P occupied) with
    the sign (-1)^{occupied orbitals below j} of each step; None if the
    result vanishes, else (new_state, sign)."""
    sign = 1
    for j, dag in reversed(ops):
        occ = (state >> j) & 1
        if occ == (1 if dag else 0):
            return None
        if bin(state & ((1 << j) - 1)).count("1") % 2:
            sign = -sign
        state ^= 1 << j
    return state, sign


def _g(eri, P, Q, R, S):
    """<PQ|RS> = (PR|QS) for spin orbitals (spin deltas sigma_P = sigma_R and
    sigma_Q = sigma_S), the chemist-to-physicist reading of Eq. (eham)."""
    if P % 2 != R % 2 or Q % 2 != S % 2:
        return 0.0
    return float(eri[P // 2, R // 2, Q // 2, S // 2])


def slater_condon(h, eri, x: int, xp: int, e_core: float = 0.0):
    """<x|H|x'> for determinants x, x' (Python ints) by the Slater-Condon
    rules, straight from the integrals (no Pauli strings):
    equal: sum_I h_II + 1/2 sum_{I,J} <IJ||IJ>;
    one orbital I -> A: s (h_IA + sum_{K common} <IK||AK>);
    two orbitals I,J -> A,B: s <IJ||AB>;
    where <PQ||RS> = <PQ|RS> - <PQ|SR> and s is the sign of
    a+_I a_A |x'> (resp. a+_I a+_J a_B a_A |x'>) = s |x>.  Zero otherwise."""
    d = x ^ xp
    nd = bin(d).count("1")
    if nd == 0:
        occ = [P for P in range(x.bit_length()) if (x >> P) & 1]
        e = e_core
        for P in occ:
            e += float(h[P // 2, P // 2])
        for P in occ:
            for Q in occ:
                e += 0.5 * (_g(eri, P, Q, P, Q) - _g(eri, P, Q, Q, P))
        return e
    if nd == 2:
        (I,) = [P for P in range(d.bit_length()) if (x >> P) & 1 and (d >> P) & 1]
        (A,) = [P for P in range(d.bit_length()) if (xp >> P) & 1 and (d >> P) & 1]
        if I % 2 != A % 2:
            return 0.0
        _, s = _ladder(xp, [(I, True), (A, False)])
        v = float(h[I // 2, A // 2])
        common = x & xp
        for K in range(common.bit_length()):
            if (common >> K) & 1:
                v += _g(eri, I, K, A, K) - _g(eri, I, K, K, A)
        return s * v
    if nd == 4:
        I, J = [P for P in range(d.bit_length()) if (x >> P) & 1 and (d >> P) & 1]
        A, B = [P for P in range(d.bit_length()) if (xp >> P) & 1 and (d >> P) & 1]
        _, s = _ladder(xp, [(I, True), (J, True), (B, False), (A, False)])
        return s * (_g(eri, I, J, A, B) - _g(eri, I, J, B, A))
    return 0.0


def words_to_int(row) -> int:
    """Packed little-endian uint64 words -> Python int."""
    return sum(int(v) << (64 * k) for k, v in enumerate(np.asarray(row, dtype=np.uint64)))


def eloc_slater_condon(h, eri, lut, lut_logpsi, rows):
    """E_loc(x) = sum_{x' in lut} <x|H|x'> psi(x')/psi(x) over the sample
    table (Eq. Eloc restricted to S, Sec. 3.4) with the matrix elements of
    ``slater_condon``: a second path to the sample-aware local energy that
    does not go through the Jordan-Wigner strings.  Also returns
    sum_x' |<x|H|x'> psi(x')/psi(x)| per row.  ``lut`` [n, W] packed,
    ``lut_logpsi`` [n, 2], ``rows`` indices into lut."""
    lut = np.ascontiguousarray(lut, dtype=np.uint64)
    lp = np.asarray(lut_logpsi, dtype=np.float64)
    out = np.zeros(len(rows), dtype=complex)
    scale = np.zeros(len(rows))
    for k, i in enumerate(rows):
        diff = sum(popcount(lut[:, w] ^ lut[i, w]) for w in range(lut.shape[1]))
        x = words_to_int(lut[i])
        for j in np.nonzero(diff <= 4)[0]:
            hv = slater_condon(h, eri, x, words_to_int(lut[j]))
            if hv == 0.0:
                continue
            r = np.exp(lp[j, 0] - lp[i, 0] + 1j * (lp[j, 1] - lp[i, 1]))
            out[k] += hv * r
            scale[k] += abs(hv * r)
    return out, np.maximum(1.0, scale)


def pauli_matrix(xy, yz, coef, n_qubits, states):
    """<s_i|H|s_j> from the folded strings: H_{x x'} = sum_t coef_t
    (-1)^{popc(x' & yz_t)} [x = x' ^ xy_t] (Eq. sham with Alg. 1 folding).
    ``states`` are occupation integers (n_qubits <= 62)."""
    assert n_qubits <= 62
    st = np.asarray(states, dtype=np.int64)
    idx = {int(s): i for i, s in enumerate(st)}
    M = np.zeros((len(st), len(st)))
    xyi = xy[:, 0].astype(np.int64)
    yzi = yz[:, 0].astype(np.int64)
    for j, xp in enumerate(st):
        x = xp ^ xyi
        sgn = np.where(popcount((xp & yzi).astype(np.uint64)) % 2 == 1, -1.0, 1.0)
        for t in range(len(coef)):
            i = idx.get(int(x[t]))
            if i is not None:
                M[i, j] += coef[t] * sgn[t]
    return M


def sector_ints(n_spatial, n_alpha, n_beta):
    from itertools import combinations
    out = []
    for a in combinations(range(n_spatial), n_alpha):
        for b in combinations(range(n_spatial), n_beta):
            v = 0
            for p in a:
                v |= 1 << (2 * p)
            for p in b:
                v |= 1 << (2 * p + 1)
            out.append(v)
    return np.array(sorted(out), dtype=np.int64)


def ed_ground(h, eri, n_alpha, n_beta, e_core: float = 0.0):
    """Exact ground state in one (n_alpha, n_beta) sector from the
    determinant-rule matrix and numpy.linalg.eigh.  Returns (E0, states,
    vector) with states ascending."""
    n = h.shape[0]
    st = sector_ints(n, n_alpha, n_beta)
    M = determinant_matrix(h, eri, st, e_core)
    w, v = np.linalg.eigh(M)
    return w[0], st, v[:, 0]


def coupled(xy, yz, coef, x, n_alpha, n_beta):
    """Row of H at the packed bitstring x: (x'[k,W], H_{x x'}[k]) for every
    x' with the sector's electron counts reached by some string
    (accidental zeros kept), sorted by key."""
    W = xy.shape[1]
    x = np.ascontiguousarray(np.asarray(x, dtype=np.uint64).reshape(W))
    cap = len(coef) + 1
    ox = np.zeros((cap, W), dtype=np.uint64)
    oh = np.zeros(cap)
    k = lib().oracle_coupled(W, len(coef), _ptr(xy), _ptr(yz), _ptr(coef), _ptr(x),
                             n_alpha, n_beta, _ptr(ox), _ptr(oh), cap)
    if k < 0:
        raise RuntimeError("oracle_coupled failed")
    ox, oh = ox[:k], oh[:k]
    o = _key_order(ox)
    return ox[o], oh[o]


def eloc_lut(xy, yz, coef, lut, lut_logpsi, x, n_alpha, n_beta):
    """Eq. (Eloc) with the sum over x' restricted to the sample table
    (Sec. 3.4 (4), Alg. 2).  ``lut`` [n,W] sorted ascending, ``lut_logpsi``
    [n,2] (log|psi|, phase); ``x`` [m,W] rows of lut.  Returns complex [m]."""
    W = xy.shape[1]
    lut = np.ascontiguousarray(lut, dtype=np.uint64)
    lp = np.ascontiguousarray(lut_logpsi, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.uint64)
    out = np.zeros((len(x), 2))
    rc = lib().oracle_eloc_lut(W, len(coef), _ptr(xy), _ptr(yz), _ptr(coef), len(lut),
                               _ptr(lut), _ptr(lp), len(x), _ptr(x), n_alpha, n_beta,
                               _ptr(out))
    if rc != 0:
        raise ValueError("a sample is not in the table")
    return out[:, 0] + 1j * out[:, 1]


def eloc_exact(xy, yz, coef, x, n_alpha, n_beta, logpsi_fn):
    """Eq. (Eloc) over every coupled x' (no sample restriction); log psi of
    x and of each x' from ``logpsi_fn(packed[m,W]) -> (la[m], phase[m])``."""
    out = np.zeros(len(x), dtype=np.complex128)
    for i in range(len(x)):
        xs, hs = coupled(xy, yz, coef, x[i], n_alpha, n_beta)
        la, ph = logpsi_fn(np.vstack([np.asarray(x[i]).reshape(1, -1), xs]))
        r = np.exp((la[1:] - la[0]) + 1j * (ph[1:] - ph[0]))
        out[i] = np.sum(hs * r)
    return out
