"""Seeded synthetic inputs shared by the CUDA path, its tests, the benchmark
and the CPU oracle.

This module draws random numbers and arranges them into arrays; it holds none
of the method's arithmetic (no Jordan-Wigner algebra, no local energy, no
network evaluation).  Both sides of every parity test read their inputs from
here and nowhere else.

Stand-ins.  The paper's molecules (Table 1, the benzene 6-31G run of Sec. 4.4)
come from PySCF integrals that are not available here, so every molecule is a
synthetic one with dense random integrals of the same shape:

* h_pq symmetric, diagonal -U(1,3), off-diagonal N(0, 0.1);
* (pq|rs) = sum_{k<rank} L_kpq L_krs with each L_k symmetric N(0, 0.2),
  which gives the 8-fold symmetry of real chemist-notation integrals.

The draw order is fixed: numpy ``default_rng(seed)``; n diagonal values of h;
the strict upper triangle of h, row-major; then for k = 0..rank-1 the upper
triangle (with diagonal) of L_k, row-major.

Bitstrings are packed little-endian into uint64 words: qubit j is bit (j % 64)
of word (j // 64); qubit 2p is the alpha spin orbital of spatial orbital p and
qubit 2p+1 its beta partner (the interleaved Jordan-Wigner ordering of
Sec. 3.3).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass(frozen=True)
class Workload:
    """One synthetic molecule, sample batch and ansatz shape."""

    name: str
    n_qubits: int          # N spin orbitals (qubits)
    n_alpha: int
    n_beta: int
    seed: int              # integral seed; ansatz params use seed + 100
    rank: int              # rank of the two-electron factorisation
    n_unique: int          # N_u unique samples per batch
    d_model: int
    n_layers: int
    n_heads: int
    weights: str = "uniform"  # "uniform" | "zipf" | "sampler"

    @property
    def n_spatial(self) -> int:
        return self.n_qubits // 2

    @property
    def n_words(self) -> int:
        return (self.n_qubits + 63) // 64


# The five workloads: 12 qubits (whole 3a/3b sector), 40 qubits / 20
# electrons, 76 qubits / 30 electrons, 120 qubits / 40 electrons, and the
# 30-qubit / 14-electron training run.
WORKLOADS = {
    "n12": Workload("n12", 12, 3, 3, 0, 8, 400, 32, 2, 4),
    "n40": Workload("n40", 40, 10, 10, 1, 16, 16384, 64, 4, 8, "sampler"),
    "n76": Workload("n76", 76, 15, 15, 2, 24, 65536, 64, 4, 8),
    "n120": Workload("n120", 120, 20, 20, 3, 32, 131072, 128, 6, 8, "zipf"),
    "n30": Workload("n30", 30, 7, 7, 4, 8, 8192, 64, 4, 8, "sampler"),
}

PHASE_HIDDEN = 512  # phase MLP widths N x 512 x 512 x 1 (Sec. 4.1)


def integrals(n_spatial: int, seed: int, rank: int):
    """Dense random one- and two-electron integrals (h[n,n], eri[n,n,n,n]).

    ``eri`` is in chemist order, eri[p,q,r,s] = (pq|rs).
    """
    n = n_spatial
    rng = np.random.default_rng(seed)
    h = np.zeros((n, n))
    h[np.arange(n), np.arange(n)] = -rng.uniform(1.0, 3.0, size=n)
    iu = np.triu_indices(n, 1)
    off = rng.normal(0.0, 0.1, size=iu[0].size)
    h[iu] = off
    h[(iu[1], iu[0])] = off
    L = np.zeros((rank, n, n))
    iu0 = np.triu_indices(n, 0)
    for k in range(rank):
        v = rng.normal(0.0, 0.2, size=iu0[0].size)
        L[k][iu0] = v
        L[k][(iu0[1], iu0[0])] = v
    eri = np.einsum("kpq,krs->pqrs", L, L, optimize=True)
    return h, np.ascontiguousarray(eri)


def pack_occupations(occ: np.ndarray) -> np.ndarray:
    """[B, N] 0/1 array -> [B, W] uint64 packed words."""
    occ = np.asarray(occ, dtype=np.uint64)
    B, N = occ.shape
    W = (N + 63) // 64
    out = np.zeros((B, W), dtype=np.uint64)
    for j in range(N):
        out[:, j // 64] |= occ[:, j] << np.uint64(j % 64)
    return out


def unpack_bits(x: np.ndarray, n_qubits: int) -> np.ndarray:
    """[B, W] uint64 -> [B, N] uint8 occupations."""
    x = np.asarray(x, dtype=np.uint64)
    out = np.zeros((x.shape[0], n_qubits), dtype=np.uint8)
    for j in range(n_qubits):
        out[:, j] = (x[:, j // 64] >> np.uint64(j % 64)) & np.uint64(1)
    return out


def sector_states(n_spatial: int, n_alpha: int, n_beta: int) -> np.ndarray:
    """Every bitstring with n_alpha alpha and n_beta beta electrons, packed and
    sorted ascending by (word[W-1], ..., word[0])."""
    from itertools import combinations

    N = 2 * n_spatial
    rows = []
    for a in combinations(range(n_spatial), n_alpha):
        for b in combinations(range(n_spatial), n_beta):
            occ = np.zeros(N, dtype=np.uint8)
            occ[[2 * p for p in a]] = 1
            occ[[2 * p + 1 for p in b]] = 1
            rows.append(occ)
    packed = pack_occupations(np.array(rows))
    return sort_keys(packed)


def sort_keys(x: np.ndarray) -> np.ndarray:
    """Sort packed bitstrings ascending, most significant word first."""
    x = np.asarray(x, dtype=np.uint64)
    order = np.lexsort([x[:, w] for w in range(x.shape[1])])
    return np.ascontiguousarray(x[order])


def random_sector_samples(n_spatial: int, n_alpha: int, n_beta: int,
                          n_unique: int, seed: int) -> np.ndarray:
    """``n_unique`` distinct sector bitstrings drawn uniformly, sorted."""
    rng = np.random.default_rng(seed)
    N = 2 * n_spatial
    seen = set()
    out = []
    while len(out) < n_unique:
        need = n_unique - len(out)
        batch = max(64, 2 * need)
        a = np.argsort(rng.random((batch, n_spatial)), axis=1)[:, :n_alpha]
        b = np.argsort(rng.random((batch, n_spatial)), axis=1)[:, :n_beta]
        occ = np.zeros((batch, N), dtype=np.uint8)
        rows = np.arange(batch)[:, None]
        occ[rows, 2 * a] = 1
        occ[rows, 2 * b + 1] = 1
        packed = pack_occupations(occ)
        for row in packed:
            key = tuple(int(v) for v in row)
            if key not in seen:
                seen.add(key)
                out.append(row)
                if len(out) == n_unique:
                    break
    return sort_keys(np.array(out, dtype=np.uint64))


def clustered_sector_samples(n_spatial: int, n_alpha: int, n_beta: int, n_unique: int,
                             seed: int, n_centers: int = 8, orbitals=None) -> np.ndarray:
    """``n_unique`` distinct sector bitstrings concentrated around a few random
    centres: each is a centre with 0-2 electrons moved within their spin
    (the shape of a sample set drawn from a peaked wave function, where many
    samples are coupled to each other).  ``orbitals`` restricts occupations
    to a subset of spatial orbitals.  Sorted."""
    rng = np.random.default_rng(seed)
    orbs = np.arange(n_spatial) if orbitals is None else np.asarray(orbitals)
    N = 2 * n_spatial
    centres = []
    for _ in range(n_centers):
        a = rng.choice(orbs, n_alpha, replace=False)
        b = rng.choice(orbs, n_beta, replace=False)
        centres.append((set(a.tolist()), set(b.tolist())))
    seen = set()
    out = []
    guard = 0
    while len(out) < n_unique:
        guard += 1
        if guard > 200 * n_unique + 10000:
            raise ValueError("cannot draw that many distinct clustered samples")
        a, b = centres[rng.integers(n_centers)]
        a, b = set(a), set(b)
        for _ in range(rng.integers(0, 3)):
            spin = a if rng.random() < 0.5 else b
            occ = sorted(spin)
            free = sorted(set(orbs.tolist()) - spin)
            if occ and free:
                spin.remove(occ[rng.integers(len(occ))])
                spin.add(free[rng.integers(len(free))])
        bits = np.zeros(N, dtype=np.uint8)
        bits[[2 * p for p in a]] = 1
        bits[[2 * p + 1 for p in b]] = 1
        key = bits.tobytes()
        if key in seen:
            continue
        seen.add(key)
        out.append(bits)
    return sort_keys(pack_occupations(np.array(out)))


def random_logpsi(n: int, seed: int, amp_std: float = 1.0, phase_std: float = 1.0) -> np.ndarray:
    """[n, 2] table of (log|psi|, phase) values, N(0, amp_std) and
    N(0, phase_std): a stand-in wave-function table for sample-aware sums."""
    rng = np.random.default_rng(seed)
    return np.stack([rng.normal(0.0, amp_std, n), rng.normal(0.0, phase_std, n)], axis=1)


def uniform_counts(n_unique: int, n_draws: int, seed: int) -> np.ndarray:
    """Counts from ``n_draws`` uniform draws with replacement over n_unique
    states (zero counts kept)."""
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, n_unique, size=n_draws)
    return np.bincount(idx, minlength=n_unique).astype(np.uint64)


def zipf_counts(n_unique: int, s: float, seed: int, total: float = 1e6) -> np.ndarray:
    """Heavy-tailed counts w_i = max(1, round(total * r_i^-s / H_{N_u,s})) over
    a random permutation of ranks r_i = 1..N_u."""
    rng = np.random.default_rng(seed)
    ranks = rng.permutation(n_unique) + 1
    hs = np.sum(np.arange(1, n_unique + 1, dtype=np.float64) ** (-s))
    w = np.maximum(1.0, np.round(total * ranks.astype(np.float64) ** (-s) / hs))
    return w.astype(np.uint64)


def ansatz_shapes(n_qubits: int, d_model: int, n_layers: int,
                  hidden: int = PHASE_HIDDEN):
    """Ordered (name, shape) list of every ansatz parameter.

    Linear weights are [out, in].  The qkv projection stacks Q, K, V rows.
    """
    T = n_qubits // 2
    d = d_model
    shapes = [("tok_emb", (5, d)), ("pos_emb", (T, d))]
    for l in range(n_layers):
        p = f"l{l}."
        shapes += [
            (p + "ln1.g", (d,)), (p + "ln1.b", (d,)),
            (p + "attn.wqkv", (3 * d, d)), (p + "attn.bqkv", (3 * d,)),
            (p + "attn.wo", (d, d)), (p + "attn.bo", (d,)),
            (p + "ln2.g", (d,)), (p + "ln2.b", (d,)),
            (p + "ffn.w1", (4 * d, d)), (p + "ffn.b1", (4 * d,)),
            (p + "ffn.w2", (d, 4 * d)), (p + "ffn.b2", (d,)),
        ]
    shapes += [("lnf.g", (d,)), ("lnf.b", (d,)),
               ("head.w", (4, d)), ("head.b", (4,)),
               ("phase.w1", (hidden, n_qubits)), ("phase.b1", (hidden,)),
               ("phase.w2", (hidden, hidden)), ("phase.b2", (hidden,)),
               ("phase.w3", (1, hidden)), ("phase.b3", (1,))]
    return shapes


def ansatz_params(n_qubits: int, d_model: int, n_layers: int, seed: int,
                  std: float = 0.02, bias_std: float = 0.0,
                  phase_std: float | None = None) -> dict:
    """Random-init ansatz parameters as float32 arrays, keyed by name.

    Weights and embeddings N(0, std), LayerNorm gains 1, shifts and biases
    N(0, bias_std) (zero by default).  ``phase_std`` overrides the std of the
    phase-MLP weights (tests use O(1/sqrt(fan_in)) to get non-trivial phases).
    """
    rng = np.random.default_rng(seed)
    out = {}
    for name, shape in ansatz_shapes(n_qubits, d_model, n_layers):
        if name.endswith(".g"):
            arr = np.ones(shape)
        elif name.split(".")[-1].startswith("b"):
            arr = rng.normal(0.0, bias_std, size=shape) if bias_std else np.zeros(shape)
        else:
            s = std
            if phase_std is not None and name.startswith("phase."):
                s = phase_std
            arr = rng.normal(0.0, s, size=shape)
        out[name] = arr.astype(np.float32)
    return out


def workload_integrals(wl: Workload):
    return integrals(wl.n_spatial, wl.seed, wl.rank)


def workload_params(wl: Workload, **kw) -> dict:
    return ansatz_params(wl.n_qubits, wl.d_model, wl.n_layers, wl.seed + 100, **kw)
