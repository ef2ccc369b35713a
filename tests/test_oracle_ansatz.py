"""Pins of the oracle ansatz: an independent torch.nn.functional build of the
same network (library LayerNorm, scaled-dot-product attention, GELU,
log-softmax), torch autograd and central finite differences for the
hand-written reverse mode, normalisation over the sector (Eq. auto with the
renormalised mask of Sec. 3.3), causality, and the mask's brute-force
reachability meaning."""
import math

import numpy as np
import pytest
import torch
import torch.nn.functional as F

from oracle import ansatz as OA
from oracle import hamiltonian as OH
from paper_2306_16705_gb300 import inputs as I


def torch_reference(params, bits, n_alpha, n_beta, n_heads):
    """The same ansatz from torch library layers, FP64, differentiable."""
    P = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True) for k, v in params.items()}
    d = P["tok_emb"].shape[1]
    T = P["pos_emb"].shape[0]
    L = sum(1 for k in P if k.endswith("ln1.g"))
    B, N = bits.shape
    n = N // 2
    b = torch.tensor(bits.astype(np.int64))
    order = [n - 1 - t for t in range(n)]
    tok = torch.stack([b[:, 2 * p] + 2 * b[:, 2 * p + 1] for p in order], dim=1)
    inp = torch.cat([torch.full((B, 1), 4, dtype=torch.int64), tok[:, :-1]], dim=1)
    x = F.embedding(inp, P["tok_emb"]) + P["pos_emb"][None]
    for l in range(L):
        p = f"l{l}."
        a = F.layer_norm(x, (d,), P[p + "ln1.g"], P[p + "ln1.b"], eps=1e-5)
        qkv = F.linear(a, P[p + "attn.wqkv"], P[p + "attn.bqkv"])
        q, k, v = qkv.split(d, dim=-1)
        sh = lambda t: t.reshape(B, T, n_heads, d // n_heads).transpose(1, 2)
        o = F.scaled_dot_product_attention(sh(q), sh(k), sh(v), is_causal=True)
        x = x + F.linear(o.transpose(1, 2).reshape(B, T, d), P[p + "attn.wo"], P[p + "attn.bo"])
        a2 = F.layer_norm(x, (d,), P[p + "ln2.g"], P[p + "ln2.b"], eps=1e-5)
        x = x + F.linear(F.gelu(F.linear(a2, P[p + "ffn.w1"], P[p + "ffn.b1"])),
                         P[p + "ffn.w2"], P[p + "ffn.b2"])
    x = F.layer_norm(x, (d,), P["lnf.g"], P["lnf.b"], eps=1e-5)
    z = F.linear(x, P["head.w"], P["head.b"])
    # mask: child (ya, yb) allowed iff counts stay <= n and can still reach n
    ya, yb = tok & 1, tok >> 1
    ca = torch.cumsum(ya, 1) - ya
    cb = torch.cumsum(yb, 1) - yb
    rem = (T - 1 - torch.arange(T))[None]
    allowed = []
    for c in range(4):
        aa, bb = ca + (c & 1), cb + (c >> 1)
        allowed.append((aa <= n_alpha) & (bb <= n_beta) & (aa + rem >= n_alpha)
                       & (bb + rem >= n_beta))
    allowed = torch.stack(allowed, -1)
    lp = torch.log_softmax(z.masked_fill(~allowed, float("-inf")), dim=-1)
    la = 0.5 * lp.gather(-1, tok[..., None])[..., 0].sum(1)
    xf = b.to(torch.float64)
    r = F.relu(F.linear(xf, P["phase.w1"], P["phase.b1"]))
    r = F.relu(F.linear(r, P["phase.w2"], P["phase.b2"]))
    ph = F.linear(r, P["phase.w3"], P["phase.b3"])[:, 0]
    return la, ph, P


def _model(n_qubits=12, d=32, L=2, seed=3):
    return I.ansatz_params(n_qubits, d, L, seed, std=0.3, bias_std=0.1, phase_std=0.2)


def test_forward_matches_torch_library_build():
    wl = I.WORKLOADS["n12"]
    params = _model()
    bits = I.unpack_bits(I.sector_states(6, 3, 3), 12)
    la, ph = OA.forward(params, bits, 3, 3, 4)
    tla, tph, _ = torch_reference(params, bits, 3, 3, 4)
    assert np.abs(la - tla.detach().numpy()).max() < 1e-12
    assert np.abs(ph - tph.detach().numpy()).max() < 1e-12


def test_backward_matches_torch_autograd():
    params = _model(n_qubits=10, d=16, L=2, seed=5)
    bits = I.unpack_bits(I.random_sector_samples(5, 2, 3, 30, seed=1), 10)
    rng = np.random.default_rng(0)
    dla, dph = rng.normal(size=30), rng.normal(size=30)
    _, _, cache = OA.forward(params, bits, 2, 3, 4, want_cache=True)
    G = OA.backward(cache, dla, dph)
    tla, tph, P = torch_reference(params, bits, 2, 3, 4)
    (torch.tensor(dla) @ tla + torch.tensor(dph) @ tph).backward()
    for k in params:
        ref = P[k].grad.numpy()
        assert np.abs(G[k] - ref).max() <= 1e-10 * max(1.0, np.abs(ref).max()), k


def test_backward_matches_finite_differences():
    params = _model(n_qubits=8, d=8, L=1, seed=7)
    bits = I.unpack_bits(I.random_sector_samples(4, 2, 2, 12, seed=2), 8)
    rng = np.random.default_rng(1)
    dla, dph = rng.normal(size=12), rng.normal(size=12)
    _, _, cache = OA.forward(params, bits, 2, 2, 2, want_cache=True)
    G = OA.backward(cache, dla, dph)

    def f(pp):
        la, ph = OA.forward(pp, bits, 2, 2, 2)
        return dla @ la + dph @ ph

    for k in ["tok_emb", "l0.attn.wqkv", "l0.ln1.g", "l0.ffn.w1", "lnf.b", "head.w",
              "phase.w1", "phase.b3", "pos_emb"]:
        flat = params[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(3, flat.size), replace=False):
            pp = {kk: vv.astype(np.float64).copy() for kk, vv in params.items()}
            hstep = 1e-5
            pp[k].reshape(-1)[idx] += hstep
            fp = f(pp)
            pp[k].reshape(-1)[idx] -= 2 * hstep
            fm = f(pp)
            fd = (fp - fm) / (2 * hstep)
            assert abs(fd - G[k].reshape(-1)[idx]) < 1e-6 * max(1.0, abs(fd)), (k, idx)


@pytest.mark.parametrize("n,na,nb", [(6, 3, 3), (5, 2, 1), (4, 0, 2)])
def test_normalised_over_sector(n, na, nb):
    params = I.ansatz_params(2 * n, 16, 2, 9, std=0.5, bias_std=0.2)
    bits = I.unpack_bits(I.sector_states(n, na, nb), 2 * n)
    la, _ = OA.forward(params, bits, na, nb, 4)
    assert abs(np.exp(2 * la).sum() - 1.0) < 1e-12


def test_causality():
    params = _model()
    S = I.sector_states(6, 3, 3)
    bits = I.unpack_bits(S, 12)
    cond = OA.conditionals(params, bits, 3, 3, 4)
    tok = OA.tokens(bits)
    # states sharing the first k tokens share the first k+1 conditionals
    for k in range(1, 5):
        groups = {}
        for i in range(len(S)):
            groups.setdefault(tuple(tok[i, :k]), []).append(i)
        for members in groups.values():
            ref = cond[members[0], :k + 1]
            for m in members[1:]:
                assert np.abs(cond[m, :k + 1] - ref).max() < 1e-13


def test_mask_is_reachability():
    """A child is allowed exactly when some completion lands in the sector."""
    n, na, nb = 4, 2, 1
    S = I.sector_states(n, na, nb)
    tok = OA.tokens(I.unpack_bits(S, 2 * n))
    prefixes = {tuple(r[:k]) for r in tok for k in range(n + 1)}
    # walk every prefix of every possible token string
    import itertools
    for k in range(n):
        for pref in itertools.product(range(4), repeat=k):
            if tuple(pref) not in prefixes:
                continue
            arr = np.array([list(pref) + [0] * (n - k)])
            allowed = OA.valid_children(arr, na, nb)[0, k]
            for v in range(4):
                assert allowed[v] == (tuple(pref) + (v,) in prefixes)
