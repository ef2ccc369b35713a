"""Oracle: the QiankunNet-style ansatz in plain numpy FP64.

TEST INFRASTRUCTURE (see the package docstring).

Sec. 3.1 splits psi(x) = |psi(x)| e^{i phi(x)}: a decoder-only transformer
gives |psi|^2 as a product of conditionals (Eq. auto), an MLP gives phi.
Two qubits (one spatial orbital) form one token (Sec. 3.3) so each
conditional is over 4 values; the number mask of Sec. 3.3 zeroes children
that break the electron counts and the rest is renormalised.

Readings where the paper is silent (listed with the others in the design
notes): GPT-2 style pre-LN decoder layers, FFN width 4d with erf-GELU,
learned positional embeddings, causal attention, final LayerNorm, a d->4
head, LayerNorm eps 1e-5; token value 2*y_beta + y_alpha for spatial orbital
p = n-1-t at position t (reverse qubit order); input sequence = start token
(id 4) followed by the first T-1 tokens; the mask also removes children
from which the remaining orbitals can no longer reach n_alpha / n_beta;
log|psi| = 1/2 sum_t log pi~(x_t | x_<t); phase MLP N -> 512 -> 512 -> 1 with
ReLU on the 0/1 occupations in qubit order.
"""
from __future__ import annotations

import math

import numpy as np

LN_EPS = 1e-5


def dims(params):
    d = params["tok_emb"].shape[1]
    T = params["pos_emb"].shape[0]
    L = 0
    while f"l{L}.ln1.g" in params:
        L += 1
    N = params["phase.w1"].shape[1]
    return d, T, L, N


def tokens(bits):
    """[B, N] occupations -> [B, T] tokens in sampling order."""
    B, N = bits.shape
    n = N // 2
    tok = np.zeros((B, n), dtype=np.int64)
    for t in range(n):
        p = n - 1 - t
        tok[:, t] = bits[:, 2 * p].astype(np.int64) + 2 * bits[:, 2 * p + 1].astype(np.int64)
    return tok


def valid_children(tok, n_alpha, n_beta):
    """[B, T, 4] bool: child v allowed at position t given tokens < t
    (Sec. 3.3 caps plus the reachability floor)."""
    B, T = tok.shape
    ya = tok & 1
    yb = tok >> 1
    ca = np.concatenate([np.zeros((B, 1), np.int64), np.cumsum(ya, axis=1)[:, :-1]], axis=1)
    cb = np.concatenate([np.zeros((B, 1), np.int64), np.cumsum(yb, axis=1)[:, :-1]], axis=1)
    rem = (T - 1 - np.arange(T))[None, :]
    out = np.zeros((B, T, 4), dtype=bool)
    for v in range(4):
        a = ca + (v & 1)
        b = cb + (v >> 1)
        out[:, :, v] = (a <= n_alpha) & (b <= n_beta) & (a + rem >= n_alpha) & (b + rem >= n_beta)
    return out


def _ln_fwd(x, g, b):
    mu = x.mean(axis=-1, keepdims=True)
    xc = x - mu
    var = (xc * xc).mean(axis=-1, keepdims=True)
    rstd = 1.0 / np.sqrt(var + LN_EPS)
    xh = xc * rstd
    return xh * g + b, (xh, rstd)


def _ln_bwd(dy, cache, g):
    xh, rstd = cache
    dg = (dy * xh).reshape(-1, dy.shape[-1]).sum(axis=0)
    db = dy.reshape(-1, dy.shape[-1]).sum(axis=0)
    dxh = dy * g
    dx = rstd * (dxh - dxh.mean(axis=-1, keepdims=True)
                 - xh * (dxh * xh).mean(axis=-1, keepdims=True))
    return dx, dg, db


def _erf(x):
    from scipy.special import erf
    return erf(x)


def _gelu(x):
    return 0.5 * x * (1.0 + _erf(x / math.sqrt(2.0)))


def _gelu_grad(x):
    return 0.5 * (1.0 + _erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def forward(params, bits, n_alpha, n_beta, n_heads, want_cache=False):
    """log|psi| and phi for a batch of occupations ``bits`` [B, N]."""
    P = {k: np.asarray(v, dtype=np.float64) for k, v in params.items()}
    d, T, L, N = dims(P)
    B = bits.shape[0]
    dh = d // n_heads
    tok = tokens(bits)
    inp = np.concatenate([np.full((B, 1), 4, np.int64), tok[:, :-1]], axis=1)
    h = P["tok_emb"][inp] + P["pos_emb"][None, :T, :]
    cache = {"inp": inp, "tok": tok, "layers": []}
    causal = np.tril(np.ones((T, T), dtype=bool))
    for l in range(L):
        p = f"l{l}."
        c = {"h_in": h}
        a, c["ln1"] = _ln_fwd(h, P[p + "ln1.g"], P[p + "ln1.b"])
        c["a"] = a
        qkv = a @ P[p + "attn.wqkv"].T + P[p + "attn.bqkv"]
        q = qkv[..., 0:d].reshape(B, T, n_heads, dh).transpose(0, 2, 1, 3)
        k = qkv[..., d:2 * d].reshape(B, T, n_heads, dh).transpose(0, 2, 1, 3)
        v = qkv[..., 2 * d:3 * d].reshape(B, T, n_heads, dh).transpose(0, 2, 1, 3)
        s = (q @ k.transpose(0, 1, 3, 2)) / math.sqrt(dh)
        s = np.where(causal[None, None], s, -np.inf)
        s = s - s.max(axis=-1, keepdims=True)
        e = np.exp(s)
        pr = e / e.sum(axis=-1, keepdims=True)
        o = (pr @ v).transpose(0, 2, 1, 3).reshape(B, T, d)
        c.update(q=q, k=k, v=v, pr=pr, o=o)
        h = h + o @ P[p + "attn.wo"].T + P[p + "attn.bo"]
        c["h_mid"] = h
        a2, c["ln2"] = _ln_fwd(h, P[p + "ln2.g"], P[p + "ln2.b"])
        c["a2"] = a2
        u = a2 @ P[p + "ffn.w1"].T + P[p + "ffn.b1"]
        gu = _gelu(u)
        c.update(u=u, gu=gu)
        h = h + gu @ P[p + "ffn.w2"].T + P[p + "ffn.b2"]
        cache["layers"].append(c)
    hf, cache["lnf"] = _ln_fwd(h, P["lnf.g"], P["lnf.b"])
    cache["hf"] = hf
    z = hf @ P["head.w"].T + P["head.b"]
    valid = valid_children(tok, n_alpha, n_beta)
    zm = np.where(valid, z, -np.inf)
    zmax = zm.max(axis=-1, keepdims=True)
    lse = zmax + np.log(np.exp(zm - zmax).sum(axis=-1, keepdims=True))
    logp = zm - lse
    sel = np.take_along_axis(logp, tok[..., None], axis=-1)[..., 0]
    la = 0.5 * sel.sum(axis=1)
    cache.update(valid=valid, logp=logp)
    # phase MLP
    x = bits.astype(np.float64)
    z1 = x @ P["phase.w1"].T + P["phase.b1"]
    r1 = np.maximum(z1, 0.0)
    z2 = r1 @ P["phase.w2"].T + P["phase.b2"]
    r2 = np.maximum(z2, 0.0)
    ph = (r2 @ P["phase.w3"].T + P["phase.b3"])[:, 0]
    cache.update(x=x, z1=z1, r1=r1, z2=z2, r2=r2, P=P, n_heads=n_heads)
    if want_cache:
        return la, ph, cache
    return la, ph


def conditionals(params, bits, n_alpha, n_beta, n_heads):
    """pi~(v | x_<t) for every position: [B, T, 4] (masked, renormalised)."""
    _, _, cache = forward(params, bits, n_alpha, n_beta, n_heads, want_cache=True)
    return np.exp(cache["logp"])


def backward(cache, dla, dph):
    """Reverse mode of ``forward``: gradients of sum_b dla_b log|psi_b| +
    dph_b phi_b with respect to every parameter (dict of FP64 arrays)."""
    P = cache["P"]
    nh = cache["n_heads"]
    d, T, L, N = dims(P)
    B = dla.shape[0]
    dh = d // nh
    G = {k: np.zeros_like(v) for k, v in P.items()}
    # phase MLP
    dphc = dph[:, None]
    G["phase.w3"] += dphc.T @ cache["r2"]
    G["phase.b3"] += dphc.sum(axis=0)
    dr2 = dphc @ P["phase.w3"]
    dz2 = dr2 * (cache["z2"] > 0)
    G["phase.w2"] += dz2.T @ cache["r1"]
    G["phase.b2"] += dz2.sum(axis=0)
    dr1 = dz2 @ P["phase.w2"]
    dz1 = dr1 * (cache["z1"] > 0)
    G["phase.w1"] += dz1.T @ cache["x"]
    G["phase.b1"] += dz1.sum(axis=0)
    # masked log-softmax head: d sel_t / d z_{t,u} = [u = tok_t] - pi~_u (valid u)
    tok = cache["tok"]
    pi = np.exp(cache["logp"])
    onehot = np.zeros_like(pi)
    np.put_along_axis(onehot, tok[..., None], 1.0, axis=-1)
    dz = (0.5 * dla)[:, None, None] * (onehot - pi)
    dz = np.where(cache["valid"], dz, 0.0)
    hf = cache["hf"]
    G["head.w"] += np.einsum("btu,btd->ud", dz, hf)
    G["head.b"] += dz.sum(axis=(0, 1))
    dhf = dz @ P["head.w"]
    dh_, G["lnf.g"], G["lnf.b"] = _ln_bwd(dhf, cache["lnf"], P["lnf.g"])
    for l in reversed(range(L)):
        p = f"l{l}."
        c = cache["layers"][l]
        # FFN
        G[p + "ffn.w2"] += np.einsum("btj,bti->ji", dh_, c["gu"])
        G[p + "ffn.b2"] += dh_.sum(axis=(0, 1))
        dgu = dh_ @ P[p + "ffn.w2"]
        du = dgu * _gelu_grad(c["u"])
        G[p + "ffn.w1"] += np.einsum("btj,bti->ji", du, c["a2"])
        G[p + "ffn.b1"] += du.sum(axis=(0, 1))
        da2 = du @ P[p + "ffn.w1"]
        dx, dg, db = _ln_bwd(da2, c["ln2"], P[p + "ln2.g"])
        G[p + "ln2.g"] += dg
        G[p + "ln2.b"] += db
        dh_ = dh_ + dx
        # attention
        G[p + "attn.wo"] += np.einsum("btj,bti->ji", dh_, c["o"])
        G[p + "attn.bo"] += dh_.sum(axis=(0, 1))
        do = (dh_ @ P[p + "attn.wo"]).reshape(B, T, nh, dh).transpose(0, 2, 1, 3)
        pr, q, k, v = c["pr"], c["q"], c["k"], c["v"]
        dv = pr.transpose(0, 1, 3, 2) @ do
        dpr = do @ v.transpose(0, 1, 3, 2)
        ds = pr * (dpr - (dpr * pr).sum(axis=-1, keepdims=True))
        dq = ds @ k / math.sqrt(dh)
        dk = ds.transpose(0, 1, 3, 2) @ q / math.sqrt(dh)
        dqkv = np.concatenate([t.transpose(0, 2, 1, 3).reshape(B, T, d) for t in (dq, dk, dv)],
                              axis=-1)
        G[p + "attn.wqkv"] += np.einsum("btj,bti->ji", dqkv, c["a"])
        G[p + "attn.bqkv"] += dqkv.sum(axis=(0, 1))
        da = dqkv @ P[p + "attn.wqkv"]
        dx, dg, db = _ln_bwd(da, c["ln1"], P[p + "ln1.g"])
        G[p + "ln1.g"] += dg
        G[p + "ln1.b"] += db
        dh_ = dh_ + dx
    # embeddings
    G["pos_emb"] += dh_.sum(axis=0)
    np.add.at(G["tok_emb"], cache["inp"].reshape(-1), dh_.reshape(-1, d))
    return G
