"""Oracle: energy statistics, the gradient estimator, exact enumeration of the
autoregressive distribution, and the Adam update.

TEST INFRASTRUCTURE (see the package docstring).
"""
from __future__ import annotations

import numpy as np

from . import ansatz


def energy_stats(eloc, weights):
    """Eq. (energy) with unique samples: E = sum_i w_i E_loc,i / sum_i w_i
    (complex), Var = sum_i w_i |E_loc,i - E|^2 / sum_i w_i."""
    w = np.asarray(weights, dtype=np.float64)
    e = np.asarray(eloc, dtype=np.complex128)
    sw = w.sum()
    E = (w * e).sum() / sw
    var = (w * np.abs(e - E) ** 2).sum() / sw
    return E, var


def grad_seeds(eloc, weights):
    """Per-sample weights of d log|psi| and d phi in the estimator of Sec. 2.1:
    grad E = 2 Re E_p[(E_loc - E_p[E_loc]) grad ln psi*] with
    ln psi* = log|psi| - i phi, i.e. seeds 2 w Re(E_loc - E)/sum w and
    2 w Im(E_loc - E)/sum w (E the complex weighted mean)."""
    w = np.asarray(weights, dtype=np.float64)
    E, _ = energy_stats(eloc, w)
    dev = np.asarray(eloc) - E
    sw = w.sum()
    return 2.0 * w * dev.real / sw, 2.0 * w * dev.imag / sw


def energy_grad(params, bits, eloc, weights, n_alpha, n_beta, n_heads):
    """Gradient estimator of Sec. 2.1 with E_loc held fixed: dict of FP64
    arrays keyed like ``params``."""
    dla, dph = grad_seeds(eloc, weights)
    _, _, cache = ansatz.forward(params, bits, n_alpha, n_beta, n_heads, want_cache=True)
    return ansatz.backward(cache, dla, dph)


def exact_distribution(params, sector_bits, n_alpha, n_beta, n_heads):
    """p(x) = |psi(x)|^2 over every sector state (Eq. auto), FP64."""
    la, _ = ansatz.forward(params, sector_bits, n_alpha, n_beta, n_heads)
    return np.exp(2.0 * la)


def adamw_step(theta, grad, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.01):
    """One AdamW update (Loshchilov & Hutter 2019, decoupled weight decay), the
    optimiser of Sec. 4.1: shrink theta by (1 - lr * weight_decay), then take
    the Adam step below with the same moments."""
    return adam_step((1.0 - lr * weight_decay) * theta, grad, m, v, step, lr, beta1, beta2, eps)


def lr_warmup(step, d_model, warmup=4000):
    """Learning rate of training step ``step`` (1-based), Sec. 4.1:
    d_model^-1/2 * min(step^-1/2, step * warmup^-3/2)."""
    return d_model ** -0.5 * min(step ** -0.5, step * warmup ** -1.5)


def adam_step(theta, grad, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1), no weight decay.
    ``step`` is the 1-based step count after this update."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
