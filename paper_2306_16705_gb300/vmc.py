"""VMC step on the GPU (Sec. 2.1, Fig. serial_flow): batch autoregressive
sampling -> log psi -> sample-aware local energy -> energy statistics ->
gradient -> Adam or AdamW, every stage through the C ABI of libnnqs.so.

``schedule="paper"`` follows the training recipe of Sec. 4.1: the warm-up
learning rate d_model^-0.5 min(i^-0.5, i S_w^-1.5) with S_w = 4000, and a
sample count N_s of 10^5 for the first 100 iterations, then raised towards
10^12.  The paper gives no rate for the rise; here N_s grows tenfold every
100 iterations, and is held at the last value the sampler's unique-prefix
table could take when a larger one overflows it.

``EnergyFunction`` exposes the same estimator as a torch.autograd.Function:
its forward returns Re E and keeps the hand-written gradient
2 Re E_p[(E_loc - E) d ln psi*] (computed by nnqs_energy_grad, E_loc held
fixed) for its backward.
"""
from __future__ import annotations

import torch

from . import binding as B


class EnergyFunction(torch.autograd.Function):
    """E(params) over the given unique samples and counts.  Backward returns
    dE/dparams from the library's reverse mode (no autograd tape)."""

    @staticmethod
    def forward(ctx, params, ham, model, samples, weights, prec):
        stats, el, grad = B.energy_grad(ham, model, params.detach(), samples, weights, prec,
                                        check=True, dtype=params.dtype)
        ctx.save_for_backward(grad)
        ctx.eloc = el
        ctx.stats = stats
        return stats[0].to(params.dtype)

    @staticmethod
    def backward(ctx, grad_out):
        (grad,) = ctx.saved_tensors
        return grad_out * grad, None, None, None, None, None


def sample_seed(seed: int, it: int) -> int:
    """Sampler seed of VMC iteration ``it`` for a run seeded ``seed``: the
    Philox stream of each (run, iteration) pair is distinct."""
    return int(seed) * 1_000_003 + int(it)


def paper_n_samples(it: int, ns0: int = 10 ** 5, ns_max: int = 10 ** 12, first: int = 100,
                    every: int = 100) -> int:
    """N_s of VMC iteration ``it`` (0-based) under the Sec. 4.1 recipe: ns0
    for the first ``first`` iterations, then tenfold every ``every``
    iterations up to ns_max."""
    if it < first:
        return int(ns0)
    return int(min(ns_max, ns0 * 10 ** ((it - first) // every + 1)))


class VMC:
    """Training state: parameters, Adam moments and reusable workspaces.

    optimizer: "adam" or "adamw" (decoupled weight decay ``weight_decay``);
    schedule: None (constant ``lr`` and ``n_samples``) or "paper" (Sec. 4.1
    warm-up learning rate with ``warmup`` steps, and paper_n_samples)."""

    def __init__(self, ham: B.Hamiltonian, model: B.Model, params: torch.Tensor, prec=B.MIXED,
                 n_samples: int = 16384, max_unique: int = 1 << 16, lr: float = 1e-3,
                 betas=(0.9, 0.999), eps: float = 1e-8, seed: int = 0, optimizer: str = "adam",
                 weight_decay: float = 0.01, schedule: str | None = None, warmup: int = 4000,
                 tree_reuse: bool | None = None):
        if optimizer not in ("adam", "adamw") or schedule not in (None, "paper"):
            raise ValueError("optimizer must be adam or adamw, schedule None or paper")
        self.optimizer, self.weight_decay, self.schedule, self.warmup = optimizer, weight_decay, schedule, warmup
        self.ns_hold = None  # largest N_s the unique-prefix table took (paper schedule)
        self.ham, self.model, self.prec = ham, model, prec
        self.params = params.contiguous()
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.t = 0
        self.n_samples, self.max_unique = int(n_samples), int(max_unique)
        # the energy gradient reads the forward's quantities from the tree the
        # sampler decoded (NNQS_SAMPLE_KEEP + nnqs_energy_grad_sampled) where
        # that applies; tree_reuse=False keeps the separate forward
        ok = bool(B.lib().nnqs_energy_grad_sampled_supported(model.handle, prec, self.max_unique))
        if tree_reuse and not ok:
            raise ValueError("tree reuse needs BF16 / split-BF16 arithmetic, d_model 64 and max_unique <= 65536")
        self.tree_reuse = ok if tree_reuse is None else bool(tree_reuse)
        self.lr, self.betas, self.eps = lr, betas, eps
        self.seed = int(seed)
        self._ws_sample = None
        self._ws_grad = None
        self.grad = torch.empty_like(self.params)
        # size both workspaces once for the largest sample set a step can hold
        self._ws_grad_for(self.max_unique)
        self.last_samples = None
        self.last_weights = None
        self.last_stats = None

    def current_lr(self) -> float:
        """Learning rate of the next update."""
        if self.schedule == "paper":
            return B.lr_warmup(self.t + 1, self.model.cfg.d_model, self.warmup)
        return self.lr

    def current_n_samples(self) -> int:
        """N_s of the next step."""
        if self.schedule != "paper":
            return self.n_samples
        ns = paper_n_samples(self.t)
        return ns if self.ns_hold is None else min(ns, self.ns_hold)

    def sample(self, seed=None):
        seed = sample_seed(self.seed, self.t) if seed is None else seed
        flags = B.SAMPLE_KEEP if self.tree_reuse else 0
        nb = B.lib().nnqs_sample_workspace_size(self.model.handle, self.max_unique, self.prec, flags)
        if self._ws_sample is None or self._ws_sample.numel() < nb:
            self._ws_sample = B.workspace(nb, self.params.device)
        ns = self.current_n_samples()
        while True:
            try:
                out = B.sample(self.model, self.params, ns, seed, self.max_unique, self.prec,
                               check=False, ws=self._ws_sample, flags=flags)
            except B.NNQSError as e:
                # paper schedule: hold N_s below the value that overflowed the table
                if self.schedule != "paper" or e.status != B.E_TABLE_FULL or ns <= 1:
                    raise
                ns //= 10
                self.ns_hold = ns
                continue
            return out

    def step(self, check: bool = False, marks=None) -> torch.Tensor:
        """One VMC iteration; returns the device stats tensor [Re E, Im E, Var,
        sum w] (no host synchronisation beyond the sampler's).  ``marks``: a
        list that receives a CUDA event after sampling, after the energy and
        gradient, and after the update (stage timing)."""
        x, w = self.sample()
        if marks is not None:
            marks.append(torch.cuda.Event(enable_timing=True))
            marks[-1].record()
        if self.tree_reuse:
            stats, _, _ = B.energy_grad_sampled(self.ham, self.model, self.params, self._ws_sample, self.max_unique,
                                                x, w, self.prec, check=check, ws=self._ws_grad_for(x.shape[0]),
                                                want_eloc=False, grad_out=self.grad)
        else:
            stats, _, _ = B.energy_grad(self.ham, self.model, self.params, x, w, self.prec,
                                        check=check, ws=self._ws_grad_for(x.shape[0]),
                                        want_eloc=False, grad_out=self.grad)
        if marks is not None:
            marks.append(torch.cuda.Event(enable_timing=True))
            marks[-1].record()
        self.t += 1
        lr = self.lr if self.schedule is None else B.lr_warmup(self.t, self.model.cfg.d_model, self.warmup)
        if self.optimizer == "adamw":
            B.adamw_step(self.params, self.grad, self.m, self.v, self.t, lr, self.betas[0], self.betas[1],
                         self.eps, self.weight_decay)
        else:
            B.adam_step(self.params, self.grad, self.m, self.v, self.t, lr, self.betas[0], self.betas[1],
                        self.eps)
        if marks is not None:
            marks.append(torch.cuda.Event(enable_timing=True))
            marks[-1].record()
        self.last_samples, self.last_weights, self.last_stats = x, w, stats
        return stats

    def _ws_grad_for(self, n):
        nb = B.lib().nnqs_energy_grad_workspace_size(self.ham.handle, self.model.handle, n, self.prec)
        if self._ws_grad is None or self._ws_grad.numel() < nb:
            self._ws_grad = B.workspace(int(nb), self.params.device)
        return self._ws_grad

    def state_dict(self) -> dict:
        return {"params": self.params.detach().cpu(), "m": self.m.cpu(), "v": self.v.cpu(),
                "t": self.t, "seed": self.seed, "ns_hold": self.ns_hold}

    def load_state_dict(self, sd: dict):
        self.params.copy_(sd["params"].to(self.params.device))
        self.m.copy_(sd["m"].to(self.m.device))
        self.v.copy_(sd["v"].to(self.v.device))
        self.t = int(sd["t"])
        self.seed = int(sd["seed"])
        self.ns_hold = sd.get("ns_hold")
