"""Thin Python binding of include/nnqs.h (ctypes).

Argument marshalling only: torch tensors supply device memory and the
current CUDA stream; every step of the computation runs in libnnqs.so.  The
functions keep the C names without the ``nnqs_`` prefix.  Loading fails
loudly when the library has not been built (there is no fallback).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import _build

_lib = None

OK, E_INVAL, E_NOMEM, E_CUDA, E_TABLE_FULL, E_TIMEOUT, E_SECTOR, E_NONFINITE, E_UNSUPPORTED, \
    E_DUPLICATE, E_WORKSPACE = range(11)
SA, EXACT = 0, 1
FP64, MIXED, FP32, BF16X3, FP8 = 0, 1, 2, 3, 4
SWEEP_AUTO, SWEEP_GROUPS, SWEEP_PAIRS, SWEEP_TERMS = 0, 1, 2, 3

_STATUS_NAMES = {0: "NNQS_OK", 1: "NNQS_E_INVAL", 2: "NNQS_E_NOMEM", 3: "NNQS_E_CUDA",
                 4: "NNQS_E_TABLE_FULL", 5: "NNQS_E_TIMEOUT", 6: "NNQS_E_SECTOR",
                 7: "NNQS_E_NONFINITE", 8: "NNQS_E_UNSUPPORTED", 9: "NNQS_E_DUPLICATE",
                 10: "NNQS_E_WORKSPACE"}


class NNQSError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class ModelCfg(ctypes.Structure):
    _fields_ = [("n_qubits", ctypes.c_int32), ("n_alpha", ctypes.c_int32),
                ("n_beta", ctypes.c_int32), ("d_model", ctypes.c_int32),
                ("n_layers", ctypes.c_int32), ("n_heads", ctypes.c_int32),
                ("phase_hidden", ctypes.c_int32), ("reserved", ctypes.c_int32)]


_SIGS = {
    # name: (restype, argtypes)
    "nnqs_last_error": (ctypes.c_char_p, []),
    "nnqs_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "nnqs_version": (ctypes.c_char_p, []),
    "nnqs_workspace_status": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "nnqs_build_pauli": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_void_p]),
    "nnqs_build_pauli_host": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_double, ctypes.c_double, ctypes.c_void_p]),
    "nnqs_ham_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "nnqs_ham_export": (ctypes.c_int, [ctypes.c_void_p] * 5),
    "nnqs_ham_free": (None, [ctypes.c_void_p]),
    "nnqs_ham_build_ungrouped": (ctypes.c_int, [ctypes.c_void_p]),
    "nnqs_ham_layout_bytes": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "nnqs_model_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "nnqs_model_free": (None, [ctypes.c_void_p]),
    "nnqs_model_param_count": (ctypes.c_int64, [ctypes.c_void_p]),
    "nnqs_model_param_offset": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_void_p,
                                               ctypes.c_void_p]),
    "nnqs_logpsi_workspace_size": (ctypes.c_size_t, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int]),
    "nnqs_logpsi": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                   ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                   ctypes.c_void_p]),
    "nnqs_logpsi_backward_workspace_size": (ctypes.c_size_t, [ctypes.c_void_p, ctypes.c_int64,
                                                              ctypes.c_int]),
    "nnqs_logpsi_backward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_int64, ctypes.c_int, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_size_t, ctypes.c_void_p]),
    "nnqs_eloc_workspace_size": (ctypes.c_size_t, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                                   ctypes.c_int64, ctypes.c_int, ctypes.c_int]),
    "nnqs_eloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                 ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "nnqs_eloc_sa_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                            ctypes.c_void_p]),
    "nnqs_exact_coupled_workspace_size": (ctypes.c_size_t, [ctypes.c_void_p, ctypes.c_int64]),
    "nnqs_exact_coupled": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                          ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                          ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_size_t,
                                          ctypes.c_void_p]),
    "nnqs_coupled_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                         ctypes.c_void_p]),
    "nnqs_energy_stats_workspace_size": (ctypes.c_size_t, [ctypes.c_int64]),
    "nnqs_energy_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                         ctypes.c_void_p]),
    "nnqs_energy_grad_workspace_size": (ctypes.c_size_t, [ctypes.c_void_p, ctypes.c_void_p,
                                                          ctypes.c_int64, ctypes.c_int]),
    "nnqs_energy_grad": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                        ctypes.c_void_p]),
    "nnqs_energy_grad_sampled_supported": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64]),
    "nnqs_energy_grad_sampled_workspace_size": (ctypes.c_size_t, [ctypes.c_void_p, ctypes.c_void_p,
                                                                  ctypes.c_int64, ctypes.c_int]),
    "nnqs_energy_grad_sampled": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int64,
                                                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                                ctypes.c_void_p]),
    "nnqs_sample_workspace_size": (ctypes.c_size_t, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                                     ctypes.c_int]),
    "nnqs_sample": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64,
                                   ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                   ctypes.c_void_p]),
    "nnqs_profile_enable": (None, [ctypes.c_int]),
    "nnqs_profile_reset": (None, []),
    "nnqs_profile_read": (ctypes.c_int, [ctypes.c_int, ctypes.c_char_p, ctypes.c_int, ctypes.c_void_p,
                                         ctypes.c_void_p]),
    "nnqs_profile_work": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    "nnqs_launch_count": (ctypes.c_uint64, []),
    "nnqs_measure_peaks_sink_size": (ctypes.c_size_t, []),
    "nnqs_measure_peaks": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "nnqs_adam_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_int64, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_void_p]),
    "nnqs_adamw_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_int64, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_void_p]),
    "nnqs_lr_warmup": (ctypes.c_double, [ctypes.c_int64, ctypes.c_int, ctypes.c_int64]),
}


def lib_path() -> str:
    return _build.LIB


def lib():
    """libnnqs.so, declared.  Raises if it has not been built."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libnnqs.so is not built ({path}); run __graft_entry__.build() "
                               "or python -m paper_2306_16705_gb300._build")
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status):
    if status != OK:
        raise NNQSError(status, lib().nnqs_last_error().decode())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def workspace(nbytes: int, device=None) -> torch.Tensor:
    """A device buffer for the *_workspace_size contract (256-byte aligned)."""
    t = torch.empty(max(int(nbytes), 256) + 256, dtype=torch.uint8, device=device or "cuda")
    off = (-t.data_ptr()) % 256
    return t[off:off + max(int(nbytes), 256)]


def workspace_status(ws: torch.Tensor):
    """Raise NNQSError if a kernel recorded an error in ``ws`` (synchronises)."""
    bad = ctypes.c_int64(-1)
    st = lib().nnqs_workspace_status(_ptr(ws), _stream(), ctypes.byref(bad))
    if st != OK:
        raise NNQSError(st, lib().nnqs_last_error().decode())


def version() -> str:
    return lib().nnqs_version().decode()


# ---------------------------------------------------------------- Hamiltonian
class Hamiltonian:
    """Handle of a grouped Pauli-string Hamiltonian on the current device."""

    def __init__(self, handle):
        self._h = handle

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        buf = (ctypes.c_int64 * 6)()
        _check(lib().nnqs_ham_info(self._h, buf))
        keys = ["n_qubits", "n_words", "n_terms", "n_groups", "max_group", "device_bytes"]
        return dict(zip(keys, list(buf)))

    def build_ungrouped(self):
        """nnqs_ham_build_ungrouped: per-string X/Y masks on the device (for
        the NNQS_SWEEP_TERMS sweep)."""
        _check(lib().nnqs_ham_build_ungrouped(self._h))

    def layout_bytes(self) -> dict:
        """nnqs_ham_layout_bytes: bytes of the grouped and ungrouped layouts."""
        buf = (ctypes.c_int64 * 4)()
        _check(lib().nnqs_ham_layout_bytes(self._h, buf))
        return dict(zip(["grouped", "ungrouped", "grouped_bytewise", "ungrouped_bytewise"], list(buf)))

    def export(self):
        """Host copies (xy[G,W], off[G+1], yz[T,W], coef[T]) of the tables."""
        i = self.info()
        W, G, T = i["n_words"], i["n_groups"], i["n_terms"]
        xy = np.zeros((G, W), dtype=np.uint64)
        off = np.zeros(G + 1, dtype=np.int64)
        yz = np.zeros((T, W), dtype=np.uint64)
        coef = np.zeros(T)
        _check(lib().nnqs_ham_export(self._h, xy.ctypes.data, off.ctypes.data, yz.ctypes.data,
                                     coef.ctypes.data))
        return xy, off, yz, coef

    def coupled(self, x, n_alpha, n_beta):
        """Host: coupled states of one bitstring and H_{x x'} (group order)."""
        i = self.info()
        W = i["n_words"]
        x = np.ascontiguousarray(np.asarray(x, dtype=np.uint64).reshape(W))
        cap = i["n_groups"]
        xp = np.zeros((max(cap, 1), W), dtype=np.uint64)
        hx = np.zeros(max(cap, 1))
        cnt = ctypes.c_int64(0)
        _check(lib().nnqs_coupled_host(self._h, x.ctypes.data, n_alpha, n_beta, xp.ctypes.data,
                                       hx.ctypes.data, cap, ctypes.byref(cnt)))
        return xp[:cnt.value], hx[:cnt.value]

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.nnqs_ham_free(self._h)
            self._h = None


def build_pauli(h, eri, e_core: float = 0.0, drop_tol: float = 1e-12,
                device: bool = True) -> Hamiltonian:
    """nnqs_build_pauli (device=False: nnqs_build_pauli_host) on host
    integrals (numpy)."""
    h = np.ascontiguousarray(h, dtype=np.float64)
    eri = np.ascontiguousarray(eri, dtype=np.float64)
    out = ctypes.c_void_p()
    fn = lib().nnqs_build_pauli if device else lib().nnqs_build_pauli_host
    _check(fn(h.shape[0], h.ctypes.data, eri.ctypes.data, float(e_core), float(drop_tol),
              ctypes.byref(out)))
    return Hamiltonian(out)


# ---------------------------------------------------------------- model
class Model:
    """Handle of the ansatz configuration (parameters stay in torch)."""

    def __init__(self, n_qubits, n_alpha, n_beta, d_model, n_layers, n_heads, phase_hidden=512):
        self.cfg = ModelCfg(n_qubits, n_alpha, n_beta, d_model, n_layers, n_heads, phase_hidden, 0)
        out = ctypes.c_void_p()
        _check(lib().nnqs_model_create(ctypes.byref(self.cfg), ctypes.byref(out)))
        self._h = out
        self.n_qubits, self.n_alpha, self.n_beta = n_qubits, n_alpha, n_beta
        self.n_words = (n_qubits + 63) // 64

    @property
    def handle(self):
        return self._h

    @property
    def n_params(self) -> int:
        return int(lib().nnqs_model_param_count(self._h))

    def offset(self, name):
        off, num = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().nnqs_model_param_offset(self._h, name.encode(), ctypes.byref(off),
                                             ctypes.byref(num)))
        return off.value, num.value

    def pack(self, params: dict, device="cuda") -> torch.Tensor:
        """Named arrays -> the flat FP32 device vector of the ABI layout."""
        flat = np.zeros(self.n_params, dtype=np.float32)
        for name, arr in params.items():
            o, n = self.offset(name)
            a = np.asarray(arr, dtype=np.float32).reshape(-1)
            if a.size != n:
                raise ValueError(f"{name}: {a.size} values, layout wants {n}")
            flat[o:o + n] = a
        return torch.from_numpy(flat).to(device)

    def unpack(self, flat, like: dict) -> dict:
        f = flat.detach().cpu().numpy() if isinstance(flat, torch.Tensor) else np.asarray(flat)
        out = {}
        for name, arr in like.items():
            o, n = self.offset(name)
            out[name] = f[o:o + n].reshape(np.shape(arr))
        return out

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.nnqs_model_free(self._h)
            self._h = None


def logpsi(model: Model, params: torch.Tensor, x: torch.Tensor, prec=FP64, check=True):
    """nnqs_logpsi: [n, 2] float64 (log|psi|, phase)."""
    n = x.shape[0]
    out = torch.empty((n, 2), dtype=torch.float64, device=x.device)
    nb = lib().nnqs_logpsi_workspace_size(model.handle, n, prec)
    ws = workspace(nb, x.device)
    _check(lib().nnqs_logpsi(model.handle, _ptr(params), _ptr(x), n, prec, _ptr(out), _ptr(ws), nb,
                             _stream()))
    if check:
        workspace_status(ws)
    return out


def logpsi_backward(model: Model, params, x, seed, prec=FP64, check=True, dtype=None):
    """nnqs_logpsi_backward: gradient [P] of sum seed . (log|psi|, phase),
    float64 for NNQS_FP64 (unless ``dtype`` says otherwise), else float32."""
    n = x.shape[0]
    dtype = dtype or (torch.float64 if prec == FP64 else torch.float32)
    grad = torch.empty(model.n_params, dtype=dtype, device=params.device)
    g64 = grad if dtype == torch.float64 else None
    g32 = grad if dtype == torch.float32 else None
    nb = lib().nnqs_logpsi_backward_workspace_size(model.handle, n, prec)
    ws = workspace(nb, params.device)
    _check(lib().nnqs_logpsi_backward(model.handle, _ptr(params), _ptr(x), n, prec,
                                      _ptr(seed.contiguous()), _ptr(g64), _ptr(g32), _ptr(ws), nb,
                                      _stream()))
    if check:
        workspace_status(ws)
    return grad


def eloc(ham: Hamiltonian, lut: torch.Tensor, lut_logpsi=None, n_alpha=0, n_beta=0, mode=SA,
         model: Model | None = None, params=None, prec=FP64, flags=SWEEP_AUTO, row_begin=0,
         n_rows=None, check=True, ws=None):
    """nnqs_eloc: [n_rows, 2] float64 local energies of lut[row_begin:...]."""
    n_lut = lut.shape[0]
    if n_rows is None:
        n_rows = n_lut - row_begin
    out = torch.empty((n_rows, 2), dtype=torch.float64, device=lut.device)
    nb = lib().nnqs_eloc_workspace_size(ham.handle, model.handle if model else None, n_lut, n_rows,
                                        mode, prec)
    if ws is None or ws.numel() < nb:
        ws = workspace(nb, lut.device)
    _check(lib().nnqs_eloc(ham.handle, model.handle if model else None, _ptr(params), _ptr(lut),
                           _ptr(lut_logpsi), n_lut, row_begin, n_rows, n_alpha, n_beta, mode, prec,
                           flags, _ptr(out), _ptr(ws), ws.numel(), _stream()))
    if check:
        workspace_status(ws)
    return out


def exact_coupled(ham: Hamiltonian, lut: torch.Tensor, n_alpha, n_beta, row_cap, row_begin=0,
                  n_rows=None, cap_unique=None, check=True):
    """nnqs_exact_coupled: (unique [n_U, W] int64 bits, row_count [n_rows]
    int32, row_idx [n_rows, row_cap] int32, row_hxx [n_rows, row_cap] f64)."""
    n_lut = lut.shape[0]
    W = ham.info()["n_words"]
    if n_rows is None:
        n_rows = n_lut - row_begin
    if cap_unique is None:
        cap_unique = max(1, n_rows * int(row_cap))
    dev = lut.device
    uniq = torch.empty((cap_unique, W), dtype=torch.int64, device=dev)
    cnt = torch.empty(max(n_rows, 1), dtype=torch.int32, device=dev)
    idx = torch.empty((max(n_rows, 1), max(int(row_cap), 1)), dtype=torch.int32, device=dev)
    hxx = torch.empty((max(n_rows, 1), max(int(row_cap), 1)), dtype=torch.float64, device=dev)
    nu = ctypes.c_int64(0)
    nb = lib().nnqs_exact_coupled_workspace_size(ham.handle, n_rows)
    ws = workspace(nb, dev)
    _check(lib().nnqs_exact_coupled(ham.handle, _ptr(lut), n_lut, row_begin, n_rows, n_alpha, n_beta,
                                    _ptr(uniq), cap_unique, ctypes.byref(nu), _ptr(cnt), _ptr(idx),
                                    _ptr(hxx), int(row_cap), _ptr(ws), nb, _stream()))
    if check:
        workspace_status(ws)
    return uniq[:nu.value], cnt[:n_rows], idx[:n_rows], hxx[:n_rows]


def energy_stats(eloc_t: torch.Tensor, weights: torch.Tensor, check=True):
    """nnqs_energy_stats: float64 [4] = Re E, Im E, Var, sum w."""
    n = eloc_t.shape[0]
    stats = torch.empty(4, dtype=torch.float64, device=eloc_t.device)
    nb = lib().nnqs_energy_stats_workspace_size(n)
    ws = workspace(nb, eloc_t.device)
    _check(lib().nnqs_energy_stats(_ptr(eloc_t), _ptr(weights), n, _ptr(stats), _ptr(ws), nb,
                                   _stream()))
    if check:
        workspace_status(ws)
    return stats


def energy_grad(ham: Hamiltonian, model: Model, params, samples, weights, prec=FP64, check=True,
                ws=None, want_eloc=True, dtype=None, grad_out=None):
    """nnqs_energy_grad: (stats[4], eloc[n,2] or None, grad [P]); the gradient
    is float64 for NNQS_FP64 unless ``dtype`` says otherwise."""
    n = samples.shape[0]
    stats = torch.empty(4, dtype=torch.float64, device=samples.device)
    el = torch.empty((n, 2), dtype=torch.float64, device=samples.device) if want_eloc else None
    dtype = dtype or (grad_out.dtype if grad_out is not None else
                      (torch.float64 if prec == FP64 else torch.float32))
    grad = grad_out if grad_out is not None else torch.empty(model.n_params, dtype=dtype,
                                                             device=samples.device)
    g64 = grad if grad.dtype == torch.float64 else None
    g32 = grad if grad.dtype == torch.float32 else None
    nb = lib().nnqs_energy_grad_workspace_size(ham.handle, model.handle, n, prec)
    if ws is None or ws.numel() < nb:
        ws = workspace(nb, samples.device)
    _check(lib().nnqs_energy_grad(ham.handle, model.handle, _ptr(params), _ptr(samples),
                                  _ptr(weights), n, prec, _ptr(stats), _ptr(el), _ptr(g64),
                                  _ptr(g32), _ptr(ws), ws.numel(), _stream()))
    if check:
        workspace_status(ws)
    return stats, el, grad


SAMPLE_RECOMPUTE = 1
SAMPLE_KEEP = 2


def energy_grad_sampled(ham: Hamiltonian, model: Model, params, sample_ws, max_unique: int, samples, weights,
                        prec=BF16X3, check=True, ws=None, want_eloc=True, grad_out=None):
    """nnqs_energy_grad_sampled: energy_grad's outputs, the forward's
    quantities taken from the tree of the last sample(..., flags=SAMPLE_KEEP)
    call with workspace ``sample_ws`` (whose samples and weights these are)."""
    n = samples.shape[0]
    stats = torch.empty(4, dtype=torch.float64, device=samples.device)
    el = torch.empty((n, 2), dtype=torch.float64, device=samples.device) if want_eloc else None
    grad = grad_out if grad_out is not None else torch.empty(model.n_params, dtype=torch.float32,
                                                             device=samples.device)
    g64 = grad if grad.dtype == torch.float64 else None
    g32 = grad if grad.dtype == torch.float32 else None
    nb = lib().nnqs_energy_grad_sampled_workspace_size(ham.handle, model.handle, n, prec)
    if ws is None or ws.numel() < nb:
        ws = workspace(nb, samples.device)
    _check(lib().nnqs_energy_grad_sampled(ham.handle, model.handle, _ptr(params), _ptr(sample_ws),
                                          sample_ws.numel(), int(max_unique), _ptr(samples), _ptr(weights), n,
                                          prec, _ptr(stats), _ptr(el), _ptr(g64), _ptr(g32), _ptr(ws),
                                          ws.numel(), _stream()))
    if check:
        workspace_status(ws)
    return stats, el, grad


def sample(model: Model, params, n_samples: int, seed: int, max_unique: int, prec=FP64,
           check=True, ws=None, flags=0):
    """nnqs_sample: (samples [n_u, W] uint64 as int64 tensor, weights [n_u]).
    With SAMPLE_KEEP in ``flags`` the workspace ``ws`` (allocated by the
    caller for that flag) then holds what energy_grad_sampled reads."""
    W = model.n_words
    dev = params.device
    s = torch.empty((max_unique, W), dtype=torch.int64, device=dev)
    w = torch.empty(max_unique, dtype=torch.int64, device=dev)
    nu = ctypes.c_int64(0)
    nb = lib().nnqs_sample_workspace_size(model.handle, max_unique, prec, flags)
    if ws is None or ws.numel() < nb:
        ws = workspace(nb, dev)
    _check(lib().nnqs_sample(model.handle, _ptr(params), int(n_samples), int(seed), prec, flags,
                             max_unique, _ptr(s), _ptr(w), ctypes.byref(nu), _ptr(ws), ws.numel(),
                             _stream()))
    if check:
        workspace_status(ws)
    return s[:nu.value], w[:nu.value]


def adam_step(params, grad, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """nnqs_adam_step, in place."""
    _check(lib().nnqs_adam_step(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), params.numel(), int(step),
                                float(lr), float(beta1), float(beta2), float(eps), _stream()))


def adamw_step(params, grad, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.01):
    """nnqs_adamw_step, in place."""
    _check(lib().nnqs_adamw_step(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), params.numel(), int(step),
                                 float(lr), float(beta1), float(beta2), float(eps), float(weight_decay),
                                 _stream()))


def lr_warmup(step, d_model, warmup=4000):
    """nnqs_lr_warmup (host)."""
    return lib().nnqs_lr_warmup(int(step), int(d_model), int(warmup))


def to_device_bits(x: np.ndarray, device="cuda") -> torch.Tensor:
    """uint64 [n, W] numpy -> int64 tensor with the same bits."""
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.uint64).view(np.int64)).to(device)


def from_device_bits(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().numpy().view(np.uint64)


def profile_enable(on: bool = True):
    lib().nnqs_profile_enable(1 if on else 0)


def profile_reset():
    lib().nnqs_profile_reset()


def launch_count() -> int:
    return int(lib().nnqs_launch_count())


def measure_peaks(device=None) -> dict:
    """nnqs_measure_peaks: measured XOR+popcount tests/s, 32-bit integer
    ops/s, FP64 and FP32 FMA flop/s of the current device."""
    nb = lib().nnqs_measure_peaks_sink_size()
    sink = workspace(nb, device)
    out = (ctypes.c_double * 4)()
    _check(lib().nnqs_measure_peaks(out, _ptr(sink), nb, _stream()))
    return {"xor_popc64_per_s": out[0], "int32_ops_per_s": out[1], "fp64_flops": out[2],
            "fp32_flops": out[3]}


def profile() -> dict:
    """Per kernel family: launches, total device ms (while enabled), and the
    algorithmic flops / bytes the library attributed to its launches."""
    L = lib()
    n = L.nnqs_profile_read(-1, None, 0, None, None)
    out = {}
    for i in range(n):
        name = ctypes.create_string_buffer(128)
        la = ctypes.c_uint64(0)
        ms = ctypes.c_double(0)
        L.nnqs_profile_read(i, name, 128, ctypes.byref(la), ctypes.byref(ms))
        fl = ctypes.c_double(0)
        by = ctypes.c_double(0)
        L.nnqs_profile_work(i, ctypes.byref(fl), ctypes.byref(by))
        out[name.value.decode()] = {"launches": la.value, "ms": ms.value, "flops": fl.value,
                                    "bytes": by.value}
    return out
