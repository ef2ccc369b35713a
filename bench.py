#!/usr/bin/env python
"""Benchmark of one VMC step of the NNQS-Transformer method on the GPU.

A step (every row of the hot path): batch autoregressive sampling of
N_s = 16384 samples from the transformer ansatz, log psi of the unique
samples, sample-aware local energy over the merged Pauli-string Hamiltonian
(Alg. 2), energy statistics, the gradient estimator's reverse mode, and an
Adam update.  Workload: 40 spin orbitals, 20 electrons, dense random
integrals (seed 1, rank 16; 233,001 Pauli strings in 46,171 X/Y groups),
transformer d_model 64, 4 layers, 8 heads, phase MLP 40x512x512x1,
random-init parameters (std 0.02).

Metric: logical (sample x Pauli-term) local-energy evaluations per second of
the whole step, N_u * N_h / step time; ms_per_step is the VMC step time.
The plain FP64 path's step time is reported beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "n40"
N_SAMPLES = 16384
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12  # CUDA-core FMA: SMs x lanes x 2 x max clock
# the tcgen05 kernels of the ansatz (forward, fused reverse mode, sampler decode, the remaining GEMMs)
TENSOR_KERNELS = ("k_fwd_fused", "k_bwd_attn", "k_bwd_ffn", "k_decode_step", "k_tc_gemm")
# DRAM read + write bytes per launch of this step's kernels, from ncu captures of the current kernels; a
# kernel leaves this table when it changes.  The reverse-mode halves: one launch each at 16,384 samples of
# 20 tokens (profiles/k_bwd_fused_energy_grad_n40.md); k_decode_step: the mean over the 20 launches of one
# sampling of this workload, 0.9 MB at the first token step to 477 MB at the last
# (profiles/k_decode_step_sample_n40.md).
KERNEL_TRAFFIC_BYTES = {"k_bwd_ffn": 167.9e6 + 50.0e6, "k_bwd_attn": 167.9e6 + 48.1e6, "k_decode_step": 155.9e6}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="bf16x3", choices=["bf16x3", "mixed", "fp32", "fp64", "fp8"])
    ap.add_argument("--fp64-steps", type=int, default=2, help="steps of the plain FP64 path (0 = skip)")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=-1, help="end-to-end steps (default steps/2, min 2)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n-samples", type=int, default=N_SAMPLES, help="N_s per step (smaller for profiling)")
    ap.add_argument("--no-layouts", action="store_true", help="skip the grouped/ungrouped layout comparison")
    ap.add_argument("--no-peaks", action="store_true", help="skip the integer / FP64 / FP32 pipe measurements")
    ap.add_argument("--exact-rows", type=int, default=1024,
                    help="rows of the exact-mode side line (0 = skip)")
    ap.add_argument("--n120-steps", type=int, default=3, help="timed steps of the 120-qubit side line (0 = skip)")
    ap.add_argument("--case", default=None,
                    choices=["sweep-pairs", "sweep-groups", "sweep-pairs-sampled", "sweep-groups-sampled", "logpsi",
                             "logpsi-unfused", "grad", "grad-unfused", "eloc-exact"],
                    help="time one hot-path call alone (for profiling) instead of the VMC step")
    ap.add_argument("--workload", default=WORKLOAD, help="workload of --case (n40, n76, n120, n30, n12)")
    ap.add_argument("--n", type=int, default=16384, help="samples (table rows) of --case")
    ap.add_argument("--rows", type=int, default=0, help="rows of --case sweeps / exact mode (0 = all)")
    ap.add_argument("--ladder", action="store_true",
                    help="add the local-energy speed-up ladder (Sec. 4.3) to the CPU baseline (about a minute)")
    return ap.parse_args()


# ---------------------------------------------------------------- clocks
class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int, enabled: bool):
        self.index, self.enabled, self.proc, self.lines = index, enabled, None, []

    def __enter__(self):
        if self.enabled:
            try:
                self.proc = subprocess.Popen(
                    ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                     "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
                self.thread = threading.Thread(target=self._read, daemon=True)
                self.thread.start()
            except OSError:
                self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- reference arm / CPU baseline
class OracleStep:
    """Times the CPU oracle on a bounded sample of the workload.  A step is
    log psi (numpy FP64) of ``n_fwd`` samples, the sample-aware local energy
    (plain C, OpenMP over rows) of ``n_rows`` rows against the full
    N_u-sample table, and the reverse mode for those rows; the step time is
    extrapolated linearly to N_u samples.  The oracle has no sampler (it
    enumerates p exactly on small systems): the table is a uniform draw of
    N_u sector states, the distribution a random-init ansatz gives, with a
    stand-in log psi table (its values do not change the cost)."""

    def __init__(self, wl):
        from oracle import hamiltonian as OH
        from paper_2306_16705_gb300 import inputs as I

        self.wl = wl
        h, eri = I.workload_integrals(wl)
        self.strings = OH.build(h, eri)
        self.n_terms = len(self.strings[2])
        self.n_groups = len({tuple(r) for r in self.strings[0].tolist()})
        self.S = I.random_sector_samples(wl.n_spatial, wl.n_alpha, wl.n_beta, N_SAMPLES, seed=wl.seed)
        self.lp = I.random_logpsi(N_SAMPLES, seed=wl.seed, amp_std=0.1)
        self.params = I.workload_params(wl)

    def run(self, n_fwd: int, n_rows: int):
        from oracle import ansatz as OA
        from oracle import hamiltonian as OH
        from oracle import vmc as OV
        from paper_2306_16705_gb300 import inputs as I

        wl = self.wl
        rows = self.S[:n_rows]
        t0 = time.perf_counter()
        OA.forward(self.params, I.unpack_bits(self.S[:n_fwd], wl.n_qubits), wl.n_alpha, wl.n_beta, wl.n_heads)
        t1 = time.perf_counter()
        el = OH.eloc_lut(*self.strings, self.S, self.lp, rows, wl.n_alpha, wl.n_beta)
        OV.energy_grad(self.params, I.unpack_bits(rows, wl.n_qubits), el, np.ones(n_rows), wl.n_alpha, wl.n_beta,
                       wl.n_heads)
        t2 = time.perf_counter()
        step_s = (t1 - t0) / n_fwd * N_SAMPLES + (t2 - t1) / n_rows * N_SAMPLES
        return {"step_s": step_s, "sampled_s": t2 - t0, "rows_s": t2 - t1, "n_rows": n_rows, "n_terms": self.n_terms,
                "pairs_per_s": N_SAMPLES * self.n_terms / step_s,
                "sample": f"log psi of {n_fwd} and local energy + reverse mode of {n_rows} of the {N_SAMPLES} "
                          f"samples (table of all {N_SAMPLES}); step time extrapolated linearly to "
                          f"{N_SAMPLES}; no sampler"}


def sized_oracle_run(bench: "OracleStep", target_s: float):
    """bench.run with the row sample grown (from 48 rows) until the timed
    oracle work takes about target_s seconds (at most 4,096 rows)."""
    first = bench.run(512, 48)
    if first["sampled_s"] >= 0.8 * target_s:
        return first
    rows_budget = target_s - (first["sampled_s"] - first["rows_s"])
    n_rows = int(48 * rows_budget / max(first["rows_s"], 1e-3))
    n_rows = max(48, min(4096, n_rows // 16 * 16))  # at most 4,096 rows: a few GB of oracle activations
    return bench.run(512, n_rows)


# The speed-up ladder of Sec. 4.3 (Fig. speedup-eloc) on molecule-shaped
# synthetic systems: 20, 28 and 38 spin orbitals with 12, 20 and 24 electrons
# (the STO-3G sizes of C2, LiCl and C2H4O) and the paper's unique-sample
# counts; random integrals (rank 8), N_u uniform sector draws, a stand-in
# log psi table.
LADDER = (("n20", 10, 6, 6, 10553, 5), ("n28", 14, 10, 10, 9271, 6), ("n38", 19, 12, 12, 25622, 7))


def run_ladder(budget_s: float = 2.0):
    """E_loc of every sample of S by the three CPU rungs (oracle/ladder.c,
    OpenMP over rows on all host cores) and by the library's sample-aware
    sweep on the GPU.  A CPU rung is timed on the first k rows, k a multiple
    of the core count grown until the call takes budget_s, and extrapolated
    linearly to N_u rows; the GPU rung runs all N_u rows (CUDA events, best
    of 3 batches of 5 calls after 0.3 s of warm-up calls).  The GPU values are checked against the +LUT
    rung's on the timed rows."""
    import torch
    from oracle import hamiltonian as OH
    from oracle import ladder as OL
    from paper_2306_16705_gb300 import binding as B
    from paper_2306_16705_gb300 import inputs as I

    nc = cores()
    out = {}
    for name, n, na, nb, nu, seed in LADDER:
        N = 2 * n
        h, eri = I.integrals(n, seed, 8)
        gxy, goff, gyz, gcoef = OH.group(*OH.build(h, eri))
        S = I.random_sector_samples(n, na, nb, nu, seed=seed)
        lp = I.random_logpsi(nu, seed=seed, amp_std=0.1)
        table = OL.tuple_table(S, lp, N)
        secs, rows_timed, vals = {}, {}, {}
        for rung in OL.RUNGS:
            k = min(nu, nc)
            while True:
                t0 = time.perf_counter()
                v = OL.eloc(rung, N, gxy, goff, gyz, gcoef, S, lp, S[:k], table)
                dt = time.perf_counter() - t0
                if dt >= budget_s or k >= nu:
                    break
                grow = max(2, int(budget_s / max(dt, 1e-4)))
                k = min(nu, (k * grow + nc - 1) // nc * nc)
            secs[rung], rows_timed[rung], vals[rung] = dt * nu / k, k, v
        ham = B.build_pauli(h, eri)
        Sd = B.to_device_bits(S)
        lpd = torch.from_numpy(np.ascontiguousarray(lp)).cuda()
        got = B.eloc(ham, Sd, lpd, na, nb)
        # the GPU sat idle during the CPU rungs: run it for ~0.3 s so the
        # clocks are up, then take the best of 3 batches of 5 calls
        t_end = time.perf_counter() + 0.3
        while time.perf_counter() < t_end:
            B.eloc(ham, Sd, lpd, na, nb, check=False)
            torch.cuda.synchronize()
        st = torch.cuda.current_stream()
        best = float("inf")
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(5):
                got = B.eloc(ham, Sd, lpd, na, nb, check=False)
            e1.record(st)
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1) / 5 / 1e3)
        secs["gpu"] = best
        g = got.cpu().numpy()
        k = rows_timed["lut"]
        ref = vals["lut"]
        diff = float(np.max(np.abs((g[:k, 0] + 1j * g[:k, 1]) - ref)) / max(1.0, float(np.abs(ref).max())))
        out[name] = {
            "n_qubits": N, "electrons": na + nb, "n_u": nu, "n_terms": int(len(gcoef)), "n_groups": int(len(gxy)),
            "seconds": secs, "speedup_vs_bare": {r: secs["bare"] / secs[r] for r in secs},
            "cpu_rows_timed": rows_timed, "gpu_vs_lut_max_scaled_diff": diff}
    return {"cores": nc, "note": "CPU rungs: OpenMP over rows, timed on the first k rows and extrapolated to "
                                  "N_u; GPU: the whole N_u rows", "systems": out}


def cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def workload_config(n_terms, n_groups, n_samples, n_u_mean, world):
    """The config object of the benchmark line (both arms)."""
    return {"workload": f"n40: 40 spin orbitals, 20 electrons, N_s={n_samples}, d=64 L=4 H=8, "
                        f"{n_terms} Pauli strings / {n_groups} groups",
            "n_terms": n_terms, "n_groups": n_groups, "n_u_mean": n_u_mean,
            "parallelism": "replicas" if world > 1 else "1 GPU",
            "l2": "flushed between steps (256 MB memset)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_2306_16705_gb300 import inputs as I

    oracle.build()
    wl = I.WORKLOADS[WORKLOAD]
    bench = OracleStep(wl)
    for _ in range(max(0, min(args.warmup, 1))):
        bench.run(64, 8)
    # each step a bounded sample: about 10 s of oracle work, less when many
    # steps are asked for, so that the run stays within a few minutes
    target_s = max(1.0, min(10.0, 150.0 / max(1, args.steps)))
    ts, sampled = [], []
    last = None
    for _ in range(args.steps):
        last = sized_oracle_run(bench, target_s) if last is None else bench.run(512, last["n_rows"])
        ts.append(last["step_s"])
        sampled.append(last["sampled_s"])
    step_s = float(np.mean(ts))
    value = N_SAMPLES * last["n_terms"] / step_s
    unit = "pairs/s"
    # ms_per_step is the wall time of each step's bounded sample (what this
    # run spent); value is the whole step's rate measured on that sample
    line = {
        "impl": "reference", "metric": "local-energy (sample x Pauli-term) evals/sec, whole VMC step",
        "value": value, "unit": unit, "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": float(np.mean(sampled)) * 1e3, "extrapolated_ms_per_step": step_s * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": workload_config(last["n_terms"], bench.n_groups, N_SAMPLES, float(N_SAMPLES), 1),
        "cpu_baseline": {"value": value, "unit": unit, "cores": cores(), "kind": "oracle",
                         "sample": last["sample"] + "; ms_per_step = the sample's wall time, "
                                   "extrapolated_ms_per_step = the whole step's"},
        "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)



def model_flops_per_sample(wl) -> float:
    """Method FLOPs of one ansatz forward (Sec. 3.1): the decoder layers'
    four products (q|k|v, out-projection, FFN in and out), causal attention
    (scores and weighted sum), the head and the phase MLP."""
    T, d, L, H = wl.n_qubits // 2, wl.d_model, wl.n_layers, wl.n_heads
    F, P, N = 4 * d, 512, wl.n_qubits
    layers = 2.0 * T * L * (4 * d * d + 2 * d * F)
    attn = 2.0 * L * H * (T * (T + 1) / 2) * (d // H) * 2
    return layers + attn + 2.0 * T * d * 4 + 2.0 * (N * P + P * P + P)


def sweep_roofline(prof: dict, peaks: dict, W: int) -> dict | None:
    """Roofline of the sample-aware sweep (Alg. 2) against the measured
    XOR+popcount rate: a pair-sweep test is W XOR+popcount tests, a group-sweep
    test 2W (one per spin), a string-sweep test 5W."""
    per = {"k_sweep_pairs": W, "k_sweep_groups": 2 * W, "k_sweep_terms": 5 * W}
    fams = [(k, prof[k]) for k in per if k in prof and prof[k]["ms"] > 0]
    if not fams or not peaks.get("xor_popc64_per_s"):
        return None
    k, f = max(fams, key=lambda kv: kv[1]["ms"])
    tests = f["flops"]  # the launch sites count (row, group / sample / string) tests
    rate = tests * per[k] / (f["ms"] / 1e3)
    return {"kernel": k, "bound": "alu", "achieved": rate, "peak": peaks["xor_popc64_per_s"],
            "unit": "xor+popc64/s", "frac": rate / peaks["xor_popc64_per_s"],
            "tests_per_launch": tests / max(1, f["launches"]), "popc_per_test": per[k],
            "launches": f["launches"], "avg_launch_ms": f["ms"] / max(1, f["launches"]),
            "hbm_gbs": f["bytes"] / (f["ms"] / 1e3) / 1e9,
            "peak_source": "nnqs_measure_peaks (measured in this run)"}


def run_exact_side_line(ham, model, wl, params, x, prec, n_rows, peaks, tflops_peak):
    """Exact-mode local energy (Eq. Eloc over every coupled x', Sec. 3.4 (2))
    of the first n_rows samples of a step: coupled-set expansion and dedup,
    the tensor-core ansatz forward over the unique coupled states, the fused
    sweep.  Also 64 rows through the plain FP64 path for the error."""
    import torch

    from paper_2306_16705_gb300 import binding as B

    rows = x[:n_rows].contiguous()
    # |U|: the deduplicated coupled set the call below builds
    Ud, cnt, _, _ = B.exact_coupled(ham, rows, wl.n_alpha, wl.n_beta, row_cap=16384)
    n_u = int(Ud.shape[0])
    n_x = int(cnt.sum().item())
    del Ud
    B.eloc(ham, rows[:32], None, wl.n_alpha, wl.n_beta, mode=B.EXACT, model=model, params=params, prec=prec)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    # the call timed alone (CUDA events on the stream), then once more with
    # every launch bracketed by events for the per-kernel split
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    got = B.eloc(ham, rows, None, wl.n_alpha, wl.n_beta, mode=B.EXACT, model=model, params=params, prec=prec)
    e1.record(st)
    e1.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    B.profile_reset()
    B.profile_enable(True)
    B.eloc(ham, rows, None, wl.n_alpha, wl.n_beta, mode=B.EXACT, model=model, params=params, prec=prec)
    torch.cuda.synchronize()
    prof = B.profile()
    B.profile_enable(False)
    prof_ms = sum(v["ms"] for v in prof.values())
    ansatz_ms = sum(v["ms"] for k, v in prof.items()
                    if k not in ("k_insert_rows", "k_expand", "k_compact", "k_diag", "k_sweep_exact",
                                 "k_reduce_partials"))
    # the ansatz's share of the profiled call, applied to the call timed alone
    ansatz_ms = ansatz_ms / max(prof_ms, 1e-9) * t * 1e3
    fl = model_flops_per_sample(wl) * n_u
    tc = prof.get("k_fwd_fused") or prof.get("k_tc_gemm") or {"flops": 0.0, "ms": 0.0}
    info = ham.info()
    e64 = B.eloc(ham, rows[:64], None, wl.n_alpha, wl.n_beta, mode=B.EXACT, model=model, params=params,
                 prec=B.FP64)
    d = (got[:64] - e64).abs().max().item()
    return {
        "rows": n_rows, "unique_coupled_states": n_u, "coupled_pairs": n_x, "ms": t * 1e3,
        "coupled_states_per_s": n_u / t, "coupled_pairs_per_s": n_x / t,
        "logical_pairs_per_s": n_rows * info["n_terms"] / t,
        "ansatz_ms": ansatz_ms, "ansatz_model_tflops": fl / (ansatz_ms / 1e3) / 1e12,
        "ansatz_frac_of_burst_bf16": fl / (ansatz_ms / 1e3) / 1e12 / tflops_peak,
        "transformer_kernel_tflops": tc["flops"] / (tc["ms"] / 1e3) / 1e12 if tc["ms"] else None,
        "stage_ms": {k: round(v["ms"], 3) for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])[:8]},
        "max_abs_diff_vs_fp64_first64": d,
        "max_rel_diff_vs_fp64_first64": d / max(1.0, e64.abs().max().item()),
        "note": "prec " + {B.BF16X3: "bf16x3", B.MIXED: "mixed", B.FP32: "fp32", B.FP64: "fp64", B.FP8: "fp8"}[prec] +
                "; ms = the call timed alone; forward FLOPs = unique coupled states x method FLOPs per sample; "
                "stage_ms and ansatz share from a second, per-launch-profiled call"}


def run_n120_side_line(steps, warmup, peaks, clocks_on, local):
    """The 120-qubit, 40-electron workload (seed 3, rank 32; 19,233,001
    strings in 4,111,711 groups; d=128, 6 layers, 8 heads), shaped like the
    benzene 6-31G run of Sec. 4.4: a VMC step samples N_s = 131,072 from the
    random-init ansatz, replaces the counts by Zipf(1.2) weights, runs the
    energy gradient in BF16X3 (local energy by the pair sweep, reverse mode
    over recomputed activation chunks) and an Adam update."""
    import torch

    from paper_2306_16705_gb300 import binding as B
    from paper_2306_16705_gb300 import inputs as I

    wl = I.WORKLOADS["n120"]
    h, eri = I.workload_integrals(wl)
    t0 = time.perf_counter()
    ham = B.build_pauli(h, eri)
    build_s = time.perf_counter() - t0
    info = ham.info()
    model = B.Model(wl.n_qubits, wl.n_alpha, wl.n_beta, wl.d_model, wl.n_layers, wl.n_heads)
    p0 = model.pack(I.workload_params(wl))
    params = p0.clone()
    m, v = torch.zeros_like(params), torch.zeros_like(params)
    grad = torch.empty_like(params)
    ns = 131072
    zipf = torch.from_numpy(I.zipf_counts(ns, 1.2, seed=3).astype(np.int64)).cuda()
    nb = B.lib().nnqs_sample_workspace_size(model.handle, ns, B.BF16X3, 0)
    ws_s = B.workspace(nb)
    ws_g = B.workspace(B.lib().nnqs_energy_grad_workspace_size(ham.handle, model.handle, ns, B.BF16X3))
    st = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def step(i, marks):
        x, w = B.sample(model, params, ns, seed=5000 + i, max_unique=ns, prec=B.BF16X3, check=False, ws=ws_s)
        marks[1].record(st)
        stats, _, _ = B.energy_grad(ham, model, params, x, zipf[:x.shape[0]], B.BF16X3, check=False, ws=ws_g,
                                    want_eloc=False, grad_out=grad)
        marks[2].record(st)
        B.adam_step(params, grad, m, v, 1, lr=1e-3)
        return x.shape[0], stats

    for i in range(warmup):
        params.copy_(p0)
        step(i, [torch.cuda.Event(enable_timing=True) for _ in range(3)])
    torch.cuda.synchronize()
    ts, stages, nus = [], {"sample": 0.0, "energy_grad": 0.0, "adam": 0.0}, []
    with Clocks(local, clocks_on) as clk:
        for i in range(steps):
            params.copy_(p0)
            m.zero_()
            v.zero_()
            flush.zero_()
            mk = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            mk[0].record(st)
            nu, stats = step(i, mk)
            mk[3].record(st)
            mk[3].synchronize()
            ts.append(mk[0].elapsed_time(mk[3]))
            stages["sample"] += mk[0].elapsed_time(mk[1])
            stages["energy_grad"] += mk[1].elapsed_time(mk[2])
            stages["adam"] += mk[2].elapsed_time(mk[3])
            nus.append(nu)
    # one more step with every launch timed, for the per-kernel split
    torch.cuda.synchronize()
    B.profile_reset()
    B.profile_enable(True)
    params.copy_(p0)
    step(steps, [torch.cuda.Event(enable_timing=True) for _ in range(3)])
    prof = B.profile()
    B.profile_enable(False)
    ms = float(np.mean(ts))
    nu = float(np.mean(nus))
    out = {
        "workload": "n120: 120 spin orbitals, 40 electrons, N_s=131072 (Zipf s=1.2 weights), d=128 L=6 H=8, "
                    "19233001 Pauli strings / 4111711 groups",
        "prec": "bf16x3", "steps": steps, "warmup": warmup, "ms_per_step": ms, "step_ms": [round(t, 2) for t in ts],
        "n_u_mean": nu, "value": nu * info["n_terms"] / (ms / 1e3), "unit": "pairs/s",
        "stage_ms_per_step": {k: round(v / steps, 3) for k, v in stages.items()},
        "energy_ha": float(stats[0].item()), "hamiltonian_build_s": build_s,
        "kernels_ms": {k: round(v["ms"], 3) for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])[:10]},
        "sweep_roofline": sweep_roofline(prof, peaks, 2),
    }
    sw = prof.get("k_sweep_pairs") or prof.get("k_sweep_groups")
    if sw:
        out["sweep_ms"] = sw["ms"]
    if clocks_on:
        out["clocks"] = clk.summary()
    return out


def single_core_oracle(wl_name: str, n_rows: int) -> dict:
    """The oracle's sample-aware local energy of n_rows rows against the
    full table, pinned to one host core (OpenMP and BLAS set to one thread
    by the caller's environment), extrapolated linearly to N_u rows."""
    from oracle import hamiltonian as OH
    from paper_2306_16705_gb300 import inputs as I

    wl = I.WORKLOADS[wl_name]
    h, eri = I.workload_integrals(wl)
    strings = OH.build(h, eri)
    S = I.random_sector_samples(wl.n_spatial, wl.n_alpha, wl.n_beta, N_SAMPLES, seed=wl.seed)
    lp = I.random_logpsi(N_SAMPLES, seed=wl.seed, amp_std=0.1)
    t0 = time.perf_counter()
    OH.eloc_lut(*strings, S, lp, S[:n_rows], wl.n_alpha, wl.n_beta)
    dt = time.perf_counter() - t0
    n_terms = len(strings[2])
    return {"value": n_rows * n_terms / dt, "unit": "pairs/s (local energy only)", "cores": 1,
            "kind": "oracle", "sample": f"sample-aware local energy of {n_rows} of the {N_SAMPLES} rows against "
                                        f"the full table, one core ({dt:.1f} s)"}


def run_single_core(n_rows: int = 1024) -> dict | None:
    """single_core_oracle in a child process bound to one core."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import os, json, sys; sys.path.insert(0, %r); "
            "os.sched_setaffinity(0, {sorted(os.sched_getaffinity(0))[0]}); "
            "import bench; print(json.dumps(bench.single_core_oracle(%r, %d)))" % (ROOT, WORKLOAD, n_rows))
    p = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=600)
    if p.returncode != 0:
        return {"failed": p.stderr[-300:]}
    return json.loads(p.stdout.strip().splitlines()[-1])


# ---------------------------------------------------------------- our arm
def replica_seed(rank: int) -> int:
    """Run seed of replica ``rank``: every rank samples its own batches."""
    return 1000 + int(rank)


def aggregate_ranks(ms_step: float, n_u_total: int, dist, device):
    """Replicas: the job's step time is the slowest rank's, its work the sum of
    every rank's unique samples."""
    import torch

    t = torch.tensor([ms_step], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    nu = torch.tensor([n_u_total], device=device, dtype=torch.float64)
    dist.all_reduce(nu)
    return float(t.item()), int(nu.item())


def run_ours(args):
    import torch

    from paper_2306_16705_gb300 import binding as B
    from paper_2306_16705_gb300 import inputs as I
    from paper_2306_16705_gb300.vmc import VMC

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    B.lib()
    precs = {"bf16x3": B.BF16X3, "mixed": B.MIXED, "fp32": B.FP32, "fp64": B.FP64, "fp8": B.FP8}
    prec = precs[args.prec]
    wl = I.WORKLOADS[WORKLOAD]
    h, eri = I.workload_integrals(wl)
    ham = B.build_pauli(h, eri)
    info = ham.info()
    model = B.Model(wl.n_qubits, wl.n_alpha, wl.n_beta, wl.d_model, wl.n_layers, wl.n_heads)
    params0 = model.pack(I.workload_params(wl))

    def make(p):
        # replicas: each rank samples its own batch (different seeds)
        return VMC(ham, model, params0.clone(), prec=p, n_samples=args.n_samples, max_unique=1 << 15,
                   seed=replica_seed(rank))

    peaks_run = {} if args.no_peaks else B.measure_peaks()
    vmc = make(prec)
    p_init = vmc.params.clone()
    for _ in range(args.warmup):
        vmc.step()
    vmc.params.copy_(p_init)
    vmc.m.zero_()
    vmc.v.zero_()
    vmc.t = 0
    torch.cuda.synchronize()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > L2 (129 MB)
    stream = torch.cuda.current_stream()

    def timed(n_steps, v, stages=None, state=None):
        # every timed step starts from the same random-init parameters, Adam
        # state and step count (restored outside the timed region; the Adam
        # update itself runs inside), so each step draws the same samples;
        # `state` (params, m, v, t) fixes that start across several calls
        p0, m0, v0, t0 = state if state is not None else (v.params.clone(), v.m.clone(), v.v.clone(), v.t)
        ts, nu = [], 0
        for _ in range(n_steps):
            v.params.copy_(p0)
            v.m.copy_(m0)
            v.v.copy_(v0)
            v.t = t0
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            marks = [] if stages is not None else None
            v.step(marks=marks)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
            nu += int(v.last_samples.shape[0])
            if stages is not None:
                stages["sample"] += e0.elapsed_time(marks[0])
                stages["energy_grad"] += marks[0].elapsed_time(marks[1])
                stages["adam"] += marks[1].elapsed_time(marks[2])
        return ts, nu

    state0 = (vmc.params.clone(), vmc.m.clone(), vmc.v.clone(), vmc.t)
    l0 = B.launch_count()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local, not args.no_clocks) as clk:
        times, n_u_total = timed(args.steps, vmc, state=state0)
    torch.cuda.synchronize()
    launches = B.launch_count() - l0
    # the same steps again (same start state, so the same samples) with every
    # launch bracketed by CUDA events: per-kernel device times for the roofline
    B.profile_reset()
    B.profile_enable(True)
    stages = {"sample": 0.0, "energy_grad": 0.0, "adam": 0.0}
    prof_times, _ = timed(args.steps, vmc, stages, state=state0)
    prof = B.profile()
    B.profile_enable(False)
    ms_step = float(np.mean(times))
    if dist:
        ms_step, n_u_total = aggregate_ranks(ms_step, n_u_total, dist, "cuda")
    pairs = n_u_total * info["n_terms"]
    value = pairs / (ms_step * args.steps / 1e3)

    # dominant kernel family and its roofline
    fam = max(prof.items(), key=lambda kv: kv[1]["ms"])
    name, f = fam
    avg_ms = f["ms"] / max(1, f["launches"])
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    tpk = float(peaks.get("bf16_tflops_sustained", 1700.0))
    tpk_src = "MEASURED_PEAKS.json bf16_tflops_sustained" if peaks else "fallback 1.7 PFLOP/s sustained"
    hpk = float(peaks.get("hbm_gbs", 6800.0))

    def kernel_roofline(kname, kf):
        avg = kf["ms"] / max(1, kf["launches"])
        if kname in TENSOR_KERNELS:
            # the ansatz's products are dense contractions: the bound is the
            # tensor pipe (sustained BF16, the kernels run inside a long step),
            # counted in the method's FLOPs (one product per layer, not the
            # three BF16 products of split operands); the HBM rate of the bytes
            # the launch sites attribute is given beside it
            gbs = kf["bytes"] / (kf["ms"] / 1e3) / 1e9
            tflops = kf["flops"] / (kf["ms"] / 1e3) / 1e12
            traffic = (KERNEL_TRAFFIC_BYTES.get(kname) if args.n_samples == N_SAMPLES and args.prec == "bf16x3"
                       else None)
            return {"kernel": kname, "bound": "tensor", "achieved": tflops, "peak": tpk, "unit": "TFLOP/s",
                    "frac": tflops / tpk, "traffic": traffic, "peak_source": tpk_src + " (of measured)",
                    "flops_per_launch": kf["flops"] / max(1, kf["launches"]),
                    "hbm": {"achieved_gbs": gbs, "peak_gbs": hpk, "frac": gbs / hpk,
                            "algorithmic_bytes_per_launch": kf["bytes"] / max(1, kf["launches"]),
                            "peak_source": "MEASURED_PEAKS.json hbm_gbs" if peaks else "fallback 6.8 TB/s"},
                    "launches": kf["launches"], "avg_launch_ms": avg}
        if kname == "k_gemm":
            fpk = peaks_run.get("fp32_flops", FP32_PEAK_TFLOPS * 1e12) / 1e12
            achieved = kf["flops"] / (kf["ms"] / 1e3) / 1e12
            return {"kernel": kname, "bound": "alu", "achieved": achieved, "peak": fpk,
                    "unit": "TFLOP/s", "frac": achieved / fpk, "traffic": None,
                    "peak_source": "nnqs_measure_peaks FP32 FMA (measured)" if peaks_run else "derived FP32 peak",
                    "launches": kf["launches"], "avg_launch_ms": avg}
        if kname.startswith("k_sweep") and sweep_roofline(prof, peaks_run, 1):
            return sweep_roofline(prof, peaks_run, 1)
        return {"kernel": kname, "bound": "unknown", "achieved": None, "peak": None, "unit": None,
                "frac": None, "traffic": None, "launches": kf["launches"], "avg_launch_ms": avg}

    roof = kernel_roofline(name, f)
    # the whole ansatz (forward + reverse mode + sampler) in method FLOPs
    # against the sustained tensor peak, and the sweep against the measured
    # XOR+popcount rate
    fwd = model_flops_per_sample(wl)
    n_u_step = n_u_total / max(1, args.steps * world)
    rooflines = {"sweep": sweep_roofline(prof, peaks_run, 1),
                 "tensor_kernels": {k: kernel_roofline(k, prof[k]) for k in TENSOR_KERNELS if k in prof},
                 "energy_grad_ansatz": {
                     "bound": "tensor", "unit": "TFLOP/s", "peak": tpk,
                     "flops_per_step": 3.0 * fwd * n_u_step,
                     "note": "method FLOPs of one forward and its reverse mode (2x) over the step's unique samples, "
                             "divided by the energy-gradient stage time (which also holds the local energy)"}}
    eg_ms = stages["energy_grad"] / args.steps
    rooflines["energy_grad_ansatz"]["achieved"] = 3.0 * fwd * n_u_step / (eg_ms / 1e3) / 1e12
    rooflines["energy_grad_ansatz"]["frac"] = rooflines["energy_grad_ansatz"]["achieved"] / tpk

    line = {
        "metric": "local-energy (sample x Pauli-term) evals/sec, whole VMC step",
        "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step, "step_ms": [round(t, 3) for t in times], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"bf16x3": "bf16 hi+lo split operands (forward), bf16 (reverse mode), f32 accumulate / "
                            "f64 local energy",
                  "fp32": "f32 ansatz / f64 local energy", "mixed": "bf16+f32 ansatz / f64 local energy",
                  "fp8": "e4m3 (forward), bf16 (reverse mode), f32 accumulate / f64 local energy",
                  "fp64": "f64"}[args.prec],
        "data": "synthetic (random integrals seed 1 rank 16; random-init ansatz)",
        "config": workload_config(info["n_terms"], info["n_groups"], args.n_samples,
                                  n_u_total / (args.steps * world), world),
        "gpu_launches": launches,
        "roofline": roof,
        "rooflines": rooflines,
        "peaks_measured": peaks_run,
        "profiled_ms_per_step": float(np.mean(prof_times)),
        "stage_ms_per_step": {k: round(v / args.steps, 3) for k, v in stages.items()},
        "kernels_ms": {k: round(v["ms"], 4) for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])[:12]},
    }
    if not args.no_clocks:
        line["clocks"] = clk.summary()

    # plain FP64 path on the same workload
    if args.fp64_steps > 0 and prec != B.FP64:
        v64 = make(B.FP64)
        v64.step()
        torch.cuda.synchronize()
        t64, nu64 = timed(args.fp64_steps, v64)
        ms64 = float(np.mean(t64))
        # energy of the same samples and parameters through every precision
        x, w = vmc.last_samples, vmc.last_weights
        e = {k: float(B.energy_grad(ham, model, vmc.params, x, w, p)[0][0]) for k, p in precs.items()}
        line["fp64_plain"] = {"ms_per_step": ms64, "value": nu64 * info["n_terms"] / (ms64 * args.fp64_steps / 1e3),
                              "unit": "pairs/s", "speedup_of_fast_path": ms64 / ms_step,
                              "energy_ha": e["fp64"],
                              "energy_diff_ha": abs(e[args.prec] - e["fp64"]),
                              "energy_diff_by_prec_ha": {k: abs(v - e["fp64"]) for k, v in e.items() if k != "fp64"}}
        if peaks_run.get("fp64_flops"):
            # the ansatz's method FLOPs (forward + reverse mode) of the step
            # against the measured FP64 FMA rate: the plain path's CUDA-core bound
            fl64 = 3.0 * model_flops_per_sample(wl) * nu64 / args.fp64_steps / (ms64 / 1e3)
            line["fp64_plain"]["roofline"] = {
                "bound": "alu", "unit": "TFLOP/s", "achieved": fl64 / 1e12, "peak": peaks_run["fp64_flops"] / 1e12,
                "frac": fl64 / peaks_run["fp64_flops"],
                "peak_source": "nnqs_measure_peaks FP64 FMA (measured in this run)",
                "note": "method FLOPs of one forward and its reverse mode over the step's samples / step time"}
        # the other fast paths' step times
        others = {}
        for k in ("bf16x3", "mixed", "fp32", "fp8"):
            if k == args.prec:
                continue
            vo = make(precs[k])
            vo.step()
            to, nuo = timed(max(2, args.fp64_steps), vo)
            mso = float(np.mean(to))
            others[k] = {"ms_per_step": mso, "value": nuo * info["n_terms"] / (mso * len(to) / 1e3),
                         "unit": "pairs/s", "energy_diff_ha": abs(e[k] - e["fp64"])}
        line["other_paths"] = others

    # layout comparison (Sec. 3.4): bytes of the grouped and ungrouped string
    # tables, and one sample-aware E_loc call per sweep on this step's samples
    if rank == 0 and world == 1 and not args.no_layouts:
        x, w = vmc.last_samples, vmc.last_weights
        lp = B.logpsi(model, vmc.params, x, prec)
        ham.build_ungrouped()
        lay = {"bytes": ham.layout_bytes(), "sweep_ms": {}}
        outs = {}
        for name, fl in (("groups", B.SWEEP_GROUPS), ("pairs", B.SWEEP_PAIRS), ("terms", B.SWEEP_TERMS)):
            B.eloc(ham, x, lp, wl.n_alpha, wl.n_beta, flags=fl)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            outs[name] = B.eloc(ham, x, lp, wl.n_alpha, wl.n_beta, flags=fl)
            e1.record(stream)
            e1.synchronize()
            lay["sweep_ms"][name] = e0.elapsed_time(e1)
        ref = outs["groups"]
        lay["max_abs_diff_vs_groups"] = {k: float((v - ref).abs().max()) for k, v in outs.items() if k != "groups"}
        lay["reduction_packed"] = 1 - lay["bytes"]["grouped"] / lay["bytes"]["ungrouped"]
        lay["reduction_bytewise"] = 1 - lay["bytes"]["grouped_bytewise"] / lay["bytes"]["ungrouped_bytewise"]
        line["layout_comparison"] = lay

    if rank == 0 and world == 1 and args.exact_rows > 0:
        try:
            line["exact_mode"] = run_exact_side_line(ham, model, wl, vmc.params, vmc.last_samples, prec,
                                                     args.exact_rows, peaks_run,
                                                     float(peaks.get("bf16_tflops", 1890.0)))
        except Exception as exc:
            line["exact_mode"] = {"failed": str(exc)}
    if rank == 0 and world == 1 and args.n120_steps > 0:
        try:
            line["n120"] = run_n120_side_line(args.n120_steps, 1, peaks_run, not args.no_clocks, local)
        except Exception as exc:
            line["n120"] = {"failed": str(exc)}

    # end to end through the public API with host buffers: parameters in
    # from pinned memory, energy statistics and parameters out, every step
    p_host = vmc.params.detach().cpu().pin_memory()
    st_host = torch.empty(4, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    e2e_t = []
    p_host.copy_(p_init.cpu())
    m0, v0 = torch.zeros_like(vmc.m), torch.zeros_like(vmc.v)
    for _ in range(max(2, args.steps // 2) if args.e2e_steps < 0 else args.e2e_steps):
        vmc.m.copy_(m0)
        vmc.v.copy_(v0)
        vmc.t = 0
        p_host.copy_(p_init.cpu())
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        vmc.params.copy_(p_host, non_blocking=True)
        stats = vmc.step()
        st_host.copy_(stats, non_blocking=True)
        p_host.copy_(vmc.params, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_t.append(e0.elapsed_time(e1))
    ms_e2e = float(np.mean(e2e_t)) if e2e_t else float("nan")
    nbytes = vmc.params.numel() * 4
    line["e2e"] = {"value": int(vmc.last_samples.shape[0]) * info["n_terms"] * world / (ms_e2e / 1e3),
                   "unit": "pairs/s", "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes + 32,
                   "ms_per_step": ms_e2e}

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            base = sized_oracle_run(OracleStep(wl), 10.0)
            line["cpu_baseline"] = {"value": base["pairs_per_s"], "unit": "pairs/s", "cores": cores(),
                                    "kind": "oracle", "sample": base["sample"]}
        except Exception as exc:  # keep the GPU line even if the oracle cannot build here
            line["cpu_baseline"] = {"value": None, "unit": "pairs/s", "cores": cores(), "kind": "oracle",
                                    "sample": f"failed: {exc}"}
        try:
            line["cpu_baseline"]["single_core"] = run_single_core()
        except Exception as exc:
            line["cpu_baseline"]["single_core"] = {"failed": str(exc)}
        if args.ladder:
            try:
                line["cpu_baseline"]["ladder"] = run_ladder()
            except Exception as exc:
                line["cpu_baseline"]["ladder"] = {"failed": str(exc)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_case(args):
    """One hot-path call on a named workload, timed alone (three warm-up
    calls, then the mean of five with CUDA events): the sample-aware sweeps
    over uniform sector samples with a stand-in log psi table or over the
    sampler's own draws from the random-init ansatz (-sampled), the ansatz
    forward (fused, or layer by layer), the forward with its reverse mode for
    a random seed vector (fused, or layer by layer), or exact-mode E_loc of
    the first rows.
    For profilers: the kernel of interest runs 8 times (3 warm-up + 5)."""
    import torch

    from paper_2306_16705_gb300 import binding as B
    from paper_2306_16705_gb300 import inputs as I

    if args.case in ("logpsi-unfused", "grad-unfused"):
        os.environ["NNQS_FUSED_FORWARD"] = "0"
        os.environ["NNQS_FUSED_BACKWARD"] = "0"
    wl = I.WORKLOADS[args.workload]
    S = I.random_sector_samples(wl.n_spatial, wl.n_alpha, wl.n_beta, args.n, seed=3)
    x = B.to_device_bits(S)
    rows = args.rows or args.n
    prec = {"bf16x3": B.BF16X3, "mixed": B.MIXED, "fp32": B.FP32, "fp64": B.FP64, "fp8": B.FP8}[args.prec]
    if args.case.startswith("sweep") or args.case == "eloc-exact":
        h, eri = I.workload_integrals(wl)
        ham = B.build_pauli(h, eri)
    if args.case.endswith("-sampled"):
        # the step's own input: unique samples drawn by the sampler from the
        # random-init ansatz, with their log psi
        model = B.Model(wl.n_qubits, wl.n_alpha, wl.n_beta, wl.d_model, wl.n_layers, wl.n_heads)
        flat = model.pack(I.workload_params(wl))
        x, _ = B.sample(model, flat, args.n, seed=1000, max_unique=max(1 << 15, 2 * args.n), prec=B.BF16X3)
        rows = min(rows, x.shape[0])
        lp = B.logpsi(model, flat, x, B.BF16X3)
        fl = B.SWEEP_PAIRS if args.case.startswith("sweep-pairs") else B.SWEEP_GROUPS
        call = lambda: B.eloc(ham, x, lp, wl.n_alpha, wl.n_beta, flags=fl, n_rows=rows, check=False)
    elif args.case.startswith("sweep"):
        lp = torch.from_numpy(I.random_logpsi(args.n, seed=4, amp_std=0.1)).cuda()
        fl = B.SWEEP_PAIRS if args.case == "sweep-pairs" else B.SWEEP_GROUPS
        call = lambda: B.eloc(ham, x, lp, wl.n_alpha, wl.n_beta, flags=fl, n_rows=rows, check=False)
    else:
        model = B.Model(wl.n_qubits, wl.n_alpha, wl.n_beta, wl.d_model, wl.n_layers, wl.n_heads)
        flat = model.pack(I.workload_params(wl))
        if args.case == "eloc-exact":
            call = lambda: B.eloc(ham, x[:rows], None, wl.n_alpha, wl.n_beta, mode=B.EXACT, model=model,
                                  params=flat, prec=prec, check=False)
        elif args.case.startswith("grad"):
            # the ansatz forward and its reverse mode for a seed vector d E / d log psi
            rng = np.random.default_rng(5)
            seed = torch.from_numpy(np.stack([rng.normal(size=args.n), rng.normal(size=args.n)], 1)).cuda()
            call = lambda: B.logpsi_backward(model, flat, x, seed, prec)
        else:
            call = lambda: B.logpsi(model, flat, x, prec, check=False)
    heavy = args.case == "eloc-exact"  # seconds per call at full size: one warm-up, two timed
    n_warm, n_timed = (1, 2) if heavy else (3, 5)
    for _ in range(n_warm):
        call()
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(n_timed):
        out = call()
    e1.record(st)
    e1.synchronize()
    line = {"case": args.case, "workload": args.workload, "n": args.n, "rows": rows, "prec": args.prec,
            "ms_per_call": e0.elapsed_time(e1) / n_timed}
    if heavy:
        # the exact local energies of the rows beside the sample-aware ones
        # (sum over x' in the table only, Alg. 2) with the same log psi
        Ud, cnt, _, _ = B.exact_coupled(ham, x[:rows], wl.n_alpha, wl.n_beta, row_cap=0, check=False,
                                        cap_unique=rows * ham.info()["n_groups"])
        lp = B.logpsi(model, flat, x, prec)
        sa = B.eloc(ham, x, lp, wl.n_alpha, wl.n_beta, n_rows=rows)
        line.update({"unique_coupled_states": int(Ud.shape[0]),
                     "coupled_states_per_s": int(Ud.shape[0]) / (line["ms_per_call"] / 1e3),
                     "mean_eloc_exact": float(out[:, 0].mean()), "mean_eloc_sample_aware": float(sa[:, 0].mean())})
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.case:
        run_case(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
