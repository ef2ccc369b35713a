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
# DRAM read + write bytes per k_tc_gemm launch of this step, from one ncu capture of the current kernel
# at this workload (profiles/k_tc_gemm_energy_grad_n40.md); None once the kernel changes
TC_GEMM_TRAFFIC_BYTES = 358.4e6


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="bf16x3", choices=["bf16x3", "mixed", "fp32", "fp64"])
    ap.add_argument("--fp64-steps", type=int, default=2, help="steps of the plain FP64 path (0 = skip)")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=-1, help="end-to-end steps (default steps/2, min 2)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n-samples", type=int, default=N_SAMPLES, help="N_s per step (smaller for profiling)")
    ap.add_argument("--no-layouts", action="store_true", help="skip the grouped/ungrouped layout comparison")
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
    ts = []
    last = None
    for _ in range(args.steps):
        last = sized_oracle_run(bench, target_s) if last is None else bench.run(512, last["n_rows"])
        ts.append(last["step_s"])
    step_s = float(np.mean(ts))
    value = N_SAMPLES * last["n_terms"] / step_s
    unit = "pairs/s"
    line = {
        "impl": "reference", "metric": "local-energy (sample x Pauli-term) evals/sec, whole VMC step",
        "value": value, "unit": unit, "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": step_s * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": "n40: 40 spin orbitals, 20 electrons, N_u=16384, d=64 L=4 H=8",
                   "n_terms": last["n_terms"], "l2": "CPU run"},
        "cpu_baseline": {"value": value, "unit": unit, "cores": cores(), "kind": "oracle",
                         "sample": last["sample"]},
        "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm
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
    precs = {"bf16x3": B.BF16X3, "mixed": B.MIXED, "fp32": B.FP32, "fp64": B.FP64}
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
                   seed=1000 + rank)

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

    def timed(n_steps, v, stages=None):
        # every timed step starts from the same random-init parameters and
        # Adam state (restored outside the timed region; the Adam update
        # itself runs inside), so each step samples the same distribution
        p0, m0, v0, t0 = v.params.clone(), v.m.clone(), v.v.clone(), v.t
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

    l0 = B.launch_count()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local, not args.no_clocks) as clk:
        times, n_u_total = timed(args.steps, vmc)
    torch.cuda.synchronize()
    launches = B.launch_count() - l0
    # the same number of steps again with every launch bracketed by CUDA
    # events: per-kernel device times for the roofline
    B.profile_reset()
    B.profile_enable(True)
    stages = {"sample": 0.0, "energy_grad": 0.0, "adam": 0.0}
    prof_times, _ = timed(args.steps, vmc, stages)
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
    if name == "k_tc_gemm":
        # the ansatz's layers are thin (K, N <= 4 d): ~25 flop per byte, far
        # below the tensor ridge, so the bound is HBM; the tensor rate is given beside
        pk = float(peaks.get("hbm_gbs", 6800.0))
        tpk = float(peaks.get("bf16_tflops_sustained", 1700.0))
        gbs = f["bytes"] / (f["ms"] / 1e3) / 1e9
        tflops = f["flops"] / (f["ms"] / 1e3) / 1e12
        traffic = (TC_GEMM_TRAFFIC_BYTES if TC_GEMM_TRAFFIC_BYTES and args.n_samples == N_SAMPLES
                   and args.prec == "bf16x3" else None)
        roof = {"kernel": name, "bound": "hbm", "achieved": gbs, "peak": pk, "unit": "GB/s", "frac": gbs / pk,
                "traffic": traffic,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs" if peaks else "fallback 6.8 TB/s",
                "tensor_tflops": tflops, "tensor_frac_of_sustained_bf16": tflops / tpk,
                "algorithmic_bytes_per_launch": f["bytes"] / max(1, f["launches"]),
                "launches": f["launches"], "avg_launch_ms": avg_ms}
    elif name == "k_gemm":
        achieved = f["flops"] / (f["ms"] / 1e3) / 1e12
        roof = {"kernel": name, "bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS, "traffic": None,
                "peak_source": "FP32 CUDA-core FMA: 152 SMs x 128 lanes x 2 x 2070 MHz (derived)",
                "launches": f["launches"], "avg_launch_ms": avg_ms}
    elif f["flops"] > 0:
        achieved = f["flops"] / (f["ms"] / 1e3)
        roof = {"kernel": name, "bound": "alu", "achieved": achieved, "unit": "work/s", "peak": None,
                "frac": None, "traffic": None, "launches": f["launches"], "avg_launch_ms": avg_ms}
    else:
        roof = {"kernel": name, "bound": "unknown", "achieved": None, "peak": None, "unit": None,
                "frac": None, "traffic": None, "launches": f["launches"], "avg_launch_ms": avg_ms}

    line = {
        "metric": "local-energy (sample x Pauli-term) evals/sec, whole VMC step",
        "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step, "step_ms": [round(t, 3) for t in times], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"bf16x3": "bf16 hi+lo split operands (forward), bf16 (reverse mode), f32 accumulate / "
                            "f64 local energy",
                  "fp32": "f32 ansatz / f64 local energy", "mixed": "bf16+f32 ansatz / f64 local energy",
                  "fp64": "f64"}[args.prec],
        "data": "synthetic (random integrals seed 1 rank 16; random-init ansatz)",
        "config": {"workload": f"n40: 40 spin orbitals, 20 electrons, N_s={args.n_samples}, "
                               "d=64 L=4 H=8, 233001 Pauli strings / 46171 groups",
                   "n_terms": info["n_terms"], "n_groups": info["n_groups"],
                   "n_u_mean": n_u_total / (args.steps * world), "parallelism": "replicas" if world > 1 else "1 GPU",
                   "l2": "flushed between steps (256 MB memset)"},
        "gpu_launches": launches,
        "roofline": roof,
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
        # the other fast paths' step times
        others = {}
        for k in ("bf16x3", "mixed", "fp32"):
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
        if args.ladder:
            try:
                line["cpu_baseline"]["ladder"] = run_ladder()
            except Exception as exc:
                line["cpu_baseline"]["ladder"] = {"failed": str(exc)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
