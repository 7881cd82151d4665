"""Benchmark: posterior-sample x Lambda log-likelihood + gradient evaluations per second.

Workload (O5-like, the paper's Sec. 3.1 scale): 2000 events with log-uniform 1k-16k
posterior samples each (~1.08e7 samples), nside-64 HEALPix LOS priors (49,152 pixels)
on a 2,048-point redshift grid, 1e7 detected injections, and a batch of K = 256
Lambda points per call.  One step = one gwc_loglik_grad call on the whole batch:
prologue, fused sample x Lambda value+gradient kernel, merge.  Inputs are synthetic
(seeded) and resident in HBM before timing; their ~0.8 GB exceeds the 129 MB L2, so no
flush is needed between steps.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle instead,
on a bounded sample of the same workload per step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "posterior-sample×Λ log-lik+grad evals/s at O5 scale vs plain GPU path"
WORKLOAD = "c3"
K_LAMBDA = 256
WORKLOAD_NAMES = {
    "c1": "c1: 10 events x 1000 samples, 1e4 injection draws (the HMC chain's workload)",
    "c2": "c2: 150 events x U{2000..8000} samples, nside-32 (12288 px) x 2048-z LOS, 1e6 injections",
    "c3": "c3: 2000 events x log-uniform 1k-16k samples (O5-like), nside-64 (49152 px) x 2048-z LOS, "
          "1e7 detected injections",
    "c5": "c5: 10000 events x 4096 samples, nside-64 x 2048-z LOS, 5e7 injections",
}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# Algorithmic work per (sample, Lambda) evaluation of the fused kernel, counted by hand
# from its source (sample_lnw and the accumulator), per stage that an evaluation reaches
# (the stages of gwc_path_census).  Each entry: (FP32 operations of the method, FP32
# operations that exist only for precision, {special-function op: count}).  FP32
# operations are adds, multiplies and fused multiply-adds (compares, min/max, selects and
# conversions are not counted); the accurate log2f of the product counts as one lg2
# (its extra accuracy work is not counted).  "Precision" is the compensation the FP32
# path carries against shared biases: the split table coordinate (x hi + lo, 6 ops), the
# low parts of alpha, beta, 1+beta and gamma+kappa (one FMA each where used).  Stages
# named *_nowin1 are charged to the evaluations of the parent stage outside the m1
# smoothing window (the closed-form C(m1)); the weight_* stages are the gradient's and
# are charged to every evaluation with a positive weight (an upper bound: the kernel
# skips the derivatives of weights below 2^-48 of the running maximum).
WORK = {
    "live": (1, 0, {}),                                         # x = d_L H0/c, range test
    "in_range": (9, 6, {}),                                     # table position, cell, z
    "mass_order": (3, 0, {"rcp": 1}),                           # 1+z, source masses
    "support": (5, 0, {"lg2": 1}),                              # log2(1+z), LOS lerp
    "value": (27, 2, {"ex2": 3, "rsqrt": 1, "rcp": 1, "lg2": 1}),  # mixture, rate, Jacobian, log, accumulate
    "value_nowin1": (3, 2, {"ex2": 1}),                         # C(m1) above the window
    "value_win1": (20, 1, {}),                                  # C(m1) from the window table
    "value_win2": (7, 0, {"rcp": 2, "ex2": 1}),                 # smoothing of m2
    "weight": (61, 0, {"rcp": 4}),                              # z-chain, J(x) quadratic, 13 statistics
    "weight_nowin1": (8, 0, {"rcp": 1}),
    "weight_win1": (48, 0, {"rcp": 5, "ex2": 1}),
    "weight_win2": (9, 0, {"rcp": 1}),
}
SFU_TYPES = ("ex2", "lg2", "rcp", "rsqrt")
SMS = 152


def work_from_census(census, grad=True):
    """FP32 (method, precision) and special-function op counts of one call, from the
    stage counts of gwc_path_census and the WORK table."""
    n = dict(census)
    n["value_nowin1"] = n["value"] - n["value_win1"]
    n["weight_nowin1"] = n["weight"] - n["weight_win1"]
    stages = [k for k in WORK if grad or not k.startswith("weight")]
    meth = sum(n[k] * WORK[k][0] for k in stages)
    prec = sum(n[k] * WORK[k][1] for k in stages)
    sfu = {t: sum(n[k] * WORK[k][2].get(t, 0) for k in stages) for t in SFU_TYPES}
    return {"fp32_method": meth, "fp32_precision": prec, "sfu": sfu}


# Throughput probes (gwc_alu_probe): CTAs per launch and iterations per chain, sized so
# that each launch takes ~10-40 ms
PROBES = {"ffma": 320_000, "ffma2": 160_000, "ex2": 40_000, "lg2": 40_000, "rcp": 40_000,
          "rsqrt": 40_000, "dfma": 5_000, "dfma_lane1": 5_000}
PROBE_BLOCKS = SMS * 8


def measure_alu_peaks(g, stream, clock_index):
    """Operations per second of each arithmetic unit (best of three timed launches after
    one untimed), with the SM clock sampled meanwhile; per SM per clock as well."""
    import torch
    sampler = ClockSampler(clock_index)
    sampler.start()
    out = {}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for unit, iters in PROBES.items():
        g.alu_probe(unit, PROBE_BLOCKS, iters, stream)
        best = float("inf")
        for _ in range(3):
            e0.record(stream)
            ops = g.alu_probe(unit, PROBE_BLOCKS, iters, stream)
            e1.record(stream)
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
        out[unit] = {"ops_per_s": ops / best, "ms": best * 1e3}
    clocks = sampler.stop()
    mhz = clocks["sm_mhz"] if clocks else None
    for unit in out:
        out[unit]["per_sm_per_clk"] = (out[unit]["ops_per_s"] / (SMS * mhz * 1e6)) if mhz else None
    return {"units": out, "clocks": clocks,
            "how": f"gwc_alu_probe: {PROBE_BLOCKS} CTAs x 256 threads x 8 independent chains, "
                   "best of 3 CUDA-event-timed launches after 1 untimed; per_sm_per_clk uses the "
                   "median SM clock sampled during the probes"}


def alu_roofline(work, seconds, peaks, kernel_mhz):
    """The binding arithmetic unit of one launch: the slower of the FP32 pipe (the better
    of scalar and packed FMA) and the special-function unit (each op type at its own
    measured rate), with the probes' rates scaled from their clock to the kernel's."""
    u = peaks["units"]
    probe_mhz = (peaks.get("clocks") or {}).get("sm_mhz")
    scale = (kernel_mhz / probe_mhz) if (kernel_mhz and probe_mhz) else 1.0
    fp32_peak = max(u["ffma"]["ops_per_s"], u["ffma2"]["ops_per_s"]) * scale
    t_fp32 = work["fp32_method"] / fp32_peak
    t_fp32_all = (work["fp32_method"] + work["fp32_precision"]) / fp32_peak
    sfu_ops = sum(work["sfu"].values())
    t_sfu = sum(work["sfu"][t] / (u[t]["ops_per_s"] * scale) for t in SFU_TYPES)
    # the issue port: an SM issues one warp-instruction per scheduler per clock, and the
    # FP32 pipe's measured peak is that rate (32 lanes x 4 schedulers, less a few percent),
    # so the method's FP32 and special-function instructions together need at least
    # (FP32 + SFU lane operations) / FP32 peak, whatever each pipe's own rate
    t_issue = (work["fp32_method"] + sfu_ops) / fp32_peak
    common = {"bound": "alu", "peak_source": "measured (gwc_alu_probe on this GPU)",
              "clock_scale": scale, "t_fp32_ms": t_fp32 * 1e3, "t_sfu_ms": t_sfu * 1e3,
              "t_issue_fp32_plus_sfu_ms": t_issue * 1e3, "frac_issue_fp32_plus_sfu": t_issue / seconds,
              "t_fp32_with_precision_ms": t_fp32_all * 1e3, "kernel_ms": seconds * 1e3,
              "fp32_method_ops": work["fp32_method"], "fp32_precision_ops": work["fp32_precision"],
              "sfu_ops": work["sfu"]}
    if t_fp32 >= t_sfu:
        ach = work["fp32_method"] / seconds / 1e12
        return dict(common, unit="Tops/s (FP32 pipe, method ops)", achieved=ach, peak=fp32_peak / 1e12,
                    frac=ach / (fp32_peak / 1e12),
                    frac_with_precision=t_fp32_all / seconds)
    sfu_peak = sfu_ops / t_sfu
    ach = sfu_ops / seconds / 1e12
    return dict(common, unit="Tops/s (SFU, this op mix)", achieved=ach, peak=sfu_peak / 1e12,
                frac=ach / (sfu_peak / 1e12), frac_fp32_with_precision=t_fp32_all / seconds)


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one fused value+gradient
# launch on the default workload and batch, from an ncu capture of the kernel and layout
# sources whose digest is recorded here; reported only while the sources still have it.
TRAFFIC = {"digest": "4e6d26ab57248f68", "workload": "c3", "K": 256, "bytes_per_launch": 1068.35e6}
KERNEL_SOURCES = ("gwc_kernels.cu", "gwc_internal.cuh", "gwc_kernels.h", "gwc_api.cu")


def _code_only(text):
    """Source text without comments, trailing blanks or blank lines (so that an edit of
    a comment keeps the digest of code that has not changed)."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(ln.rstrip() for ln in text.splitlines() if ln.strip())


def kernel_digest(read=None):
    """Digest of the code of the kernel and layout sources (see _code_only)."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        path = os.path.join("paper_2605_23538_gb300", "csrc", f)
        if read is None:
            with open(os.path.join(ROOT, path), encoding="utf-8") as fh:
                text = fh.read()
        else:
            text = read(path)
        h.update(_code_only(text).encode())
    return h.hexdigest()[:16]


def traffic_for(workload, K):
    if (TRAFFIC["digest"] == kernel_digest() and TRAFFIC["workload"] == workload
            and TRAFFIC["K"] == K):
        return TRAFFIC["bytes_per_launch"]
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def host_description():
    """nproc and the CPU model lines of lscpu (the host the oracle runs on)."""
    desc = {"nproc": os.cpu_count()}
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            k, _, v = ln.partition(":")
            if k.strip() in ("Architecture", "Model name", "CPU(s)", "Thread(s) per core", "Socket(s)"):
                desc[k.strip()] = v.strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return desc


def oracle_sample(cat, n_ev, n_inj=None):
    """The first n_ev events and the first n_inj injections of the workload; by default
    as many injections per event sample as the whole workload has (the two kinds of
    evaluation cost differently: many injections leave at the mass cut)."""
    from paper_2605_23538_gb300 import synth
    sub = synth.subset_events(cat, range(n_ev))
    if n_inj is None:
        n_inj = int(round(int(sub["offsets"][-1]) * len(cat["inj_m1"]) / len(cat["m1"])))
    n_inj = max(1, min(n_inj, len(cat["inj_m1"])))
    for k in ("inj_m1", "inj_m2", "inj_dl", "inj_lnpd"):
        sub[k] = cat[k][:n_inj]
    return sub, int(sub["offsets"][-1]) + n_inj


def cpu_baseline(cat, lam, max_seconds=20.0):
    """The FP64 oracle (value + gradient) on a bounded sample of the workload, on all host
    cores and on one core."""
    import oracle
    cores = os.cpu_count() or 1
    n_ev_max = len(cat["offsets"]) - 1
    # all cores: at least four events per core (the oracle runs events in parallel, and
    # injections in chunks of about n_inj / (4 cores)); grow the sample until one timed
    # pass takes about half of max_seconds or more
    n_ev = min(n_ev_max, 4 * cores)
    while True:
        sub, evals = oracle_sample(cat, n_ev)
        n_inj = len(sub["inj_m1"])
        t0 = time.perf_counter()
        oracle.loglik(sub, lam[:1], grad=True, n_threads=cores)
        dt = time.perf_counter() - t0
        if dt > 0.4 * max_seconds or n_ev >= n_ev_max:
            break
        grow = max(1.5, min(8.0, 0.7 * max_seconds / max(dt, 1e-3)))
        n_ev = min(n_ev_max, int(n_ev * grow))
    value = evals / dt
    # one core: a slice of the same sample sized to take about a quarter of max_seconds
    frac = min(1.0, 0.25 * max_seconds / max(dt * cores, 1e-3))
    n1_ev = max(1, int(n_ev * frac))
    sub1, evals1 = oracle_sample(cat, n1_ev)
    n1_inj = len(sub1["inj_m1"])
    t0 = time.perf_counter()
    oracle.loglik(sub1, lam[:1], grad=True, n_threads=1)
    dt1 = time.perf_counter() - t0
    return dict(value=value, unit="evals/s", cores=cores, kind="oracle",
                sample=f"1 Lambda x ({int(sub['offsets'][-1])} samples of the first {n_ev} events "
                       f"+ the first {n_inj} injections), FP64 value+gradient, {dt:.1f} s on {cores} threads",
                one_core={"value": evals1 / dt1, "unit": "evals/s", "cores": 1,
                          "sample": f"1 Lambda x ({int(sub1['offsets'][-1])} samples of the first {n1_ev} "
                                    f"events + the first {n1_inj} injections), {dt1:.1f} s"},
                host=host_description())


# HMC on the small workload (10 events x 1000 samples, 1e4 injection draws): one chain,
# trajectories of 32 leapfrog steps recorded as one CUDA graph; M^-1 = diag(scale^2)
HMC_SCALE = np.array([2.0, 0.1, 0.5, 0.5, 0.5, 5.0, 0.5, 2.0, 1.0, 0.02, 0.5, 2.0, 0.5])
HMC_LEAPFROG, HMC_EPS, HMC_TRAJ, HMC_WARM = 32, 0.005, 30, 30


def hmc_c1(g, synth, stream):
    import torch
    cat = synth.catalogue("c1")
    n = len(cat["m1"]) + len(cat["inj_m1"])
    r = np.random.default_rng(5)
    with g.Context(cat, max_K=1) as ctx:
        h = ctx.hmc(1, HMC_LEAPFROG, np.full(1, HMC_EPS), HMC_SCALE ** 2)
        q = torch.tensor(synth.FIDUCIAL[None, :], device="cuda")
        h.q.copy_(q)
        p = torch.tensor(r.standard_normal((HMC_TRAJ + HMC_WARM, 1, 13)) / HMC_SCALE, device="cuda")
        lu = torch.tensor(np.log(r.random((HMC_TRAJ + HMC_WARM, 1))), device="cuda")
        for t in range(HMC_WARM):   # the first replays of a new graph are slow
            h.run(None, p[t], lu[t], stream)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(HMC_TRAJ + 1)]
        torch.cuda.synchronize()
        acc = torch.zeros(1, dtype=torch.int32, device="cuda")
        ev[0].record(stream)
        for t in range(HMC_TRAJ):
            h.run(None, p[t + HMC_WARM], lu[t + HMC_WARM], stream)
            acc += h.accept
            ev[t + 1].record(stream)
        torch.cuda.synchronize()
        # median over trajectories: at K = 1 the GPU is nearly idle and its clock may still
        # be rising, so the first ones can be slow
        ms = float(np.median([ev[t].elapsed_time(ev[t + 1]) for t in range(HMC_TRAJ)]))
        h.close()
        # where a K = 1 evaluation's time goes: direct value+gradient calls with the
        # library's per-stage events (not inside a graph)
        out = g._outputs(1, ctx.n_events, q.device, True)
        for _ in range(10):
            g.loglik_grad(ctx._ctx, q, ctx.n_events, stream, out)
        torch.cuda.synchronize()
        ctx.profile_enable(True)
        ctx.profile_read()
        for _ in range(50):
            g.loglik_grad(ctx._ctx, q, ctx.n_events, stream, out)
        stage_ms, n_calls = ctx.profile_read()
        ctx.profile_enable(False)
    stages = {name: stage_ms[i] / max(n_calls, 1) for i, name in enumerate(("prologue", "fused", "merge"))}
    return {"workload": "c1 (10 events x 1000 samples, 1e4 draws), K = 1",
            "leapfrog_steps": HMC_LEAPFROG, "ms_per_trajectory": ms, "statistic": "median of 30",
            "evals_per_s": (HMC_LEAPFROG + 1) * n / (ms / 1e3),
            "acceptance": float(acc.item()) / HMC_TRAJ,
            "stage_ms_per_call": stages}


# The paper's KDE form of the event term (value only), on the bench's catalogue with the
# first KDE_K points of the batch: Scott bandwidth, 256-point grid, per-pixel N_eff >= 2
KDE_K = 16


# Work of the KDE kernel, counted from its source as lower bounds (gwc_kde_census): one
# evaluation of the weight w' (the value arithmetic without the LOS factor: the live,
# in_range, mass_order, support and value stages of WORK less the LOS interpolation, with
# the closed-form C(m1)) per second-pass sample with a weight, and per grid term the
# kernel's value by the product recurrence and its accumulation, T += p_LOS(z_g) e,
# e *= r, r *= q (3 FP32 operations), plus each block of 4 terms' start, d_0, e_0 =
# 2^((c d_0) d_0) and r_0 (5 FP32 operations, two ex2): 4.25 FP32 and 0.5 ex2 a term.
# The first pass's evaluations (which repeat the second's for kept samples) and the
# bandwidths' order statistics are not charged.
KDE_WORK_EVAL = (46, {"ex2": 4, "lg2": 2, "rcp": 2, "rsqrt": 1})
KDE_WORK_TERM = (4.25, {"ex2": 0.5})


def kde_timing(g, ctx, lam, n_evals, stream, peaks):
    import torch
    k = max(1, min(KDE_K, lam.shape[0]))
    lk = lam[:k].contiguous()
    out = g._outputs(k, ctx.n_events, lk.device, False)
    for _ in range(2):
        g.loglik_kde(ctx._ctx, lk, ctx.n_events, stream=stream, out=out)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    reps = 3
    ctx.profile_enable(True)
    ctx.profile_read()
    e0.record(stream)
    for _ in range(reps):
        g.loglik_kde(ctx._ctx, lk, ctx.n_events, stream=stream, out=out)
    e1.record(stream)
    torch.cuda.synchronize()
    stage_ms, n_calls = ctx.profile_read()
    ctx.profile_enable(False)
    ms = e0.elapsed_time(e1) / reps
    kde_ms = stage_ms[1] / max(n_calls, 1)
    census = ctx.kde_census(lk, stream=stream)
    fp32 = census["pass2"] * KDE_WORK_EVAL[0] + census["terms"] * KDE_WORK_TERM[0]
    sfu = {t: census["pass2"] * KDE_WORK_EVAL[1].get(t, 0) + census["terms"] * KDE_WORK_TERM[1].get(t, 0)
           for t in SFU_TYPES}
    roof = alu_roofline({"fp32_method": fp32, "fp32_precision": 0, "sfu": sfu}, kde_ms / 1e3, peaks, None)
    roof["census"] = census
    roof["work"] = "lower bound: w' once per weighted second-pass sample, 4.25 FP32 + 0.5 ex2 per grid term"
    return {"K": k, "bandwidth": "scott", "n_grid": 256, "ms_per_call": ms, "kde_kernel_ms": kde_ms,
            "value": n_evals * k / (ms / 1e3), "unit": "evals/s (value only)", "roofline": roof}


def multipeak_timing(g, synth, cat, K, n_evals, stream, steps=3):
    """The multi-peak mass model (16-entry Lambda) on the same catalogue: value+gradient
    calls at K points drawn around the paper's Table 2 values, default launch shape."""
    import torch
    lam = torch.tensor(synth.lambda_batch(K, purpose=4, model="multipeak"), device="cuda")
    with g.Context(cat, max_K=K, mass_model="multipeak") as ctx:
        out = g._outputs(K, ctx.n_events, lam.device, True, lam.shape[1])
        for _ in range(2):
            g.loglik_grad(ctx._ctx, lam, ctx.n_events, stream, out)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            g.loglik_grad(ctx._ctx, lam, ctx.n_events, stream, out)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
    return {"K": K, "n_params": 16, "ms_per_call": ms, "value": n_evals * K / (ms / 1e3),
            "unit": "evals/s (value+gradient)"}


# The reference arm's sample per step: enough events that every core has several (the
# oracle runs events in parallel, and injections in chunks of about n_inj / (4 cores)),
# about 3 s of work per step on 16 cores
REF_EVENTS = 64


def run_reference(args):
    """--impl reference: the oracle timed on the host cores, one bounded sample per step."""
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    import oracle
    from paper_2605_23538_gb300 import synth
    oracle.build()
    cat = synth.catalogue(WORKLOAD)
    lam = synth.lambda_batch(K_LAMBDA, purpose=4)
    cores = os.cpu_count() or 1
    n_ev = max(REF_EVENTS, 4 * cores)
    sub, evals = oracle_sample(cat, n_ev)
    n_inj = len(sub["inj_m1"])
    for w in range(args.warmup):
        oracle.loglik(sub, lam[w % K_LAMBDA:w % K_LAMBDA + 1], grad=True, n_threads=cores)
    t0 = time.perf_counter()
    for s in range(args.steps):
        k = (args.warmup + s) % K_LAMBDA
        oracle.loglik(sub, lam[k:k + 1], grad=True, n_threads=cores)
    dt = time.perf_counter() - t0
    value = evals * args.steps / dt
    sample = (f"per step 1 Lambda of the bench's batch x ({int(sub['offsets'][-1])} samples of the first "
              f"{n_ev} events + the first {n_inj} injections, the workload's mix), FP64 value+gradient")
    line = {"metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD_NAMES[WORKLOAD], "K": K_LAMBDA, "sample": sample},
            "cpu_baseline": {"value": value, "unit": "evals/s", "cores": cores, "kind": "oracle",
                             "sample": sample, "host": host_description()},
            "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gwc", choices=["gwc", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--plain-k", type=int, default=32, help="Lambda points timed on the plain path")
    ap.add_argument("--workload", default=WORKLOAD, choices=["c1", "c2", "c3", "c5"],
                    help="catalogue size (c3 = the O5-scale headline; c1, c2 for small profiling cases)")
    ap.add_argument("--K", type=int, default=K_LAMBDA, help="Lambda points per call")
    ap.add_argument("--no-tune", action="store_true", help="keep the default launch shape")
    ap.add_argument("--no-extras", action="store_true",
                    help="time only the value+gradient step (no value-only, plain or e2e legs)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    import paper_2605_23538_gb300 as g
    from paper_2605_23538_gb300 import build, shard, synth
    if rank == 0:
        build.build()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    K = args.K
    cat = synth.catalogue(args.workload)
    log(f"[rank {rank}] catalogue {time.perf_counter() - t0:.1f} s: {len(cat['m1'])} samples, "
        f"{len(cat['inj_m1'])} injections, LOS {cat['los'].shape}")
    n_s, n_i = len(cat["m1"]), len(cat["inj_m1"])
    ctx = g.Context(cat, max_K=K)
    info = ctx.info()
    # each rank evaluates its own Lambda batch over the full catalogue (weak scaling)
    lam_np = shard.rank_rows(shard.world_batch(K, world, lambda n: synth.lambda_batch(n, purpose=4)),
                             rank, world)
    lam = torch.tensor(lam_np, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    out = g._outputs(K, ctx.n_events, lam.device, True)
    # pick the launch shape (chunk, Lambda tile, warp group) on this batch, untimed
    tune = None if args.no_tune else ctx.autotune(lam, grad=True, stream=stream)
    info = ctx.info()

    def step():
        g.loglik_grad(ctx._ctx, lam, ctx.n_events, stream, out)

    for _ in range(max(args.warmup, 3)):
        step()
    barrier()
    ctx.profile_enable(True)
    ctx.profile_read()
    sampler = ClockSampler(local)
    sampler.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    barrier()
    clocks = sampler.stop()
    ms_total = ev0.elapsed_time(ev1)
    stage_ms, n_calls = ctx.profile_read()
    ctx.profile_enable(False)
    ms_total = shard.max_over_ranks(ms_total, device="cuda")
    evals_step = (n_s + n_i) * K
    value = evals_step * args.steps * world / (ms_total / 1e3)
    flags = out["flags"].cpu().numpy()
    fused_ms = stage_ms[1] / max(n_calls, 1)
    # untimed: which stages the batch's evaluations reach (to charge each only its work),
    # and the arithmetic units' measured rates
    census = ctx.path_census(lam, stream)
    work = work_from_census(census, grad=True)
    peaks = measure_alu_peaks(g, stream, local)
    roof = alu_roofline(work, fused_ms / 1e3, peaks, (clocks or {}).get("sm_mhz"))
    roof["traffic"] = traffic_for(args.workload, K)
    roof["census"] = census

    value_only = plain = e2e = graph_line = hmc_line = None
    if not args.no_extras:
        # value-only throughput (same batch)
        outv = g._outputs(K, ctx.n_events, lam.device, False)
        for _ in range(2):
            g.loglik(ctx._ctx, lam, ctx.n_events, stream, outv)
        barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            g.loglik(ctx._ctx, lam, ctx.n_events, stream, outv)
        ev1.record(stream)
        barrier()
        value_only = evals_step * args.steps / (ev0.elapsed_time(ev1) / 1e3)

        # the plain single-Lambda FP32 path, value+gradient, on the first plain_k points
        kp = max(1, min(args.plain_k, K))
        lam_p = lam[:kp].contiguous()
        outp = g._outputs(kp, ctx.n_events, lam.device, True)
        g.loglik_plain(ctx._ctx, lam_p, ctx.n_events, True, stream, outp)
        barrier()
        ev0.record(stream)
        psteps = 2
        for _ in range(psteps):
            g.loglik_plain(ctx._ctx, lam_p, ctx.n_events, True, stream, outp)
        ev1.record(stream)
        barrier()
        plain = (n_s + n_i) * kp * psteps / (ev0.elapsed_time(ev1) / 1e3)

        # the same call recorded once as a CUDA graph and replayed
        lam_g = lam.clone()
        graph = ctx.graph(lam_g, grad=True)
        for _ in range(2):
            graph.launch(stream)
        barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            graph.launch(stream)
        ev1.record(stream)
        barrier()
        g_ms = ev0.elapsed_time(ev1) / args.steps
        graph_line = {"value": evals_step / (g_ms / 1e3), "unit": "evals/s", "ms_per_step": g_ms}
        graph.close()

        # end to end through the host-memory entry point (Lambda in, totals and gradient out)
        for _ in range(2):
            ctx.loglik_grad_host(lam_np)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ctx.loglik_grad_host(lam_np)
        e2e_s = time.perf_counter() - t0
        e2e = {"value": evals_step * args.steps / e2e_s, "unit": "evals/s",
               "h2d_bytes_per_step": K * 13 * 8,
               "d2h_bytes_per_step": K * 8 + K * 4 + K * 13 * 8}

    kde_line = mp_line = None
    if not args.no_extras:
        hmc_line = hmc_c1(g, synth, stream)
        kde_line = kde_timing(g, ctx, lam, n_s + n_i, stream, peaks)
        mp_line = multipeak_timing(g, synth, cat, K, n_s + n_i, stream)

    base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.no_extras:
        import oracle
        oracle.build()
        base = cpu_baseline(cat, lam_np)

    if rank == 0:
        mpeaks, src = load_peaks()
        line = {
            "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms_total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_NAMES[args.workload],
                       "K": K, "n_samples": n_s, "n_injections": n_i,
                       "evals_per_step": evals_step, "parallelism": f"lambda-batch x{world}",
                       "l2": "inputs larger than L2 (resident catalogue %.2f GB), no flush"
                             % (info["device_bytes"] / 1e9),
                       "chunk": info["chunk"], "n_items": info["n_items"],
                       "lambda_tile": None if tune is None else tune["lambda_tile"],
                       "lambda_group": None if tune is None else tune["lambda_group"],
                       "autotuned": tune is not None},
            "roofline": roof,
            "alu_peaks": peaks,
            "stage_ms_per_step": {"prologue": stage_ms[0] / max(n_calls, 1), "fused": fused_ms,
                                  "merge": stage_ms[2] / max(n_calls, 1)},
            "gpu_launches": 3 * args.steps,
            "kernel_digest": kernel_digest(),
            "flags_nonzero": int(np.count_nonzero(flags)),
            "peaks": {"source": src, "hbm_gbs": mpeaks.get("hbm_gbs")},
        }
        if value_only is not None:
            line["value_only"] = {"value": value_only, "unit": "evals/s"}
            line["plain_gpu"] = {"value": plain, "unit": "evals/s", "K": kp,
                                 "speedup": value / world / plain}
            line["e2e"] = e2e
            line["graph"] = graph_line
            line["hmc_c1"] = hmc_line
            line["kde"] = kde_line
            line["multipeak"] = mp_line
        if clocks is not None:
            line["clocks"] = clocks
        if base is not None:
            line["cpu_baseline"] = base
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
