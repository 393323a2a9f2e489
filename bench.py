#!/usr/bin/env python
"""Benchmark of the batched, spline-perturbed Whittle/Wishart log-likelihood on GB300.

One step = one pass of the hot path over the paper-scale workload: spline setup (knot sort,
Akima slopes, coefficients) for every state, then the fused FP32-bulk likelihood (spline
evaluation, PSD assembly, per-bin terms, FP64 reduction) -- A, E, T; 131,072 bins uniform in
0.1-29 mHz; nu = 64; 64 walkers x 16 temperatures = 1,024 states; 0-20 in-between knots per
spline.  Data are synthetic (seeded Gamma-averaged periodogram around the injected PSD).

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle instead (the
only other place this script executes ``oracle/``), on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Whittle logL state-bins/s: batched FP32 vs plain FP64, % of roofline"
UNIT = "state-bins/s"
WORKLOAD = ("paper-scale: A,E,T; 131,072 uniform bins 0.1-29 mHz; Nseg=64; OMS 15 pm + TM 3 fm/s^2 + "
            "power-law SGWB log10 Omega=-12, n_t=2/3; 64 walkers x 16 temps = 1,024 states; 0-20 knots per spline")
# Algorithmic operations per state-bin of the fused FP32 kernel as implemented for A,E,T with an
# SGWB.  MUFU: 4 ex2 (three noise perturbations, one SGWB perturbation x power law), 1 rcp (fused
# reciprocal sum), 1 lg2 (fused log of the product).  FP32 (FMA pipe, an FMA counted once):
# 4 splines x (1 shift + 3 Horner FMA) = 16, SGWB exponent and amplitude 2, per channel noise
# (2) and PSD (2) = 12, channel product and reciprocal-sum numerator 4, reciprocal-sum FMA and
# the two nu-weighted accumulations (of the reciprocal sum and of the log) 3; ln2 and the keep
# factor are applied once per 64-bin chunk.
MUFU_EX2, MUFU_RCP, MUFU_LG2 = 4, 1, 1
MUFU_PER_STATE_BIN = MUFU_EX2 + MUFU_RCP + MUFU_LG2
FP32_PER_STATE_BIN = 37
TABLE_BYTES_PER_BIN = 12 * 4          # FP32 bin table: x, ell, nu, 3 x (G_oms, G_tm, G_h)
# The FP32 adjoint kernel per state-bin, as implemented: per spline a compensated t (two-sum and
# low parts, 9), Horner 3 and moments 6 = 72; SGWB exponent and amplitude 2; per channel noise 2,
# SGWB 1, PSD 1, g / nu = r (r - 1) 1, g E 1, forward and channel product 2, template sums 3,
# spline signal 1 = 12 (11 for the first channel) = 35; the log of the product 3 (range test and
# FMA); nu times the bin's forward, template and SGWB sums 4, SGWB accumulators 2; nu times the
# noise splines' signals 3 -- 121.  MUFU: 4 ex2, 3 rcp, 1 lg2 (of the channel product).
ADJ_FP32_PER_STATE_BIN = 121
# When every bin lies inside the knot band and |log10 f_lo| <= 2.9 |log10 f_hi| (the library's
# exactness test for t = x - x_o in FP32), t takes 3 ops instead of 9 per spline: 97 in all.
ADJ_FP32_PER_STATE_BIN_EXACT_T = 97
ADJ_MUFU = (4, 3, 1)
# FP64-pipe instructions per state-bin of the plain FP64 kernel as implemented (the library's exp10,
# exp2, log and divisions included), counted by ncu on a 131,072-bin x 64-state A,E,T case
FP64_PIPE_PER_STATE_BIN = 225


def adjoint_exact_t(wl) -> bool:
    """The condition under which the FP32 adjoint forms t without a two-sum (same rule as the
    library): bins inside [x_lo, x_hi], one sign, and |x_lo| <= 2.9 |x_hi| (for negative x)."""
    for d in range(wl.n_datasets):
        b0, b1 = int(wl.bin_offset[d]), int(wl.bin_offset[d + 1])
        if b1 == b0:
            continue
        xa, xb = math.log10(wl.f[b0]), math.log10(wl.f[b1 - 1])
        lo, hi = float(wl.x_lo[d]), float(wl.x_hi[d])
        if not (lo <= xa and xb <= hi):
            return False
        if hi < 0.0:
            if not -lo <= 2.9 * -hi:
                return False
        elif lo > 0.0:
            if not hi <= 2.9 * lo:
                return False
        else:
            return False
    return True
SPLINE_RECORD_BYTES = 64


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def _traffic_from_profile(kernel_src):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on this source."""
    prof = os.path.join(ROOT, "profiles", "loglike_fp32_paper.md")
    if not os.path.exists(prof):
        return None
    txt = open(prof).read()
    m_h = re.search(r"source_sha256:\s*([0-9a-f]{16,64})", txt)
    m_b = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    if not (m_h and m_b):
        return None
    h = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()
    return float(m_b.group(1)) if h.startswith(m_h.group(1)) else None


def make_periodogram_gpu(wl, B, torch):
    """P = S_model(theta_true of its dataset) x Gamma(nu)/nu for every dataset of the workload,
    the model PSD from the library's FP64 path; returns a host array [C, N_total]."""
    D, C, N = wl.n_datasets, wl.n_channels, wl.n_bins
    ds0 = B.Dataset(n_channels=C, freq=wl.f, nu=wl.nu, periodogram=wl.gamma,
                    response=wl.R if wl.sgwb_model else None, bin_offset=wl.bin_offset,
                    state_offset=np.arange(D + 1, dtype=np.int64), x_lo=wl.x_lo, x_hi=wl.x_hi,
                    f_ref=wl.f_ref, sgwb_model=wl.sgwb_model, tdi_form=wl.tdi_form)
    nsp = wl.n_splines
    c = torch.zeros((D, nsp), dtype=torch.int32, device="cuda")
    x = torch.zeros((D, nsp, 0), dtype=torch.float64, device="cuda")
    w = torch.zeros((D, nsp, 2), dtype=torch.float64, device="cuda")
    buf, _ = ds0.spline_setup(c, x, w, 0, 0, B.FP64)
    th = torch.as_tensor(wl.theta_true, device="cuda")
    S = ds0.model_psd(th, buf, 0)                 # dataset d: [C][N_d] at offset C * b0
    P = torch.empty((C, N), dtype=torch.float64, device="cuda")
    for d in range(D):
        b0, b1 = int(wl.bin_offset[d]), int(wl.bin_offset[d + 1])
        P[:, b0:b1] = S[C * b0:C * b1].view(C, b1 - b0)
    del S
    P *= torch.as_tensor(wl.gamma, device="cuda")
    out = P.cpu().numpy()
    ds0.close()
    return out


# The dense-covariance FP32 kernel per state-bin as implemented (A,E,T, power-law SGWB, fast path),
# FP32-pipe instructions: seven splines x (shift + 3 Horner FMA) = 28; SGWB exponent and amplitude 3;
# per channel D 4, H 1, C_cc 1 and the two range checks = 24; 1 / C_cc from one reciprocal 8; g^2, h 6;
# r, s from z 9; R_ET 3; e, s_AT s_ET, the 2x2 minors and s0 s1 s2 9; adjugate diagonal and det K 21;
# off-diagonal adjugate brackets 11; sqrt(D_a D_b) and the off-diagonal trace terms 18; diagonal
# trace terms and numerator 6; cancellation and det checks 8; the log's product, term and nu 6;
# accumulation 1 -- 161.  MUFU: 4 ex2, 6 rsqrt (z -> r, s and sqrt(D_a D_b)), 2 rcp (the product
# of the C_cc, det K), 1 lg2.
FULL_FP32_PER_STATE_BIN = 161
FULL_MUFU = {"ex2": 4, "rsqrt": 6, "rcp": 2, "lg2": 1}


def colour_periodogram(cov6, W9):
    """The averaged periodogram matrix L W L^T per bin (L the Cholesky factor of the injected
    covariance, W the workload's unit complex Wishart draws), as [9, N]: P_AA, P_EE, P_TT and the
    real and imaginary parts of P_AE, P_AT, P_ET."""
    N = cov6.shape[1]
    C = np.empty((N, 3, 3))
    C[:, 0, 0], C[:, 1, 1], C[:, 2, 2] = cov6[0], cov6[1], cov6[2]
    C[:, 0, 1] = C[:, 1, 0] = cov6[3]
    C[:, 0, 2] = C[:, 2, 0] = cov6[4]
    C[:, 1, 2] = C[:, 2, 1] = cov6[5]
    L = np.linalg.cholesky(C)
    W = np.zeros((N, 3, 3), dtype=np.complex128)
    W[:, 0, 0], W[:, 1, 1], W[:, 2, 2] = W9[0], W9[1], W9[2]
    for k, (a, b) in enumerate(((0, 1), (0, 2), (1, 2))):
        W[:, a, b] = W9[3 + 2 * k] + 1j * W9[4 + 2 * k]
        W[:, b, a] = np.conj(W[:, a, b])
    Pm = L @ W @ np.transpose(L, (0, 2, 1))
    out = np.empty((9, N))
    out[0], out[1], out[2] = Pm[:, 0, 0].real, Pm[:, 1, 1].real, Pm[:, 2, 2].real
    for k, (a, b) in enumerate(((0, 1), (0, 2), (1, 2))):
        out[3 + 2 * k], out[4 + 2 * k] = Pm[:, a, b].real, Pm[:, a, b].imag
    return out


def host_mem_available_gb():
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) / 1e6
    except OSError:
        pass
    return float("inf")


def roofs(rates, hbm_gbs, bytes_per_state_bin):
    """Ceilings in state-bins/s of the fused kernel from the measured pipe rates: the MUFU pipe
    (the kernel's mix of 4 ex2, 1 rcp, 1 lg2), the FP32 FMA pipe (37 ops, packed FMAs counted as
    two lane operations) and HBM (algorithmic bytes per state-bin)."""
    t_ex2, t_rcp = 1.0 / rates["ex2"], 1.0 / rates["rcp"]
    t_lg2 = 2.0 / rates["lg2_ex2"] - t_ex2
    if not t_lg2 > 0:
        t_lg2 = t_ex2
    mufu = 1.0 / (MUFU_EX2 * t_ex2 + MUFU_RCP * t_rcp + MUFU_LG2 * t_lg2)
    fp32_rate = max(rates["ffma"], rates["ffma2"])
    return {"mufu": mufu, "mufu_rate": MUFU_PER_STATE_BIN * mufu, "fp32": fp32_rate / FP32_PER_STATE_BIN,
            "fp32_rate": fp32_rate, "hbm": hbm_gbs * 1e9 / bytes_per_state_bin}


def roofline_entry(sb_per_s, R, hbm_gbs, bytes_per_state_bin):
    """Roofline object of the binding ceiling for a measured state-bin rate."""
    bind = min(("fp32", "mufu", "hbm"), key=lambda k: R[k])
    if bind == "hbm":
        ach = sb_per_s * bytes_per_state_bin / 1e9
        return {"bound": "hbm", "achieved": ach, "peak": hbm_gbs, "unit": "GB/s", "frac": ach / hbm_gbs}
    ops, rate, pipe = ((FP32_PER_STATE_BIN, R["fp32_rate"], "FP32 (FMA pipe)") if bind == "fp32"
                       else (MUFU_PER_STATE_BIN, R["mufu_rate"], "MUFU (XU pipe)"))
    ach = ops * sb_per_s / 1e9
    return {"bound": "alu", "pipe": pipe, "achieved": ach, "peak": rate / 1e9, "unit": "Gop/s",
            "frac": ach / (rate / 1e9), "ops_per_state_bin": ops}


def cpu_oracle_rate(wl, P, budget_s, first=0, stride=1):
    """The FP64 oracle as it stands, single-threaded, on whole states of the workload (states
    first, first + stride, ...) until ``budget_s`` seconds of CPU work are spent; returns
    (state-bins/s, states timed, seconds)."""
    import oracle
    oracle.build()
    ds = wl.dataset(0)
    ds["P"] = P
    n = 0
    t0 = time.perf_counter()
    while True:
        s = (first + n * stride) % wl.n_states
        th, kn = wl.theta[s:s + 1], {k: (v[s:s + 1] if isinstance(v, np.ndarray) else v)
                                     for k, v in wl.knots.as_dict().items()}
        oracle.loglike(ds, th, kn)
        n += 1
        el = time.perf_counter() - t0
        if el >= budget_s or n >= wl.n_states:
            break
    return n * wl.n_bins / el, n, el


def _oracle_worker(args):
    """One process of the all-core oracle timing (started with spawn: no inherited CUDA state)."""
    P, budget_s, first, stride = args
    from paper_2507_06300_gb300 import synth
    wl = synth.workload("paper")
    _, n, el = cpu_oracle_rate(wl, P, budget_s, first, stride)
    return n, el


def cpu_oracle_all_cores(wl, P, budget_s, cores):
    """The same oracle on every host core at once, one process per core, each on its own states;
    returns (state-bins/s of all processes together, states timed, wall seconds)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_worker, [(P, budget_s, k, cores) for k in range(cores)])
    wall = time.perf_counter() - t0
    n = sum(r[0] for r in res)
    span = max(r[1] for r in res)        # each process's own timed span (imports excluded)
    return n * wl.n_bins / span, n, wall


def host_cpu_info():
    """Core count and CPU model of the host (lscpu, else /proc/cpuinfo)."""
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return cores, model or "unknown", os.uname().machine


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_2507_06300_gb300 import synth
    import oracle
    wl = synth.workload("paper")
    ds = wl.dataset(0)
    zero = {"count": np.zeros((1, wl.n_splines), np.int32), "x": np.zeros((1, wl.n_splines, 1)),
            "w": np.zeros((1, wl.n_splines, 2)), "kmax": 0, "kind": 0}
    S, _ = oracle.model_psd(ds, wl.theta_true, zero)
    P = S[0] * wl.gamma
    per_step_states = max(1, int(args.ref_states))
    ds["P"] = P
    times = []
    rng_states = np.arange(wl.n_states)
    for k in range(args.warmup + args.steps):
        sel = rng_states[(k * per_step_states) % wl.n_states:][:per_step_states]
        th = wl.theta[sel]
        kn = {kk: (v[sel] if isinstance(v, np.ndarray) else v) for kk, v in wl.knots.as_dict().items()}
        t0 = time.perf_counter()
        oracle.loglike(ds, th, kn)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
    sb = per_step_states * wl.n_bins
    ms = 1e3 * sum(times) / len(times)
    value = sb / (ms / 1e3)
    sample = f"{per_step_states} whole state(s) x {wl.n_bins} bins per step of the paper-scale workload"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2507_06300_gb300 import autotune
    from paper_2507_06300_gb300 import binding as B
    from paper_2507_06300_gb300 import replicas, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def rank_max(vals):
        """Max over ranks of each value (timings: the slowest replica sets the job's time)."""
        return replicas.max_over_ranks(vals, dist if world > 1 else None, device="cuda")

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > 129 MB L2
    peaks, peak_kind = _peaks()
    rates = B.pipe_rates()            # measured MUFU / FP32 pipe rates (outside any timed region)
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        gpu_id = vis.split(",")[local] if vis else str(local)

    def prepare(wl, tiling, P=None, groups=autotune.DEFAULT_GROUPS):
        P = make_periodogram_gpu(wl, B, torch) if P is None else P
        ds = B.Dataset.from_workload(wl, P)
        count, x, w, kmax, kind = B.knots_to_device(wl.knots)
        theta = torch.as_tensor(wl.theta, device="cuda")
        if tiling:
            tb, sc, g = (int(v) for v in tiling.split(","))
            best = dict(tile_bins=tb, states_per_cta=sc, group=g, ctas_per_sm=0)
            ds.set_tiling(**best)
            table = [(best, float("nan"))]
        else:
            # tile shapes picked by the autotuner on these inputs (outside the timed region)
            best, table = autotune.autotune(ds, theta, count, x, w, kmax, kind, B.FP32, groups=groups)
            table.sort(key=lambda r: r[1])
        so, bo = wl.state_offset, wl.bin_offset
        nbin_state = np.repeat(np.diff(bo), np.diff(so))           # bins of each state's dataset
        alg_bytes = (TABLE_BYTES_PER_BIN * wl.n_bins + wl.n_states * 8 * B.N_THETA +
                     wl.n_states * wl.n_splines * (kmax + 1) * SPLINE_RECORD_BYTES)
        P = P[:3] if P.shape[0] == 9 else P      # the diagonal: normalisation and the scale of the bound
        return dict(wl=wl, P=P, ds=ds, count=count, x=x, w=w, kmax=kmax, kind=kind, theta=theta, tiling=best,
                    table=table, sb=int(nbin_state.sum()), nbin_state=nbin_state, alg_bytes=alg_bytes)

    def release(I):
        I["ds"].close()
        I.clear()
        torch.cuda.synchronize()
        torch.cuda.empty_cache()

    def timed(ev, steps, warmup, soak_s=0.0):
        for _ in range(warmup):
            flush.fill_(1.0)
            ev.replay()
        torch.cuda.synchronize()
        if soak_s > 0:
            # untimed replays of the same step (L2 flushed between them) for ~soak_s seconds, so
            # that the clock sampler running around this call sees the GPU under this load for
            # more than a couple of samples even when the timed region itself is short
            t_end = time.perf_counter() + soak_s
            while time.perf_counter() < t_end:
                for _ in range(20):
                    flush.fill_(1.0)
                    ev.replay()
                torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
              torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for k in range(steps):
            flush.fill_(float(k))
            e[k][0].record()
            ev.g_setup.replay()
            e[k][1].record()
            ev.g_ll.replay()
            e[k][2].record()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        step_ms = [a.elapsed_time(c) for a, b, c in e]
        ll_ms = [b.elapsed_time(c) for a, b, c in e]
        return sum(step_ms) / steps, sum(ll_ms) / steps

    def kernel_times(I, ev, steps):
        """Device time of each likelihood kernel (events recorded by the library on the launching
        stream around each kernel) over uncaptured calls, L2 flushed before each."""
        ds = I["ds"]
        ds.set_profiling(True)
        acc = np.zeros(3)
        for k in range(steps):
            flush.fill_(float(k))
            ev.setup()
            ev.loglike()
            acc += np.array(ds.kernel_ms())
        ds.set_profiling(False)
        return (acc / steps).tolist()

    def forward(I, steps, warmup, fp64_steps, sample_clocks=False, sharded=False):
        """FP32 (graphs, timed) and plain FP64 on the same inputs, per-kernel times, accuracy.
        Replicas (sharded=False) each run the whole workload; sharded runs split it."""
        ds, wl, kmax, kind = I["ds"], I["wl"], I["kmax"], I["kind"]
        ev32 = B.Evaluator(ds, kmax, kind, B.FP32)
        ev32.load(I["theta"], I["count"], I["x"], I["w"])
        ev32.capture()
        routed = ds.routed_list(ev32.buf)
        clocks = None
        if sample_clocks:
            with ClockSampler(gpu_id) as clk:
                ms, ll_ms = timed(ev32, steps, warmup, soak_s=1.0)
            clocks = clk.summary()
            clocks["window"] = "1 s of untimed replays of the same step, then the timed steps"
        else:
            ms, ll_ms = timed(ev32, steps, warmup)
        ms, ll_ms = rank_max([ms, ll_ms])
        kt = rank_max(kernel_times(I, ev32, max(3, min(steps // 2, 400))))
        ev64 = B.Evaluator(ds, kmax, kind, B.FP64)
        ev64.load(I["theta"], I["count"], I["x"], I["w"])
        ev64.capture()
        ms64, ll64 = rank_max(timed(ev64, max(1, fp64_steps), 1))
        # accuracy of the FP32 path against the FP64 GPU path on every state
        L32 = ev32.replay().clone()
        L64 = ev64.replay().clone()
        torch.cuda.synchronize()
        L32, L64 = L32.cpu().numpy(), L64.cpu().numpy()
        bo, so, P = wl.bin_offset, wl.state_offset, I["P"]
        lnP = wl.nu * np.log(P).sum(axis=0)
        K_d = -np.add.reduceat(lnP, bo[:-1])
        Cnu_d = wl.n_channels * np.add.reduceat(wl.nu, bo[:-1])
        ds_of = np.repeat(np.arange(wl.n_datasets), np.diff(so))
        ok = np.isfinite(L64)
        scale = np.maximum(np.abs(L64 - K_d[ds_of]), Cnu_d[ds_of])[ok]
        err = np.abs(L32[ok] - L64[ok])
        wk = int(np.flatnonzero(ok)[np.argmax(err / scale)])    # worst state relative to the bound
        sb = I["sb"]
        sb_fused = sb - int(I["nbin_state"][routed].sum())
        sb_job = (replicas.sum_over_ranks([sb], dist if world > 1 else None, device="cuda")[0] if sharded
                  else world * sb)
        r = {"value": sb_job / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "loglike_ms": ll_ms,
             "setup_ms": ms - ll_ms, "state_bins_per_step": sb, "routed_states": len(routed),
             "kernel_ms": {"fused_fp32": kt[0], "compensated": kt[1], "finalize": kt[2]},
             "fused_state_bins": sb_fused,
             "fp64_plain": {"value": sb_job / (ms64 / 1e3), "unit": UNIT, "ms_per_step": ms64,
                            "loglike_ms": ll64, "steps": max(1, fp64_steps)},
             "accuracy_fp32_vs_fp64": {"max_abs_nats": float(err.max()), "median_abs_nats": float(np.median(err)),
                                       "max_rel_to_scale": float((err / scale).max()), "states": int(ok.sum())},
             "worst_state": {"state": wk, "L32": float(L32[wk]), "L64": float(L64[wk]),
                             "scale": float(max(abs(L64[wk] - K_d[ds_of[wk]]), Cnu_d[ds_of[wk]]))},
             "tiling": I["tiling"], "autotune_top": [[t, round(v, 4)] for t, v in I["table"][:5]]}
        r["speedup_fp32_vs_fp64"] = r["value"] / r["fp64_plain"]["value"]
        fp64_rate = (sb / (ll64 / 1e3)) * FP64_PIPE_PER_STATE_BIN    # FP64-pipe instructions per second
        r["fp64_plain"]["roofline"] = {
            "bound": "alu", "pipe": "FP64", "achieved": fp64_rate / 1e9, "peak": rates["dfma"] / 1e9, "unit": "Gop/s",
            "frac": fp64_rate / rates["dfma"], "ops_per_state_bin": FP64_PIPE_PER_STATE_BIN,
            "ops_source": "ncu thread-level FP64-pipe instruction count per state-bin (profiles/loglike_fp64_ops.md)",
            "peak_source": "measured live by lisa_pipe_rates (fma.rn.f64)", "timing": "the likelihood graph only"}
        return r, ev32, clocks

    def roofline_of(I, r):
        bpsb = I["alg_bytes"] / I["sb"]
        R = roofs(rates, peaks["hbm_gbs"], bpsb)
        fused_rate = r["fused_state_bins"] / (r["kernel_ms"]["fused_fp32"] / 1e3)
        ent = roofline_entry(fused_rate, R, peaks["hbm_gbs"], bpsb)
        ent.update({"kernel": "loglike_fp32_kernel (fused FP32 likelihood)",
                    "ceilings_state_bins_per_s": {"fp32": R["fp32"], "mufu": R["mufu"], "hbm": R["hbm"]},
                    # the kernel's own mix of FMA-pipe and MUFU work run as independent chains: the
                    # two pipes overlap only in part, so the mix is slower than either pipe alone
                    "mixed_pipe": {"ceiling_state_bins_per_s": rates["mix"], "frac": fused_rate / rates["mix"],
                                   "ceiling_vs_fp32_alone": rates["mix"] / R["fp32"],
                                   "mix": "per two state-bins: 37 packed FP32 ops, 8 ex2, 2 rcp, 2 lg2",
                                   "source": "lisa_pipe_rates LISA_PIPE_MIX, measured live"},
                    "mufu_frac": fused_rate / R["mufu"], "hbm_frac": fused_rate / R["hbm"],
                    "step_frac": (r["value"] / world) / min(R["fp32"], R["mufu"], R["hbm"]),
                    "hbm_algorithmic_bytes_per_state_bin": bpsb})
        return ent

    # ---- the headline: paper-scale workload ----------------------------------------------------
    wl = synth.workload("paper")
    I = prepare(wl, args.tiling)
    head, ev32, clocks = forward(I, args.steps, args.warmup, args.fp64_steps, sample_clocks=True)
    roof = roofline_of(I, head)
    roof["peak_source"] = ("measured live by lisa_pipe_rates: FP32 = max(fma.rn.f32, fma.rn.f32x2) lane-op rate, "
                           "MUFU = the kernel's 4 ex2 + 1 rcp + 1 lg2 mix; HBM = MEASURED_PEAKS.json "
                           f"({peak_kind})")
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    roof["nominal_fp32_gops"] = n_sm * 128 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e9
    roof["n_sm"] = n_sm
    roof["traffic"] = _traffic_from_profile(os.path.join(ROOT, "paper_2507_06300_gb300", "csrc", "lisa_loglike.cu"))
    if roof["traffic"] is not None:
        roof["traffic_vs_algorithmic_bytes"] = roof["traffic"] / I["alg_bytes"]

    # end to end through the public API: pinned host inputs -> device -> log L back in pinned memory
    S = wl.n_states
    # the sampler's proposals written into the evaluator's pinned input block (one copy per call)
    h_theta, h_count, h_x, h_w = ev32.host_inputs()
    for h, t in zip((h_theta, h_count, h_x, h_w), (I["theta"], I["count"], I["x"], I["w"])):
        h.copy_(t.cpu())
    h_out = torch.empty(S, dtype=torch.float64).pin_memory()
    ev32.capture_host(h_theta, h_count, h_x, h_w, h_out)   # copies in, setup, log L, copy out: one graph
    for _ in range(args.warmup):
        ev32.loglike_host(h_theta, h_count, h_x, h_w, h_out)
    torch.cuda.synchronize()
    e2e_ms, e2e_wall = [], []
    for k in range(args.steps):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        a.record()
        ev32.loglike_host(h_theta, h_count, h_x, h_w, h_out)   # returns once log L is on the host
        b.record()
        e2e_wall.append(1e3 * (time.perf_counter() - t0))
        torch.cuda.synchronize()
        e2e_ms.append(a.elapsed_time(b))
    e2e, e2e_w = rank_max([sum(e2e_ms) / len(e2e_ms), sum(e2e_wall) / len(e2e_wall)])
    h2d = ev32.h_inputs.numel() * ev32.h_inputs.element_size()   # the pinned block copied each call
    d2h = h_out.numel() * h_out.element_size()
    P_head = I["P"]
    release(I)

    line = {"metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_bins": wl.n_bins, "n_states": S, "n_channels": wl.n_channels,
                       "kmax": int(wl.knots.kmax), "precision": "fp32-bulk, fp64 sums",
                       "l2": "flushed (256 MB write) between timed steps", "cuda_graph": True,
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "tiling": head["tiling"], "autotune_top": head["autotune_top"]},
            "fp64_plain": head["fp64_plain"], "speedup_fp32_vs_fp64": head["speedup_fp32_vs_fp64"],
            "accuracy_fp32_vs_fp64": head["accuracy_fp32_vs_fp64"],
            "loglike_ms": head["loglike_ms"], "setup_ms": head["setup_ms"], "routed_states": head["routed_states"],
            "kernel_ms": head["kernel_ms"], "roofline": roof, "pipe_rates_lane_ops_per_s": rates,
            "e2e": {"value": world * head["state_bins_per_step"] / (e2e / 1e3), "unit": UNIT,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e,
                    "host_wall_ms_per_step": e2e_w,
                    "timing": "CUDA events on the calling stream around the public call (copy in, setup, "
                              "log L, copy out, host synchronisation); the second event is recorded after "
                              "the call returns, so the span includes the host's wake-up after the copy out; "
                              "host_wall_ms_per_step is perf_counter around the same call"},
            # per step: spline_setup_kernel (setup graph), then the state-parameter, fused,
            # compensated and finalize kernels (likelihood graph)
            "gpu_launches": 5 * args.steps,
            "clocks": clocks}

    # ---- adjoint: 256 walkers x 8 temperatures, 12 + 8 knots ------------------------------------
    if "adjoint" in args.extras:
        wla = synth.workload("adjoint")
        Ia = prepare(wla, "")
        ds, kmax, kind = Ia["ds"], Ia["kmax"], Ia["kind"]
        Sa = wla.n_states

        def timed_grad(prec, steps):
            gbuf = torch.empty(ds.spline_buf_bytes(kmax, prec), dtype=torch.uint8, device="cuda")
            gws = torch.empty(ds.workspace_bytes(kmax, prec, True), dtype=torch.uint8, device="cuda")
            gout = torch.empty(Sa, dtype=torch.float64, device="cuda")
            ggr = torch.empty((Sa, B.N_THETA + ds.n_splines * (2 * kmax + 2)), dtype=torch.float64, device="cuda")

            def one():
                ds.spline_setup(Ia["count"], Ia["x"], Ia["w"], kmax, kind, prec, buf=gbuf)
                ds.psd_loglike_grad(Ia["theta"], Ia["count"], Ia["x"], Ia["w"], kmax, kind, gbuf, prec, out=gout,
                                    grad=ggr, workspace=gws)
            for _ in range(2):
                one()
            torch.cuda.synchronize()
            tot = 0.0
            for k in range(steps):
                flush.fill_(float(k))
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                one()
                b.record()
                torch.cuda.synchronize()
                tot += a.elapsed_time(b)
            return rank_max([tot / steps])[0], gout.cpu().numpy(), ggr.cpu().numpy()

        g32_ms, L32, G32 = timed_grad(B.FP32, max(3, min(args.steps // 2, 200)))
        g64_ms, L64, G64 = timed_grad(B.FP64, 1)
        ok = np.isfinite(L64)
        gscale = np.maximum(np.abs(G64[ok]).max(axis=1, keepdims=True), 1e-300)
        rel = np.abs(G32[ok] - G64[ok]) / gscale
        # components not dominated by cancellation (at least 1e-3 of their state's largest): error
        # relative to the component itself
        big = np.abs(G64[ok]) >= 1e-3 * gscale
        rel_c = (np.abs(G32[ok] - G64[ok])[big] / np.abs(G64[ok])[big]) if big.any() else np.zeros(1)

        # the adjoint kernel's own device time (library events, uncaptured calls, L2 flushed)
        kbuf = torch.empty(ds.spline_buf_bytes(kmax, B.FP32), dtype=torch.uint8, device="cuda")
        kws = torch.empty(ds.workspace_bytes(kmax, B.FP32, True), dtype=torch.uint8, device="cuda")
        ds.spline_setup(Ia["count"], Ia["x"], Ia["w"], kmax, kind, B.FP32, buf=kbuf)
        ds.set_profiling(True)
        kacc = np.zeros(3)
        nk = max(3, min(args.steps // 2, 200))
        for k in range(nk):
            flush.fill_(float(k))
            ds.psd_loglike_grad(Ia["theta"], Ia["count"], Ia["x"], Ia["w"], kmax, kind, kbuf, B.FP32, workspace=kws)
            kacc += np.array(ds.kernel_ms())
        ds.set_profiling(False)
        kadj = rank_max(list(kacc / nk))
        adj_rate = Ia["sb"] / (kadj[0] / 1e3)
        t_mufu = (ADJ_MUFU[0] / rates["ex2"] + ADJ_MUFU[1] / rates["rcp"] +
                  ADJ_MUFU[2] * max(2.0 / rates["lg2_ex2"] - 1.0 / rates["ex2"], 1.0 / rates["ex2"]))
        fp32_rate = max(rates["ffma"], rates["ffma2"])
        adj_ops = ADJ_FP32_PER_STATE_BIN_EXACT_T if adjoint_exact_t(wla) else ADJ_FP32_PER_STATE_BIN
        ceil_fp32, ceil_mufu = fp32_rate / adj_ops, 1.0 / t_mufu
        line["adjoint"] = {
            "workload": "A,E,T; 131,072 bins; 256 walkers x 8 temps = 2,048 states; 12 noise + 8 SGWB knots",
            "what": "spline setup + log L and its gradient for every state (lisa_psd_loglike_grad)",
            "unit": UNIT, "fp32_value": world * Ia["sb"] / (g32_ms / 1e3), "fp32_ms_per_step": g32_ms,
            "fp64_value": world * Ia["sb"] / (g64_ms / 1e3), "fp64_ms_per_step": g64_ms,
            "speedup_fp32_vs_fp64": g64_ms / g32_ms,
            "kernel_ms": {"adjoint_fp32": kadj[0], "compensated_and_fallback": kadj[1], "epilogue": kadj[2]},
            "grad_fp32_vs_fp64": {"median_rel_to_state_max": float(np.median(rel)),
                                  "p99_rel_to_state_max": float(np.quantile(rel, 0.99)),
                                  "components_above_1e-3_of_state_max": int(big.sum()),
                                  "their_median_rel": float(np.median(rel_c)),
                                  "their_p99_rel": float(np.quantile(rel_c, 0.99)),
                                  "their_max_rel": float(rel_c.max()),
                                  "note": "per-component bound checked by the tests: 1e-5 of the oracle's "
                                          "condition scale (sum over bins of |per-bin contribution|)"},
            "roofline": {"bound": "alu", "pipe": "FP32 (FMA pipe)" if ceil_fp32 <= ceil_mufu else "MUFU (XU pipe)",
                         "kernel": "adjoint_fp32_kernel",
                         "achieved": adj_ops * adj_rate / 1e9 if ceil_fp32 <= ceil_mufu
                         else sum(ADJ_MUFU) * adj_rate / 1e9,
                         "peak": fp32_rate / 1e9 if ceil_fp32 <= ceil_mufu else sum(ADJ_MUFU) * ceil_mufu / 1e9,
                         "unit": "Gop/s", "frac": adj_rate / min(ceil_fp32, ceil_mufu),
                         "ops_per_state_bin": adj_ops,
                         "ceilings_state_bins_per_s": {"fp32": ceil_fp32, "mufu": ceil_mufu}},
            "l2": "flushed between timed steps"}
        release(Ia)

    # ---- data preparation: synthesis + averaged periodogram at the paper-scale sizes ---------------
    if "prep" in args.extras and rank == 0:
        C_p, nb_p, n_p = 3, 131072, 64
        N_p = nb_p * n_p
        gp = torch.Generator(device="cuda").manual_seed(20250706)
        S_p = torch.rand((C_p, N_p), dtype=torch.float64, device="cuda", generator=gp) + 0.5
        z_p = torch.randn((C_p, N_p, 2), dtype=torch.float64, device="cuda", generator=gp)
        d_p = torch.empty_like(z_p)
        off_p = torch.arange(0, N_p + 1, n_p, dtype=torch.int64, device="cuda")

        def ev_time(fn, reps):
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(reps):
                fn()
            b.record()
            torch.cuda.synchronize()
            return a.elapsed_time(b) / reps

        ms_syn = ev_time(lambda: B.fd_synthesize(S_p, z_p, out=d_p), 10)
        ms_avg = ev_time(lambda: B.averaged_periodogram(d_p, 1e-4, 3.17e-8, off_p), 10)
        by_syn = C_p * N_p * (8 + 16 + 16)
        by_avg = C_p * N_p * 16 + nb_p * ((C_p + 2) * 8 + 8)
        # FP64 work per complex sample: the periodogram's two FMAs (re^2 + im^2 accumulated); the
        # synthesis is one correctly rounded FP64 square root and two multiplies (its FP64-pipe
        # issue count is not an algorithmic constant, so it is reported against HBM only)
        fl_avg = 2 * C_p * N_p
        line["prep"] = {
            "workload": "A,E,T; 131,072 bins x 64 frequency samples (8,388,608 per channel), FP64 complex; "
                        "inputs 0.4-1 GB, larger than L2",
            "fd_synthesize": {"ms": ms_syn, "bytes": by_syn,
                              "roofline": {"bound": "hbm", "achieved": by_syn / (ms_syn / 1e3) / 1e9, "peak": peaks["hbm_gbs"],
                                           "unit": "GB/s", "frac": by_syn / (ms_syn / 1e3) / 1e9 / peaks["hbm_gbs"]}},
            "averaged_periodogram": {"ms": ms_avg, "bytes": by_avg, "bins_per_s": nb_p / (ms_avg / 1e3),
                                     "roofline": {"bound": "alu", "pipe": "FP64 (DFMA)",
                                                  "achieved": fl_avg / (ms_avg / 1e3) / 1e9,
                                                  "peak": rates["dfma"] / 1e9, "unit": "Gop/s",
                                                  "frac": fl_avg / (ms_avg / 1e3) / rates["dfma"],
                                                  "peak_source": "measured live by lisa_pipe_rates (fma.rn.f64)"},
                                     "hbm": {"achieved_gbs": by_avg / (ms_avg / 1e3) / 1e9,
                                             "frac": by_avg / (ms_avg / 1e3) / 1e9 / peaks["hbm_gbs"]}},
            "peak_source": f"hbm_gbs of MEASURED_PEAKS.json ({peak_kind})"}
        del S_p, z_p, d_p, off_p

    # ---- RJ-PT sampler: A,E; 2,000 bins; 32 walkers x 4 temperatures; 200 sweeps ------------------
    if "rjpt" in args.extras and rank == 0:
        from paper_2507_06300_gb300 import rjpt
        wlr = synth.workload("small_ae")
        P_r = make_periodogram_gpu(wlr, B, torch)
        ds_r = B.Dataset.from_workload(wlr, P_r)
        Tr, Wr, kmax_r, n_sw = 4, 32, 4, 200
        x_lo_r, x_hi_r = float(wlr.x_lo[0]), float(wlr.x_hi[0])
        res = {}
        for prec_name, prec in (("fp64", B.FP64), ("fp32", B.FP32)):
            smp = rjpt.RJPTSampler(rjpt.GpuLikelihood(ds_r, kmax_r, precision=prec), betas=rjpt.paper_ladder(Tr),
                                   n_walkers=Wr, n_splines=wlr.n_splines, kmax=kmax_r, k_max_rj=kmax_r, x_lo=x_lo_r,
                                   x_hi=x_hi_r, sgwb_model=1, seed=20250706, device="cpu")
            smp.init_from_prior(theta_center=wlr.theta_true[0], rel=0.01, k0=1)
            smp.run(5, n_adapt=5)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rec = smp.run(n_sw, n_adapt=n_sw // 2)
            torch.cuda.synchronize()
            el = time.perf_counter() - t0
            acc = smp.acceptance()
            lz, _ = rjpt.stepping_stone_log_z(smp.betas, rec["logL"].reshape(-1, Tr, Wr).transpose(0, 2, 1)
                                              .reshape(-1, Tr))
            res[prec_name] = {"sweeps_per_s": n_sw / el, "s_per_run": el,
                              "likelihood_calls_per_sweep": 2,
                              "state_bins_per_s_through_sampler": 2 * n_sw * Tr * Wr * wlr.n_bins / el,
                              "acceptance": {k: [round(float(v), 3) for v in acc[k]] for k in acc},
                              "cold_chain_mean_knots": float(rec["count"].mean()),
                              "log_z_stepping_stone": lz}
        line["rjpt"] = {"workload": "A,E; 2,000 bins 0.1-29 mHz; Nseg=16; 32 walkers x 4 temperatures "
                                    "(paper ladder); 0-4 in-between knots per spline; 200 sweeps (100 adapting)",
                        "what": "RJ-PT sampler, its state in host tensors (at 128 states the per-operation "
                                "launch cost of device tensors exceeds the arithmetic): MALA (gradient from "
                                "lisa_psd_loglike_grad), knot birth/death, PT swaps; every state's log L and "
                                "gradient in one library call per move",
                        **res}
        ds_r.close()

    # ---- RJ-PT sampler at the largest configuration: A,E,T; 524,288 bins; 32 x 256 walkers -------
    if "rjpt_full" in args.extras and rank == 0:
        from paper_2507_06300_gb300 import rjpt
        wlf = synth.workload("full")
        P_f = make_periodogram_gpu(wlf, B, torch)
        ds_f = B.Dataset.from_workload(wlf, P_f)
        Tf, Wf, kmax_f = 32, 256, wlf.knots.kmax
        assert Tf * Wf == wlf.n_states
        cnt_t, x_t, w_t, _, kind_f = B.knots_to_device(wlf.knots)
        th_t = torch.as_tensor(wlf.theta, device="cuda")
        best_f, _ = autotune.autotune(ds_f, th_t, cnt_t, x_t, w_t, kmax_f, kind_f, B.FP32, groups=(4,))
        like = rjpt.GpuLikelihood(ds_f, kmax_f, kind=kind_f, precision=B.FP32, sync=True)
        smp = rjpt.RJPTSampler(like, betas=rjpt.paper_ladder(Tf), n_walkers=Wf, n_splines=wlf.n_splines, kmax=kmax_f,
                               k_max_rj=kmax_f, x_lo=float(wlf.x_lo[0]), x_hi=float(wlf.x_hi[0]), sgwb_model=2,
                               seed=20250706, device="cuda")
        # the walkers start from the workload's states (prior and posterior draws, 0-40 knots)
        smp.set_state(rjpt.State(wlf.theta.copy(), wlf.knots.count.copy(), wlf.knots.x.copy(), wlf.knots.w.copy()))
        smp.run(2, n_adapt=2)
        n_sw = max(3, min(args.steps // 150, 10))
        torch.cuda.synchronize()
        g0, c0 = like.seconds, like.calls
        t0 = time.perf_counter()
        smp.run(n_sw, n_adapt=n_sw)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        g_s, n_calls = like.seconds - g0, like.calls - c0
        sb_call = wlf.n_states * wlf.n_bins
        line["rjpt_full"] = {
            "workload": "A,E,T; 524,288 bins 0.1-29 mHz; Nseg=128; broken power-law SGWB; 32 temperatures "
                        "(paper ladder) x 256 walkers = 8,192 states; 0-40 in-between knots per spline",
            "what": "RJ-PT sweeps: MALA (log L and gradient from lisa_psd_loglike_grad, FP32) + knot birth/death + "
                    "PT swaps, the sampler's state on the GPU; states start from the workload's draws; tiles "
                    "autotuned on the forward kernel",
            "sweeps": n_sw, "sweeps_per_s": n_sw / el, "s_per_sweep": el / n_sw,
            "library_calls_per_sweep": n_calls / n_sw,
            "state_bins_per_s_through_sampler": n_calls * sb_call / el,
            "library_call_share": g_s / el,
            "sampler_arithmetic_share": 1.0 - g_s / el,
            "library_call_ms": 1e3 * g_s / max(n_calls, 1),
            "note": "library_call_ms: one synchronised call (spline setup, then log L and gradient of all states, "
                    "device tensors in and out); the rest of each sweep is the sampler's proposal, prior, accept "
                    "and swap arithmetic, batched torch operations on the device launched from the host loop",
            "tiling": best_f,
            "acceptance": {k: {"coldest": round(float(a[0]), 3), "mean": round(float(np.mean(a)), 3)}
                           for k, a in smp.acceptance().items()},
        }
        del like, smp
        ds_f.close()
        del P_f, cnt_t, x_t, w_t, th_t

    # ---- batched datasets and the full-form workload ----------------------------------------------
    line["workloads"] = {}
    if "full_cov" in args.extras:
        # the dense 3x3 covariance (six flexible noise terms) on the paper-scale workload
        wlc = synth.workload("paper", cov_model=1)
        wdiag = synth.workload("paper")                   # same bins, noise and SGWB injection
        S_true = make_periodogram_gpu(dataclasses.replace(wdiag, gamma=np.ones_like(wdiag.gamma)), B, torch)
        z = np.asarray(synth.Z_INJ)
        rz, sz = z / np.sqrt(1 + z * z), 1 / np.sqrt(1 + z * z)
        Rm = {(0, 1): rz[0], (0, 2): rz[1], (1, 2): rz[0] * rz[1] + sz[0] * sz[1] * rz[2]}
        cov6 = np.empty((6, wlc.n_bins))
        cov6[:3] = S_true
        for k, (a, b) in enumerate(((0, 1), (0, 2), (1, 2))):
            cov6[3 + k] = np.sqrt(S_true[a] * S_true[b]) * Rm[(a, b)]
        P9 = colour_periodogram(cov6, wlc.wishart)
        Ic = prepare(wlc, "", P=P9, groups=(4,))
        rc, _, _ = forward(Ic, max(5, min(args.steps // 2, 200)), args.warmup, 1)
        rate = rc["state_bins_per_step"] / (rc["kernel_ms"]["fused_fp32"] / 1e3)
        fp32_rate = max(rates["ffma"], rates["ffma2"])
        t_lg2 = max(2.0 / rates["lg2_ex2"] - 1.0 / rates["ex2"], 1.0 / rates["ex2"])
        t_mufu = (FULL_MUFU["ex2"] / rates["ex2"] + (FULL_MUFU["rsqrt"] + FULL_MUFU["rcp"]) / rates["rcp"] +
                  FULL_MUFU["lg2"] * t_lg2)
        c32, cmu = fp32_rate / FULL_FP32_PER_STATE_BIN, 1.0 / t_mufu
        rc["roofline"] = {
            "bound": "alu", "pipe": "FP32 (FMA pipe)" if c32 <= cmu else "MUFU (XU pipe)",
            "kernel": "full_fp32_kernel (dense covariance)",
            "achieved": FULL_FP32_PER_STATE_BIN * rate / 1e9 if c32 <= cmu else sum(FULL_MUFU.values()) * rate / 1e9,
            "peak": fp32_rate / 1e9 if c32 <= cmu else sum(FULL_MUFU.values()) * cmu / 1e9, "unit": "Gop/s",
            "frac": rate / min(c32, cmu), "ops_per_state_bin": FULL_FP32_PER_STATE_BIN,
            "ceilings_state_bins_per_s": {"fp32": c32, "mufu": cmu},
            "mufu_ops_per_state_bin": FULL_MUFU, "note": "rsqrt taken at the measured rcp rate"}
        rc["workload"] = ("A,E,T; 131,072 bins; Nseg=64; 1,024 states; dense 3x3 covariance per bin: three "
                          "noise, one SGWB and three correlation splines per state (0-20 knots); data: complex "
                          "Wishart draws around the model PSD with constant correlations")
        line["workloads"]["full_cov"] = rc
        release(Ic)
    for name, desc in (("batched", "1,024 A,E,T datasets of 8k-262k bins, 4 x 4 states each, 0-30 knots; "
                                    "one persistent launch per kernel, CUDA graphs"),
                       ("full", "A,E,T; 524,288 bins; Nseg=128; 32 temps x 256 walkers = 8,192 states; "
                                "broken power-law SGWB (knee 3 mHz); 0-40 knots")):
        if name not in args.extras:
            continue
        if name == "batched" and host_mem_available_gb() < 48:
            line["workloads"][name] = {"workload": desc, "skipped": "less than 48 GB of host memory free"}
            continue
        wlx = synth.workload(name)
        if world > 1:             # a fixed total split across the replicas
            wlx = replicas.shard_workload(wlx, rank, world)
        Ix = prepare(wlx, "")
        rx, _, _ = forward(Ix, max(5, min(args.steps // 2, 200)), args.warmup, 1, sharded=world > 1)
        rx["roofline"] = roofline_of(Ix, rx)
        rx["workload"] = desc
        rx["scaling"] = "strong" if world > 1 else "single GPU"
        line["workloads"][name] = rx
        release(Ix)
        del wlx

    if rank == 0 and not args.no_cpu_baseline:
        cores, cpu_model, arch = host_cpu_info()
        # the state where FP32 and FP64 disagree most (relative to the FP32 bound), checked by the
        # FP64 oracle on the host
        import oracle
        ws_ = head["worst_state"]
        s_ = ws_["state"]
        ds_ = wl.dataset(0)
        ds_["P"] = P_head
        L_or, _ = oracle.loglike(ds_, wl.theta[s_:s_ + 1],
                                 {k: (v[s_:s_ + 1] if isinstance(v, np.ndarray) else v)
                                  for k, v in wl.knots.as_dict().items()})
        line["accuracy_fp32_vs_fp64"]["worst_state_vs_oracle"] = {
            "state": s_, "fp32_minus_oracle_nats": ws_["L32"] - float(L_or[0]),
            "fp64_minus_oracle_nats": ws_["L64"] - float(L_or[0]),
            "fp32_rel_to_scale": abs(ws_["L32"] - float(L_or[0])) / ws_["scale"], "bound": 1e-6}
        rate, n, el = cpu_oracle_rate(wl, P_head, args.cpu_seconds)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"{n} whole state(s) x {wl.n_bins} bins of the same workload, {el:.1f} s",
                                "nproc": cores, "cpu_model": cpu_model, "arch": arch}
        if cores > 1 and args.cpu_seconds > 0:
            rate_all, n_all, wall = cpu_oracle_all_cores(wl, P_head, args.cpu_seconds, cores)
            line["cpu_baseline"]["all_cores"] = {
                "value": rate_all, "unit": UNIT, "cores": cores,
                "sample": f"{n_all} whole states x {wl.n_bins} bins, one process per core (spawned), "
                          f"each on its own states for ~{args.cpu_seconds:.0f} s; {wall:.1f} s wall"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    # default: 1,500 steps of ~0.35 ms, a timed region of about half a second
    ap.add_argument("--steps", type=int, default=1500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-states", type=int, default=4, help="states per reference step")
    ap.add_argument("--tiling", default="", help="tile_bins,states_per_cta,group (skips the autotuner)")
    ap.add_argument("--extras", default="adjoint,prep,rjpt,batched,full,full_cov,rjpt_full",
                    help="comma-separated extra workloads to measure: adjoint, prep, rjpt, batched, full, full_cov, "
                         "rjpt_full")
    ap.add_argument("--no-extras", action="store_true", help="measure the headline workload only")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    args.extras = set() if args.no_extras else {e.strip() for e in args.extras.split(",") if e.strip()}
    if not args.extras <= {"adjoint", "prep", "rjpt", "batched", "full", "full_cov", "rjpt_full"}:
        ap.error("--extras takes adjoint, prep, rjpt, batched, full, full_cov, rjpt_full")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
