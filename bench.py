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
# Algorithmic MUFU (SFU) operations per state-bin of the fused FP32 kernel as implemented for
# A,E,T with an SGWB: 4 ex2 (three noise perturbations, one SGWB perturbation x power law),
# 1 rcp (fused reciprocal sum), 1 lg2 (fused log of the product).
MUFU_PER_STATE_BIN = 6
MUFU_PER_SM_PER_CLK = 16           # XU lanes per SM per clock
N_SM = 152


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
    """P = S_model(theta_true) x Gamma(nu)/nu with the model PSD from the library (FP64 path)."""
    ones = np.ones((wl.n_channels, wl.n_bins))
    ds0 = B.Dataset(n_channels=wl.n_channels, freq=wl.f, nu=wl.nu, periodogram=ones,
                    response=wl.R if wl.sgwb_model else None, n_states=1, x_lo=wl.x_lo, x_hi=wl.x_hi,
                    f_ref=wl.f_ref, sgwb_model=wl.sgwb_model, tdi_form=wl.tdi_form)
    nsp = wl.n_splines
    c = torch.zeros((1, nsp), dtype=torch.int32, device="cuda")
    x = torch.zeros((1, nsp, 0), dtype=torch.float64, device="cuda")
    w = torch.zeros((1, nsp, 2), dtype=torch.float64, device="cuda")
    buf, _ = ds0.spline_setup(c, x, w, 0, 0, B.FP64)
    th = torch.as_tensor(wl.theta_true[:1], device="cuda")
    S = ds0.model_psd(th, buf, 0).reshape(wl.n_channels, wl.n_bins)
    P = (S * torch.as_tensor(wl.gamma, device="cuda")).cpu().numpy()
    ds0.close()
    return P


def cpu_oracle_rate(wl, P, budget_s):
    """The FP64 oracle as it stands, single-threaded, on whole states of the workload until
    ``budget_s`` seconds of CPU work are spent; returns (state-bins/s, states timed, seconds)."""
    import oracle
    oracle.build()
    ds = wl.dataset(0)
    ds["P"] = P
    n = 0
    t0 = time.perf_counter()
    while True:
        th, kn = wl.theta[n:n + 1], {k: (v[n:n + 1] if isinstance(v, np.ndarray) else v)
                                     for k, v in wl.knots.as_dict().items()}
        oracle.loglike(ds, th, kn)
        n += 1
        el = time.perf_counter() - t0
        if el >= budget_s or n >= wl.n_states:
            break
    return n * wl.n_bins / el, n, el


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

    from paper_2507_06300_gb300 import binding as B
    from paper_2507_06300_gb300 import synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    wl = synth.workload("paper")
    P = make_periodogram_gpu(wl, B, torch)
    ds = B.Dataset.from_workload(wl, P)
    count, x, w, kmax, kind = B.knots_to_device(wl.knots)
    theta = torch.as_tensor(wl.theta, device="cuda")
    S, N = wl.n_states, wl.n_bins
    sb_per_step = S * N

    # tile shapes picked by the autotuner on these inputs (outside the timed region)
    from paper_2507_06300_gb300 import autotune
    if args.tiling:
        tb, sc, g = (int(v) for v in args.tiling.split(","))
        best = dict(tile_bins=tb, states_per_cta=sc, group=g, ctas_per_sm=0)
        ds.set_tiling(**best)
        table = [(best, float("nan"))]
    else:
        best, table = autotune.autotune(ds, theta, count, x, w, kmax, kind, B.FP32)
        table.sort(key=lambda r: r[1])

    ev32 = B.Evaluator(ds, kmax, kind, B.FP32)
    ev32.load(theta, count, x, w)
    ev32.capture()
    routed = ds.routed_states(ev32.buf)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > 129 MB L2

    def timed(ev, steps, warmup):
        for _ in range(warmup):
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

    peaks, peak_kind = _peaks()
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        gpu_id = vis.split(",")[local] if vis else str(local)
    with ClockSampler(gpu_id) as clk:
        ms, ll_ms = timed(ev32, args.steps, args.warmup)
    clocks = clk.summary()
    if world > 1:
        t = torch.tensor([ms, ll_ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms, ll_ms = t.tolist()
    value = world * sb_per_step / (ms / 1e3)

    # plain FP64 path on the same inputs (fewer steps: it is much slower)
    ev64 = B.Evaluator(ds, kmax, kind, B.FP64)
    ev64.load(theta, count, x, w)
    ev64.capture()
    ms64, ll64 = timed(ev64, max(1, args.fp64_steps), 1)
    value64 = world * sb_per_step / (ms64 / 1e3)

    # adjoint (log L and its gradient for every state), FP32 and plain FP64, eager launches
    def timed_grad(prec, steps):
        gbuf = torch.empty(ds.spline_buf_bytes(kmax, prec), dtype=torch.uint8, device="cuda")
        gws = torch.empty(ds.workspace_bytes(kmax, prec, True), dtype=torch.uint8, device="cuda")
        gout = torch.empty(S, dtype=torch.float64, device="cuda")
        ggr = torch.empty((S, B.N_THETA + ds.n_splines * (2 * kmax + 2)), dtype=torch.float64, device="cuda")
        def one():
            ds.spline_setup(count, x, w, kmax, kind, prec, buf=gbuf)
            ds.psd_loglike_grad(theta, count, x, w, kmax, kind, gbuf, prec, out=gout, grad=ggr, workspace=gws)
        for _ in range(2):
            one()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(steps):
            one()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / steps
    grad32_ms = timed_grad(B.FP32, max(3, args.steps // 2))
    grad64_ms = timed_grad(B.FP64, 1)

    # accuracy of the FP32 path against the FP64 GPU path on every state
    L32 = ev32.replay().clone()
    L64 = ev64.replay().clone()
    torch.cuda.synchronize()
    L32, L64 = L32.cpu().numpy(), L64.cpu().numpy()
    ok = np.isfinite(L64)
    K = -np.sum(wl.nu * np.log(P).sum(axis=0))
    scale = np.maximum(np.abs(L64[ok] - K), wl.n_channels * wl.nu.sum())
    err = np.abs(L32[ok] - L64[ok])

    # end to end through the public API: pinned host inputs -> device -> log L back in pinned memory
    pin = lambda t: t.cpu().pin_memory()
    h_theta, h_count, h_x, h_w = pin(theta), pin(count), pin(x), pin(w)
    h_out = torch.empty(S, dtype=torch.float64).pin_memory()
    for _ in range(args.warmup):
        ev32.loglike_host(h_theta, h_count, h_x, h_w, h_out)
    torch.cuda.synchronize()
    e2e_ms = []
    for k in range(args.steps):
        flush.fill_(float(k))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        ev32.loglike_host(h_theta, h_count, h_x, h_w, h_out)
        b.record()
        torch.cuda.synchronize()
        e2e_ms.append(a.elapsed_time(b))
    e2e = sum(e2e_ms) / len(e2e_ms)
    if world > 1:
        t = torch.tensor([e2e], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e = t.item()
    h2d = sum(t.numel() * t.element_size() for t in (h_theta, h_count, h_x, h_w))
    d2h = h_out.numel() * h_out.element_size()

    # roofline of the dominant kernel (fused FP32 likelihood): MUFU issue bound
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    mufu_peak = N_SM * MUFU_PER_SM_PER_CLK * sm_max * 1e6 / 1e9   # Gop/s
    achieved = MUFU_PER_STATE_BIN * sb_per_step / (ll_ms / 1e3) / 1e9
    traffic = _traffic_from_profile(os.path.join(ROOT, "paper_2507_06300_gb300", "csrc", "lisa_loglike.cu"))
    hbm_alg = N * 12 * 4 + S * 8 + S * wl.n_splines * (kmax + 1) * 32   # bytes per launch (algorithmic)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_bins": N, "n_states": S, "n_channels": wl.n_channels,
                       "kmax": kmax, "precision": "fp32-bulk, fp64 sums", "l2": "flushed (256 MB write) "
                       "between timed steps", "cuda_graph": True,
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "tiling": best, "autotune_top": [[t, round(ms, 4)] for t, ms in table[:5]]},
            "fp64_plain": {"value": value64, "unit": UNIT, "ms_per_step": ms64, "steps": max(1, args.fp64_steps),
                           "loglike_ms": ll64},
            "speedup_fp32_vs_fp64": value / value64,
            "adjoint": {"unit": UNIT, "fp32_value": world * sb_per_step / (grad32_ms / 1e3), "fp32_ms_per_step": grad32_ms,
                        "fp64_value": world * sb_per_step / (grad64_ms / 1e3), "fp64_ms_per_step": grad64_ms,
                        "what": "spline setup + log L and gradient for every state (lisa_psd_loglike_grad)"},
            "accuracy_fp32_vs_fp64": {"max_abs_nats": float(err.max()), "median_abs_nats": float(np.median(err)),
                                      "max_rel_to_scale": float((err / scale).max()), "states": int(ok.sum())},
            "loglike_ms": ll_ms, "setup_ms": ms - ll_ms, "routed_states": routed,
            "roofline": {"bound": "alu", "pipe": "MUFU (XU)", "achieved": achieved, "peak": mufu_peak,
                         "unit": "Gop/s", "frac": achieved / mufu_peak, "traffic": traffic,
                         "peak_source": f"derived: {N_SM} SMs x {MUFU_PER_SM_PER_CLK} MUFU/clk x {sm_max:.0f} MHz",
                         "ops_per_state_bin": MUFU_PER_STATE_BIN,
                         "hbm_algorithmic_bytes_per_launch": hbm_alg,
                         "hbm_frac": (hbm_alg / (ll_ms / 1e3) / 1e9) / peaks["hbm_gbs"],
                         "hbm_peak_gbs": peaks["hbm_gbs"], "hbm_peak_kind": peak_kind},
            "e2e": {"value": world * sb_per_step / (e2e / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e},
            # per step: spline_setup_kernel (setup graph), then the fused, compensated and finalize
            # kernels (likelihood graph)
            "gpu_launches": 4 * args.steps,
            "clocks": clocks}
    if rank == 0 and not args.no_cpu_baseline:
        rate, n, el = cpu_oracle_rate(wl, P, args.cpu_seconds)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"{n} whole state(s) x {N} bins of the same workload, {el:.1f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ds.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-states", type=int, default=4, help="states per reference step")
    ap.add_argument("--tiling", default="", help="tile_bins,states_per_cta,group (skips the autotuner)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
