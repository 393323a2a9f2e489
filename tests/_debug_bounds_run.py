"""Runs tiny likelihood and gradient cases through the bounds-checked library and prints one JSON
line: the index-violation report after the cases, the parity results against the oracle, and the
report after the self-test.  Started by tests/test_gpu_debug_bounds.py in a child process with
LISA_DEBUG_BOUNDS=1 (the debug library is then the only copy of the library in the process)."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2507_06300_gb300 import binding as B  # noqa: E402
from paper_2507_06300_gb300 import synth  # noqa: E402
from tests._workloads import (fp32_tolerance, fp32_tolerance_full, gpu_eval, oracle_batched,  # noqa: E402
                              oracle_dataset_full)
from tests.test_gpu_grad import gpu_grad, oracle_grad_batched  # noqa: E402

FP32, FP64 = 0, 1


def worst(err, tol):
    """The largest err / tol (0 where err is 0, inf where a zero bound is exceeded)."""
    if not err.size:
        return 0.0
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.where(err == 0, 0.0, err / tol)
    return float(np.max(r))


def diagonal_case(wl):
    """log L (FP32, FP64) and the gradient (FP32, FP64) against the oracle; returns the worst
    error as a fraction of each bound (<= 1 passes)."""
    P, L, St = oracle_batched(wl)
    ok = St == 0
    out = {"states_ok": int(ok.sum())}
    L64, S64 = gpu_eval(wl, P, FP64)
    L32, S32 = gpu_eval(wl, P, FP32)
    out["status_equal"] = bool(np.array_equal(S64 & ~32, St & ~32) and np.array_equal(S32 & ~32, St & ~32))
    out["fp64_rel"] = float(np.max(np.abs(L64[ok] - L[ok]) / np.abs(L[ok])))
    out["fp32_frac_of_bound"] = worst(np.abs(L32[ok] - L[ok]), fp32_tolerance(L, wl, P)[ok])
    G_ref, G_sc = oracle_grad_batched(wl, P)
    # the gradient bounds of tests/test_gpu_grad.py (FP64: 1e-12 of each component's condition
    # scale; FP32: 1e-5 of it), with floors relative to the state's largest component for
    # components whose per-bin contributions are all exactly zero in the oracle (condition scale
    # 0: a knot whose move changes no bin's value, e.g. between equal amplitudes, where the moment
    # method sums nonzero interval terms that cancel): 1e-14 in FP64, 1e-9 in FP32 (the FP32
    # moments' rounding in that cancellation; the 64-bin case meets it at 2e-10)
    gmax = np.abs(G_ref[ok]).max(axis=1, keepdims=True)
    for name, prec in (("grad64", FP64), ("grad32", FP32)):
        Lg, G, Sg, _ = gpu_grad(wl, P, prec)
        if prec == FP64:
            bound = 1e-12 * G_sc[ok] + 1e-14 * gmax
        else:
            bound = 1e-5 * G_sc[ok] + 1e-9 * gmax
        err = np.abs(G[ok] - G_ref[ok])
        out[name + "_frac_of_bound"] = worst(err, bound)
        with np.errstate(divide="ignore", invalid="ignore"):
            r = np.where(err == 0, 0.0, err / bound)
        si, ci = np.unravel_index(int(np.argmax(r)), r.shape)
        out[name + "_worst"] = {"state": int(np.flatnonzero(ok)[si]), "component": int(ci), "err": float(err[si, ci]),
                                "bound": float(bound[si, ci]), "ref": float(G_ref[ok][si, ci]),
                                "scale": float(G_sc[ok][si, ci]), "state_max": float(gmax[si, 0])}
    return out


def main():
    assert B.debug_requested(), "LISA_DEBUG_BOUNDS=1 must be set"
    res = {"enabled": B.debug_bounds_enabled()}
    B.debug_bounds(reset=True)
    cases = {}
    # 64 bins, 3 states (A,E,T with a power-law SGWB)
    cases["tiny64"] = diagonal_case(synth.workload("tiny", n_bins=64, n_states=3))
    # prior draws with close knot pairs: the routed (compensated) path and the fallback pass
    wl = synth.workload("tiny", n_bins=3000, n_states=24, kmin=2, kmax_draw=8, theta_mode="prior")
    wl.f_ref[:] = 3e-3
    rng = np.random.default_rng(11)
    k = wl.knots
    for s in range(0, wl.n_states, 3):
        for a in range(wl.n_splines):
            if k.count[s, a] >= 2:
                k.x[s, a, 1] = k.x[s, a, 0] + rng.uniform(2e-5, 2e-4) * (1 if k.x[s, a, 0] < -2 else -1)
    cases["prior_close_knots"] = diagonal_case(wl)
    # the dense covariance, 64 bins, 3 states
    wf = synth.workload("tiny", cov_model=1, n_bins=64, n_states=3)
    ds = oracle_dataset_full(wf)
    Lr, Sr = oracle.loglike_full(ds, wf.theta, wf.knots.as_dict())
    okf = Sr == 0
    L64, _ = gpu_eval(wf, ds["P9"], FP64)
    L32, _ = gpu_eval(wf, ds["P9"], FP32)
    cases["full64"] = {"states_ok": int(okf.sum()),
                       "fp64_rel": float(np.max(np.abs(L64[okf] - Lr[okf]) / np.abs(Lr[okf]))),
                       "fp32_frac_of_bound": worst(np.abs(L32[okf] - Lr[okf]),
                                                   fp32_tolerance_full(Lr, wf, ds["P9"])[okf])}
    res["cases"] = cases
    res["after_cases"] = B.debug_bounds(reset=True)
    B.debug_bounds_selftest()
    res["after_selftest"] = B.debug_bounds(reset=True)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
