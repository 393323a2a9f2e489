"""Measurement helpers of the library: pipe-rate microbenchmark and per-kernel timing."""
import numpy as np
import pytest

from paper_2507_06300_gb300 import synth
from tests._workloads import oracle_batched

pytestmark = pytest.mark.gpu


def test_pipe_rates_are_positive_and_plausible():
    from paper_2507_06300_gb300 import binding as B
    r = B.pipe_rates(iters=256, reps=1)
    assert set(r) == set(B.PIPE_OPS)
    for k, v in r.items():
        # lane operations per second on a whole GPU: well above 1e11 and below 1e15
        assert 1e11 < v < 1e15, (k, v)
    assert r["ffma2"] >= 0.5 * r["ffma"]
    # the fused kernel's mix (38 packed FP32 ops, 8 ex2, 2 rcp, 2 lg2 per two state-bins): no
    # faster than either pipe alone allows, no slower than the two pipes one after the other
    t_fma = 38.0 * 2.0 / r["ffma2"] / 2.0                       # seconds per state-bin
    t_lg2 = max(2.0 / r["lg2_ex2"] - 1.0 / r["ex2"], 1.0 / r["ex2"])
    t_mufu = (4.0 / r["ex2"] + 1.0 / r["rcp"] + t_lg2)
    assert r["mix"] <= 1.05 / max(t_fma, t_mufu), r
    assert r["mix"] >= 0.9 / (t_fma + t_mufu), r


def test_kernel_times_of_a_recorded_call():
    import torch
    from paper_2507_06300_gb300 import binding as B
    wl = synth.workload("tiny", n_bins=3000, n_states=24)
    P, _, _ = oracle_batched(wl)
    ds = B.Dataset.from_workload(wl, P)
    count, x, w, kmax, kind = B.knots_to_device(wl.knots)
    theta = torch.as_tensor(wl.theta, device="cuda")
    with pytest.raises(B.LisaError):
        ds.kernel_ms()                                  # profiling is off
    for prec in (B.FP32, B.FP64):
        buf, _ = ds.spline_setup(count, x, w, kmax, kind, prec)
        ref = ds.psd_loglike(theta, buf, kmax, prec).clone()
        ds.set_profiling(True)
        out = ds.psd_loglike(theta, buf, kmax, prec)
        ms = ds.kernel_ms()
        ds.set_profiling(False)
        assert len(ms) == 3 and ms[0] > 0 and ms[2] > 0 and ms[1] >= 0
        if prec == B.FP64:
            assert ms[1] < 0.05                         # no compensated kernel in FP64 mode
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), ref.cpu().numpy())
    ds.close()


def test_kernel_times_of_a_recorded_gradient_call():
    import torch
    from paper_2507_06300_gb300 import binding as B
    wl = synth.workload("tiny", n_bins=3000, n_states=24)
    P, _, _ = oracle_batched(wl)
    ds = B.Dataset.from_workload(wl, P)
    count, x, w, kmax, kind = B.knots_to_device(wl.knots)
    theta = torch.as_tensor(wl.theta, device="cuda")
    buf, _ = ds.spline_setup(count, x, w, kmax, kind, B.FP32)
    L0, G0 = ds.psd_loglike_grad(theta, count, x, w, kmax, kind, buf, B.FP32)
    L0, G0 = L0.clone(), G0.clone()
    ds.set_profiling(True)
    L1, G1 = ds.psd_loglike_grad(theta, count, x, w, kmax, kind, buf, B.FP32)
    ms = ds.kernel_ms()
    ds.set_profiling(False)
    assert ms[0] > 0 and ms[2] > 0 and ms[1] < 0.05
    torch.cuda.synchronize()
    np.testing.assert_array_equal(L1.cpu().numpy(), L0.cpu().numpy())
    np.testing.assert_array_equal(G1.cpu().numpy(), G0.cpu().numpy())
    ds.close()
