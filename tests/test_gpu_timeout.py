"""The bounded-wait timeout path of the fused likelihood kernel, made to run out on purpose.

The fused FP32 kernel stages each work item's bin table into shared memory with an asynchronous
bulk copy and waits for it on an mbarrier with a bounded number of polls.  A wait that runs out
must not hang the GPU, fault or let the CTA write partial sums from a table it never received:
the kernel raises the workspace's error word, lets the copies it issued land and stops.  Here the
test switch of lisa_data_set_test_wait makes the kernel issue no copy at all, so its first wait
runs out with nothing in flight (a barrier that nothing will ever complete), with a short poll
limit.  The host then reads LISA_ERR_TIMEOUT from lisa_workspace_status, every log L of that call
is NaN, and the same data object, workspace and CUDA context give the normal result afterwards."""
import numpy as np
import pytest

from paper_2507_06300_gb300 import synth
from tests._workloads import oracle_batched

pytestmark = pytest.mark.gpu

LISA_ERR_TIMEOUT = 8


def test_fused_kernel_wait_runs_out_and_reports_timeout():
    import torch
    from paper_2507_06300_gb300 import binding as B
    wl = synth.workload("small_ae")
    P, L_or, St_or = oracle_batched(wl)
    ds = B.Dataset.from_workload(wl, P)
    count, x, w, kmax, kind = B.knots_to_device(wl.knots)
    theta = torch.as_tensor(wl.theta, device="cuda")
    buf, st = ds.spline_setup(count, x, w, kmax, kind, B.FP32)
    ws = torch.empty(ds.workspace_bytes(kmax, B.FP32), dtype=torch.uint8, device="cuda")
    ref = ds.psd_loglike(theta, buf, kmax, B.FP32, workspace=ws).cpu().numpy()
    assert ds.workspace_status(ws) == 0
    ok = St_or == 0
    assert ok.sum() > 100 and np.all(np.isfinite(ref[ok]))

    ds.set_test_wait(skip_copies=True, wait_limit=1 << 12)
    bad = ds.psd_loglike(theta, buf, kmax, B.FP32, workspace=ws).cpu().numpy()
    assert ds.workspace_status(ws) == LISA_ERR_TIMEOUT
    assert np.all(np.isnan(bad[ok]))

    ds.set_test_wait(skip_copies=False, wait_limit=1 << 20)
    again = ds.psd_loglike(theta, buf, kmax, B.FP32, workspace=ws).cpu().numpy()
    assert ds.workspace_status(ws) == 0
    np.testing.assert_array_equal(again, ref)
    ds.close()


def test_pageable_host_tensors_are_refused_by_the_end_to_end_call():
    import torch
    from paper_2507_06300_gb300 import binding as B
    wl = synth.workload("tiny")
    ds = B.Dataset.from_workload(wl, np.ones((3, wl.n_bins)))
    count, x, w, kmax, kind = B.knots_to_device(wl.knots)
    ev = B.Evaluator(ds, kmax, kind, B.FP32)
    out = torch.empty(wl.n_states, dtype=torch.float64)
    with pytest.raises(B.LisaError, match="pinned"):
        ev.loglike_host(torch.as_tensor(wl.theta), count.cpu(), x.cpu(), w.cpu(), out)
    ds.close()
