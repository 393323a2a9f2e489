"""The preallocated Evaluator (the path bench.py times): device-resident steps, the two captured
CUDA graphs (FP32) and the end-to-end call from pinned host buffers all give the same log L,
bit for bit (the reductions are deterministic), and that log L agrees with the oracle."""
import numpy as np
import pytest

from paper_2507_06300_gb300 import synth
from tests._workloads import fp32_tolerance, oracle_batched

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [1, 0])
def test_evaluator_step_graph_and_host_paths_agree(precision):
    import torch
    from paper_2507_06300_gb300 import binding as B
    wl = synth.workload("small_ae")
    P, L_or, St_or = oracle_batched(wl)
    ds = B.Dataset.from_workload(wl, P)
    count, x, w, kmax, kind = B.knots_to_device(wl.knots)
    theta = torch.as_tensor(wl.theta, device="cuda")
    ev = B.Evaluator(ds, kmax, kind, precision)
    ev.load(theta, count, x, w)
    stepped = ev.step().cpu().numpy().copy()
    replayed = stepped
    if precision == 0:                                   # the FP32 path is the one bench.py captures
        ev.capture()
        ev.out.fill_(0.0)
        replayed = ev.replay().cpu().numpy().copy()
    pin = lambda t: t.cpu().pin_memory()
    h_out = torch.empty(wl.n_states, dtype=torch.float64).pin_memory()
    ev.out.fill_(0.0)
    ev.theta.zero_()                                     # the host call must bring the inputs in
    got = ev.loglike_host(pin(theta), pin(count), pin(x), pin(w), h_out).numpy().copy()
    np.testing.assert_array_equal(replayed, stepped)
    np.testing.assert_array_equal(got, stepped)
    ok = St_or == 0
    assert np.array_equal(np.isneginf(stepped), ~ok)
    if precision == 1:
        np.testing.assert_allclose(stepped[ok], L_or[ok], rtol=1e-12, atol=0)
    else:
        tol = fp32_tolerance(L_or, wl, P)
        assert np.all(np.abs(stepped[ok] - L_or[ok]) <= tol[ok])
    ds.close()


def test_captured_host_call_copies_fresh_inputs_every_replay():
    import torch
    from paper_2507_06300_gb300 import binding as B
    wl = synth.workload("small_ae")
    P, _, _ = oracle_batched(wl)
    ds = B.Dataset.from_workload(wl, P)
    count, x, w, kmax, kind = B.knots_to_device(wl.knots)
    theta = torch.as_tensor(wl.theta, device="cuda")
    ev = B.Evaluator(ds, kmax, kind, 0).capture()
    pin = lambda t: t.cpu().pin_memory()
    h_theta, h_count, h_x, h_w = pin(theta), pin(count), pin(x), pin(w)
    h_out = torch.empty(wl.n_states, dtype=torch.float64).pin_memory()
    ev.capture_host(h_theta, h_count, h_x, h_w, h_out)
    first = ev.loglike_host(h_theta, h_count, h_x, h_w, h_out).numpy().copy()
    ev.load(theta, count, x, w)
    np.testing.assert_array_equal(first, ev.replay().cpu().numpy())
    # new values in the same pinned buffers: the replay must read them
    h_theta[:, 0] *= 1.25
    h_w[:, 0, 0] += 0.05
    second = ev.loglike_host(h_theta, h_count, h_x, h_w, h_out).numpy().copy()
    ev.load(h_theta.cuda(), count, x, h_w.cuda())
    np.testing.assert_array_equal(second, ev.replay().cpu().numpy())
    assert not np.array_equal(first, second)
    ds.close()


def test_host_input_block_is_copied_in_one_transfer_with_the_same_result():
    import torch
    from paper_2507_06300_gb300 import binding as B
    wl = synth.workload("small_ae")
    P, _, _ = oracle_batched(wl)
    ds = B.Dataset.from_workload(wl, P)
    count, x, w, kmax, kind = B.knots_to_device(wl.knots)
    theta = torch.as_tensor(wl.theta, device="cuda")
    ev = B.Evaluator(ds, kmax, kind, 0).capture()
    ev.load(theta, count, x, w)
    ref = ev.replay().cpu().numpy().copy()
    h = ev.host_inputs()
    for dst, src in zip(h, (theta, count, x, w)):
        dst.copy_(src.cpu())
    h_out = torch.empty(wl.n_states, dtype=torch.float64).pin_memory()
    ev.inputs.zero_()
    np.testing.assert_array_equal(ev.loglike_host(*h, h_out).numpy(), ref)      # eager, one copy
    ev.capture_host(*h, h_out)
    ev.inputs.zero_()
    np.testing.assert_array_equal(ev.loglike_host(*h, h_out).numpy(), ref)      # captured
    h[0][:, 1] *= 0.8
    got = ev.loglike_host(*h, h_out).numpy().copy()
    ev.load(h[0].cuda(), count, x, w)
    np.testing.assert_array_equal(got, ev.replay().cpu().numpy())
    assert not np.array_equal(got, ref)
    ds.close()
