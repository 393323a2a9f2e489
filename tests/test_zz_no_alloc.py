"""The allocation-free entry point (lisa_psd_loglike_noalloc) against lisa_psd_loglike.

lisa_psd_loglike_noalloc is for callers that cannot hand the library a scratch workspace (a
device heap already owned by another framework, a fixed memory budget, a plain C host sampler):
it keeps its scratch in a fixed 4 MiB array inside the library.  This file is collected last on
purpose; it must pass both alone in a fresh process and after the other GPU tests."""
import numpy as np
import pytest

from paper_2507_06300_gb300 import synth
from tests._workloads import fp32_tolerance, oracle_batched

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [1, 0])
def test_noalloc_matches_workspace_entry_point_twice(precision):
    import torch
    from paper_2507_06300_gb300 import binding as B
    wl = synth.workload("small_ae")
    P, L_or, St_or = oracle_batched(wl)
    ds = B.Dataset.from_workload(wl, P)
    assert ds.workspace_bytes(wl.knots.kmax, precision) <= B.NOALLOC_SCRATCH_BYTES
    count, x, w, kmax, kind = B.knots_to_device(wl.knots)
    theta = torch.as_tensor(wl.theta, device="cuda")
    buf, st = ds.spline_setup(count, x, w, kmax, kind, precision)
    ref = ds.psd_loglike(theta, buf, kmax, precision).cpu().numpy()
    ok = St_or == 0
    assert ok.sum() > 100
    # the workspace entry point against the oracle, in the tolerance of its precision
    if precision == 1:
        np.testing.assert_allclose(ref[ok], L_or[ok], rtol=1e-12, atol=0)
    else:
        assert np.all(np.abs(ref[ok] - L_or[ok]) <= fp32_tolerance(L_or, wl, P)[ok])
    for _ in range(2):                      # two calls in a row share (and reuse) the scratch
        got = ds.psd_loglike_noalloc(theta, buf, kmax, precision).cpu().numpy()
        # same kernels, same work decomposition, fixed-order sums: the same bits
        np.testing.assert_array_equal(got, ref)
    ds.close()


def test_noalloc_rejects_problems_beyond_its_scratch():
    import torch
    from paper_2507_06300_gb300 import binding as B
    wl = synth.workload("tiny", n_bins=131072, n_states=256)
    ds = B.Dataset.from_workload(wl, np.ones((3, wl.n_bins)))
    ds.set_tiling(tile_bins=64, states_per_cta=128, group=2)   # 2,048 tiles x 256 states
    assert ds.workspace_bytes(wl.knots.kmax, 0) > B.NOALLOC_SCRATCH_BYTES
    count, x, w, kmax, kind = B.knots_to_device(wl.knots)
    theta = torch.as_tensor(wl.theta, device="cuda")
    buf, _ = ds.spline_setup(count, x, w, kmax, kind, 0)
    with pytest.raises(B.LisaError, match="status 7"):
        ds.psd_loglike_noalloc(theta, buf, kmax, 0)
    ds.close()
