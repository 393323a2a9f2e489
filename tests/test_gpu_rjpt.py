"""The RJ-PT sampler driven by the library, its state on the GPU: log L and its gradient of every
walker x temperature state in one lisa_psd_loglike_grad call per move.  The log L the sampler carries must equal the
oracle's for the states it ends in (FP64 path within 1e-12 relative), and every move type must
be exercised."""
import numpy as np
import pytest

import oracle
from paper_2507_06300_gb300 import rjpt, synth
from tests._workloads import fp32_tolerance, oracle_dataset

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [1, 0])
def test_rjpt_sweeps_on_the_gpu_match_the_oracle(precision):
    from paper_2507_06300_gb300 import binding as B
    T, W, kmax = 4, 8, 8
    wl = synth.workload("small_ae", n_states=T * W)
    ds_o = oracle_dataset(wl)
    P = ds_o["P"]
    ds = B.Dataset.from_workload(wl, P)
    like = rjpt.GpuLikelihood(ds, kmax, kind=0, precision=precision)
    s = rjpt.RJPTSampler(like, betas=rjpt.paper_ladder(T), n_walkers=W, n_splines=wl.n_splines, kmax=kmax,
                         k_max_rj=6, x_lo=float(ds_o["x_lo"]), x_hi=float(ds_o["x_hi"]), sgwb_model=1, seed=4,
                         device="cuda")
    s.init_from_prior(theta_center=wl.theta_true[0], rel=0.01, k0=1)
    rec = s.run(12, n_adapt=6)
    kn = {"count": s.st.count.cpu().numpy(), "x": s.st.x.cpu().numpy(), "w": s.st.w.cpu().numpy(), "kmax": kmax,
          "kind": 0}
    L, st = oracle.loglike(ds_o, s.st.theta.cpu().numpy(), kn)
    logL = s.logL.cpu().numpy()
    ok = st == 0
    assert ok.all()
    if precision == 1:
        np.testing.assert_allclose(logL, L, rtol=1e-12, atol=0)
    else:
        tol = fp32_tolerance(L, wl, P)
        assert np.all(np.abs(logL - L) <= tol)
    acc = s.acceptance()
    assert np.all(acc["mala"] > 0) and np.all(acc["swap"] >= 0)
    assert rec["logL"].shape == (6, T, W)
    ds.close()
