"""GPU adjoint (lisa_psd_loglike_grad) against the oracle's analytic gradient and against
central finite differences of the GPU log-likelihood.

Tolerances, per component, relative to that component's condition scale sum_i |contribution of
bin i| (from the oracle): 1e-12 in FP64 mode, 1e-5 in FP32-bulk mode (plus 1e-12 of the state's
largest component: the states the FP32 call redoes in FP64).  A gradient component is a
sum over bins whose terms cancel near the likelihood's maximum; per-bin arithmetic (relative error
~1e-7 in S in FP32, ~1e-6 in d logL/dS once 1 - S is formed) can only be accurate relative to
that scale, not to the cancelled sum."""
import numpy as np
import pytest

import oracle
from paper_2507_06300_gb300 import synth
from tests._workloads import fp32_tolerance, oracle_batched, oracle_dataset

pytestmark = pytest.mark.gpu
FP32, FP64 = 0, 1


def gpu_grad(wl, P, precision, kind=None):
    import torch
    from paper_2507_06300_gb300 import binding as B
    ds = B.Dataset.from_workload(wl, P)
    count, x, w, kmax, kd = B.knots_to_device(wl.knots)
    kd = kd if kind is None else kind
    theta = torch.as_tensor(wl.theta, device="cuda")
    buf, st = ds.spline_setup(count, x, w, kmax, kd, precision)
    L, G = ds.psd_loglike_grad(theta, count, x, w, kmax, kd, buf, precision)
    L1 = ds.psd_loglike(theta, buf, kmax, precision)
    torch.cuda.synchronize()
    res = L.cpu().numpy(), G.cpu().numpy(), st.cpu().numpy(), L1.cpu().numpy()
    ds.close()
    return res


def oracle_grad_batched(wl, P):
    G, Sc = [], []
    for d in range(wl.n_datasets):
        ds = oracle_dataset(wl, d)
        th, kn = wl.states(d)
        if th.shape[0]:
            _, g, sc, _ = oracle.loglike_grad_scale(ds, th, kn.as_dict())
            G.append(g)
            Sc.append(sc)
    return np.concatenate(G), np.concatenate(Sc)


def check_grad(G, G_ref, ok, precision, scale=None):
    for s in np.flatnonzero(ok):
        err = np.abs(G[s] - G_ref[s])
        if precision == FP64:
            bound = 1e-12 * scale[s]
        else:
            # plus an FP64-level floor: states whose FP32 sums leave the FP32 range are redone in
            # FP64 by the library, accurate to FP64 rounding of the state's largest components
            bound = 1e-5 * scale[s] + 1e-12 * np.abs(G_ref[s]).max()
        bad = err > bound
        assert not bad.any(), (s, np.flatnonzero(bad)[:5], err[bad][:5], bound[bad][:5] if np.ndim(bound) else bound)


@pytest.mark.parametrize("precision", [FP64, FP32])
@pytest.mark.parametrize("variant", ["akima", "natural", "broken", "noise_only", "ae", "wide_band"])
def test_adjoint_matches_oracle_gradient(precision, variant):
    over = dict(n_bins=3000, n_states=16, kmin=0, kmax_draw=8)
    if variant == "wide_band":
        # |log10 f_min| > 2.9 |log10 f_max|: the FP32 adjoint forms t = x - x_o with a two-sum
        over.update(f_min=2e-5, f_max=2.5e-2)
    if variant == "broken":
        over["sgwb_model"] = 2
    if variant == "noise_only":
        over["sgwb_model"] = 0
    if variant == "ae":
        over["n_channels"] = 2
    wl = synth.workload("tiny", **over)
    if variant == "natural":
        wl.knots.kind = 1
    wl.f_ref[:] = 3e-3
    P, L, St = oracle_batched(wl)
    Lg, G, Sg, L1 = gpu_grad(wl, P, precision)
    G_ref, G_sc = oracle_grad_batched(wl, P)
    ok = St == 0
    np.testing.assert_array_equal(Sg, St)
    # log L from the adjoint: FP64 equals the forward entry point's; FP32 meets the FP32 bound
    if precision == FP64:
        np.testing.assert_allclose(Lg[ok], L1[ok], rtol=1e-12, atol=0)
    else:
        tol = fp32_tolerance(L, wl, P)
        assert np.all(np.abs(Lg[ok] - L[ok]) <= tol[ok])
    check_grad(G, G_ref, ok, precision, G_sc)
    # slots of absent knots carry zeros
    kmax = wl.knots.kmax
    for s in np.flatnonzero(ok):
        for a in range(wl.n_splines):
            k = wl.knots.count[s, a]
            base = 5 + a * (2 * kmax + 2)
            assert np.all(G[s, base + 1 + k: base + kmax + 1] == 0)
            assert np.all(G[s, base + kmax + 2 + k: base + 2 * kmax + 2] == 0)


@pytest.mark.parametrize("kind", [0, 1])
def test_fp32_adjoint_on_ill_conditioned_intervals(kind):
    """Prior draws with close knot pairs: intervals whose FP32 cubic cancels (conditioning T > 32,
    the states the forward path routes to its compensated kernel).  The FP32 adjoint evaluates
    their spline values in float-float; its log L must meet the FP32 bound against the oracle
    (a plain FP32 evaluation there overflows 2^P and returned -inf) and its gradient the
    per-component bound."""
    wl = synth.workload("tiny", n_bins=3000, n_states=48, kmin=2, kmax_draw=8, theta_mode="prior")
    wl.knots.kind = kind
    wl.f_ref[:] = 3e-3
    rng = np.random.default_rng(11 + kind)
    k = wl.knots
    for s in range(0, wl.n_states, 3):
        for a in range(wl.n_splines):
            if k.count[s, a] >= 2:
                k.x[s, a, 1] = k.x[s, a, 0] + rng.uniform(2e-5, 2e-4) * (1 if k.x[s, a, 0] < -2 else -1)
    P, L, St = oracle_batched(wl)
    Lg, G, Sg, L1 = gpu_grad(wl, P, FP32)
    G_ref, G_sc = oracle_grad_batched(wl, P)
    ok = St == 0
    assert ok.sum() >= wl.n_states // 2
    np.testing.assert_array_equal(Sg & ~32, St & ~32)
    tol = fp32_tolerance(L, wl, P)
    assert np.all(np.isfinite(Lg[ok]))
    assert np.all(np.abs(Lg[ok] - L[ok]) <= tol[ok]), np.max(np.abs(Lg[ok] - L[ok]) / tol[ok])
    check_grad(G, G_ref, ok, FP32, G_sc)


@pytest.mark.parametrize("kind", [0, 1])
def test_fp32_gradient_when_every_state_leaves_the_fp32_range(kind):
    """Every state's first noise spline lifted by 45 decades (the interpolant of amplitudes + c is
    the interpolant + c for both kinds), so its PSD is beyond the FP32 range at every bin and every
    interval of that spline is ill-conditioned (|c0| ~ 150 in log2 units).  The FP32 adjoint masks
    all bins, the compensated pass takes all of them and flags every state, and the fallback pass
    redoes every state from its list (more items than SMs, fetched from a counter), with the FP64
    reverse map.  log L and the gradient must meet the FP32 bounds against the oracle."""
    wl = synth.workload("tiny", n_bins=5000, n_states=96, kmin=0, kmax_draw=8)
    wl.knots.kind = kind
    wl.f_ref[:] = 3e-3
    wl.knots.w[:, 0, :] += 45.0
    P, L, St = oracle_batched(wl)
    Lg, G, Sg, L1 = gpu_grad(wl, P, FP32)
    G_ref, G_sc = oracle_grad_batched(wl, P)
    ok = St == 0
    assert ok.sum() >= wl.n_states // 2
    np.testing.assert_array_equal(Sg & ~32, St & ~32)
    assert np.all(np.isfinite(Lg[ok]))
    tol = fp32_tolerance(L, wl, P)
    assert np.all(np.abs(Lg[ok] - L[ok]) <= tol[ok]), np.max(np.abs(Lg[ok] - L[ok]) / tol[ok])
    check_grad(G, G_ref, ok, FP32, G_sc)


def test_adjoint_matches_finite_differences_of_the_gpu_loglike():
    """Central differences (h = 1e-6) of the FP64 GPU log-likelihood for a few parameters."""
    import torch
    from paper_2507_06300_gb300 import binding as B
    wl = synth.workload("tiny", n_bins=2000, n_states=4, kmin=3, kmax_draw=5)
    P, L, St = oracle_batched(wl)
    Lg, G, Sg, _ = gpu_grad(wl, P, FP64)
    ds = B.Dataset.from_workload(wl, P)
    count, x, w, kmax, kind = B.knots_to_device(wl.knots)
    theta = torch.as_tensor(wl.theta, device="cuda")

    def ev(th, xx, ww):
        buf, _ = ds.spline_setup(count, xx, ww, kmax, kind, FP64)
        return ds.psd_loglike(th, buf, kmax, FP64).cpu().numpy()

    h = 1e-6
    s = 0
    checks = [("theta", 0), ("theta", 1), ("theta", 2), ("theta", 3), ("w", (0, 0)), ("w", (1, 2)),
              ("w", (3, kmax + 1)), ("x", (0, 1)), ("x", (3, 0))]
    for which, idx in checks:
        d_th, d_x, d_w = theta.clone(), x.clone(), w.clone()
        if which == "theta":
            step = h * max(1.0, abs(wl.theta[s, idx]))
            d_th[s, idx] += step
            gi = idx
            lp = ev(d_th, x, w)[s]
            d_th[s, idx] -= 2 * step
            lm = ev(d_th, x, w)[s]
        elif which == "w":
            step = h
            a, slot = idx
            d_w[s, a, slot] += step
            lp = ev(theta, x, d_w)[s]
            d_w[s, a, slot] -= 2 * step
            lm = ev(theta, x, d_w)[s]
            gi = 5 + a * (2 * kmax + 2) + slot
        else:
            step = h
            a, j = idx
            if j >= wl.knots.count[s, a]:
                continue
            d_x[s, a, j] += step
            lp = ev(theta, d_x, w)[s]
            d_x[s, a, j] -= 2 * step
            lm = ev(theta, d_x, w)[s]
            gi = 5 + a * (2 * kmax + 2) + kmax + 2 + j
        fd = (lp - lm) / (2 * step)
        assert abs(fd - G[s, gi]) <= 1e-5 * abs(G[s, gi]) + 1e-6 * np.abs(G[s]).max(), (which, idx, fd, G[s, gi])
    ds.close()


def test_autograd_function():
    import torch
    from paper_2507_06300_gb300 import binding as B
    wl = synth.workload("tiny", n_bins=1000, n_states=6)
    P, L, St = oracle_batched(wl)
    ds = B.Dataset.from_workload(wl, P)
    count, x, w, kmax, kind = B.knots_to_device(wl.knots)
    theta = torch.as_tensor(wl.theta, device="cuda").requires_grad_(True)
    w = w.clone().requires_grad_(True)
    x = x.clone().requires_grad_(True)
    out = B.psd_loglike(ds, theta, w, x, count, kmax, kind, FP64)
    weights = torch.arange(1, wl.n_states + 1, dtype=torch.float64, device="cuda")
    (out * weights).sum().backward()
    _, G, _, _ = gpu_grad(wl, P, FP64)
    G = torch.as_tensor(G, device="cuda") * weights[:, None]
    nsp, per = wl.n_splines, 2 * kmax + 2
    torch.testing.assert_close(theta.grad, G[:, :5], rtol=1e-12, atol=0)
    body = G[:, 5:].reshape(wl.n_states, nsp, per)
    torch.testing.assert_close(w.grad, body[:, :, :kmax + 2], rtol=1e-12, atol=0)
    torch.testing.assert_close(x.grad, body[:, :, kmax + 2:], rtol=1e-12, atol=0)
    np.testing.assert_allclose(out.detach().cpu().numpy()[St == 0], L[St == 0], rtol=1e-12)
    ds.close()


@pytest.mark.parametrize("precision", [FP64, FP32])
def test_adjoint_workload_sampled_states(precision):
    """2,048 states x 131,072 bins, 12 + 8 knots: the oracle checks 3 sampled states."""
    wl = synth.workload("adjoint")
    ds = oracle_dataset(wl)
    Lg, G, Sg, L1 = gpu_grad(wl, ds["P"], precision)
    pick = np.array([0, 700, 2047])                 # cold, cold, hot
    th = wl.theta[pick]
    kn = {k: (v[pick] if isinstance(v, np.ndarray) else v) for k, v in wl.knots.as_dict().items()}
    L_ref, G_ref, G_sc, St_ref = oracle.loglike_grad_scale(ds, th, kn)
    check_grad(G[pick], G_ref, St_ref == 0, precision, G_sc)
