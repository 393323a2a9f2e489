"""Pins for the oracle's log-likelihood and gradient (Sec. III.C; Eq. splines).

* Each per-bin term is the log-density of a 1x1 complex Wishart variate, i.e. a Gamma(nu,
  scale S) density of Y = nu P: differences of log L between states must equal differences of
  scipy.stats.gamma.logpdf sums.  This also pins the covariance reading C = S.
* P = S gives log L = -sum nu sum_c (1 + ln S) and a zero gradient.
* Whittle (nu = 1, or any constant nu) for S = alpha S0: closed-form maximiser
  alpha* = mean(P/S0) and closed-form maximum.
* mpmath brute force on a few bins; invariance under knot and state permutations;
  the gradient against central finite differences; invalid states."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_2507_06300_gb300 import synth
from tests._workloads import oracle_dataset, zero_knots


@pytest.fixture(scope="module")
def tiny():
    wl = synth.workload("tiny")
    ds = oracle_dataset(wl)
    return wl, ds


def test_zero_perturbation_is_template(tiny):
    wl, ds = tiny
    th = wl.theta[:2]
    S, st = oracle.model_psd(ds, th, zero_knots(2, wl.n_splines))
    assert not st.any()
    for s in range(2):
        sn = oracle.noise_templates(ds["f"], th[s, 0], th[s, 1])[:3]
        for c in range(3):
            sh = oracle.sgwb_template(ds["f"], ds["R"][c], th[s, 2], th[s, 3], f_ref=ds["f_ref"])
            np.testing.assert_allclose(S[s, c], sn[c] + sh, rtol=1e-15)


def test_wishart_term_is_gamma_density(tiny):
    wl, ds = tiny
    th, kn = wl.states(0)
    L, st = oracle.loglike(ds, th, kn.as_dict())
    S, _ = oracle.model_psd(ds, th, kn.as_dict())
    nu = ds["nu"]
    Y = nu * ds["P"]
    g = np.array([stats.gamma.logpdf(Y, a=nu, scale=S[s]).sum() for s in range(th.shape[0])])
    ok = st == 0
    assert ok.sum() >= 2
    dL = L[ok] - L[ok][0]
    dg = g[ok] - g[ok][0]
    np.testing.assert_allclose(dL, dg, rtol=1e-10, atol=1e-7)


def test_periodogram_equal_to_psd_closed_form(tiny):
    wl, ds = tiny
    th, kn = wl.states(0)
    S, st = oracle.model_psd(ds, th[:1], kn.as_dict() | {"count": kn.count[:1], "x": kn.x[:1],
                                                        "w": kn.w[:1]})
    ds2 = dict(ds, P=S[0])
    k1 = {"count": kn.count[:1], "x": kn.x[:1], "w": kn.w[:1], "kmax": kn.kmax, "kind": 0}
    L, g, st = oracle.loglike_grad(ds2, th[:1], k1)
    expect = -np.sum(ds["nu"] * np.sum(1.0 + np.log(S[0]), axis=0))
    assert L[0] == pytest.approx(expect, rel=1e-14, abs=0)
    assert np.abs(g).max() < 1e-9 * np.abs(expect)


@pytest.mark.parametrize("nu", [1.0, 16.0])
def test_whittle_scale_maximiser(nu):
    # noise-only model S = a^2 U (single OMS term): S scales as alpha = a^2.
    f = synth.freq_grid(500)
    rng = np.random.default_rng(1)
    ds = {"n_channels": 3, "sgwb_model": 0, "f": f, "nu": np.full(f.size, nu), "x_lo": -4.0,
          "x_hi": math.log10(2.9e-2), "f_ref": 1e-3}
    S0 = oracle.noise_templates(f, 1.0, 0.0)
    ds["P"] = S0 * rng.gamma(nu, size=S0.shape) / nu * 7.0
    alpha = np.mean(ds["P"] / S0)
    kn = zero_knots(3, 3)
    a_star = math.sqrt(alpha)
    th = np.array([[a_star * 0.999, 0, 0, 0, 0], [a_star, 0, 0, 0, 0], [a_star * 1.001, 0, 0, 0, 0]])
    L, g, st = oracle.loglike_grad(ds, th, kn)
    assert L[1] > L[0] and L[1] > L[2]
    closed = -nu * np.sum(3.0 * (1.0 + math.log(alpha)) + np.sum(np.log(S0), axis=0))
    assert L[1] == pytest.approx(closed, rel=1e-13, abs=0)
    assert abs(g[1, 0]) < 1e-6 * abs(g[0, 0])


@pytest.mark.parametrize("sigma", [1e-3, 7.5, 1e4])
def test_common_rescaling_shifts_by_log_sigma(sigma):
    """Sec. III.C: with P and S both multiplied by sigma (noise-only model: amplitudes by
    sqrt(sigma)), every ratio P/S is unchanged and log L shifts by exactly -C sum(nu) ln sigma."""
    wl = synth.workload("tiny", sgwb_model=0)
    ds = oracle_dataset(wl)
    th, kn = wl.states(0)
    L, st = oracle.loglike(ds, th, kn.as_dict())
    th2 = th.copy()
    th2[:, :2] *= math.sqrt(sigma)
    L2, st2 = oracle.loglike(dict(ds, P=ds["P"] * sigma), th2, kn.as_dict())
    np.testing.assert_array_equal(st, st2)
    ok = st == 0
    shift = -3 * ds["nu"].sum() * math.log(sigma)
    np.testing.assert_allclose(L2[ok] - L[ok], shift, rtol=1e-9, atol=1e-9 * np.abs(L[ok]).max())


def test_brute_force_mpmath_few_bins(tiny):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    wl, ds = tiny
    sl = slice(40, 46)
    ds6 = dict(ds, f=ds["f"][sl], nu=ds["nu"][sl], P=ds["P"][:, sl], R=ds["R"][:, sl])
    th, kn = wl.states(0)
    L, st = oracle.loglike(ds6, th, kn.as_dict())
    S, _ = oracle.model_psd(ds6, th, kn.as_dict())
    for s in np.flatnonzero(st == 0):
        acc = mp.mpf(0)
        for i in range(6):
            for c in range(3):
                Sc = mp.mpf(float(S[s, c, i]))
                acc -= mp.mpf(float(ds6["nu"][i])) * (mp.mpf(float(ds6["P"][c, i])) / Sc + mp.log(Sc))
        assert L[s] == pytest.approx(float(acc), rel=1e-14, abs=0)


def test_permutation_invariance(tiny):
    wl, ds = tiny
    th, kn = wl.states(0)
    L, st = oracle.loglike(ds, th, kn.as_dict())
    rng = np.random.default_rng(9)
    x2, w2 = kn.x.copy(), kn.w.copy()
    for s in range(th.shape[0]):
        for a in range(kn.count.shape[1]):
            k = kn.count[s, a]
            p = rng.permutation(k)
            x2[s, a, :k] = kn.x[s, a, p]
            w2[s, a, 1:1 + k] = kn.w[s, a, 1 + p]
    L2, _ = oracle.loglike(ds, th, dict(kn.as_dict(), x=x2, w=w2))
    np.testing.assert_array_equal(L, L2)
    perm = rng.permutation(th.shape[0])
    L3, _ = oracle.loglike(ds, th[perm], dict(kn.as_dict(), count=kn.count[perm], x=kn.x[perm],
                                              w=kn.w[perm]))
    np.testing.assert_array_equal(L3, L[perm])


def _fd(ds, th, kn, which, idx, h):
    def ev(delta):
        th2, x2, w2 = th.copy(), kn["x"].copy(), kn["w"].copy()
        if which == "theta":
            th2[0, idx] += delta
        elif which == "w":
            w2[(0,) + idx] += delta
        else:
            x2[(0,) + idx] += delta
        return oracle.loglike(ds, th2, dict(kn, x=x2, w=w2))[0][0]
    return (ev(h) - ev(-h)) / (2 * h)


@pytest.mark.parametrize("sgwb_model, kind", [(1, 0), (2, 0), (1, 1)])
def test_gradient_matches_central_differences(tiny, sgwb_model, kind):
    wl, ds = tiny
    ds = dict(ds, sgwb_model=sgwb_model, f_ref=3e-3)
    rng = np.random.default_rng(21)
    nsp = 4
    kmax = 5
    count = np.array([[4, 2, 0, 3]], np.int32)
    x = np.zeros((1, nsp, kmax))
    for a in range(nsp):
        x[0, a, :count[0, a]] = np.sort(rng.uniform(-3.9, -1.6, count[0, a]))[::-1]
    w = rng.normal(0, 0.1, (1, nsp, kmax + 2))
    kn = {"count": count, "x": x, "w": w, "kmax": kmax, "kind": kind}
    th = np.array([[14.0, 3.2, -11.9, 0.5, -0.8]])
    L, g, st = oracle.loglike_grad(ds, th, kn)
    assert st[0] == 0
    G = g[0]
    checks = [("theta", q, 5 * 0 + q) for q in range(5 if sgwb_model == 2 else 4)]
    for a in range(nsp):
        base = 5 + a * (2 * kmax + 2)
        k = count[0, a]
        for slot in [0, kmax + 1] + list(range(1, k + 1)):
            checks.append(("w", (a, slot), base + slot))
        for j in range(k):
            checks.append(("x", (a, j), base + kmax + 2 + j))
    scale = np.abs(G).max()
    for which, idx, gi in checks:
        h = 1e-6 if which != "theta" else 1e-6 * max(1.0, abs(th[0, idx]))
        fd = _fd(ds, th, kn, which, idx, h)
        assert abs(fd - G[gi]) <= 1e-5 * abs(G[gi]) + 2e-6 * scale, (which, idx, fd, G[gi])
    # inactive slots carry a zero gradient
    for a in range(nsp):
        base = 5 + a * (2 * kmax + 2)
        k = count[0, a]
        assert np.all(G[base + 1 + k: base + kmax + 1] == 0)
        assert np.all(G[base + kmax + 2 + k: base + 2 * kmax + 2] == 0)


def test_invalid_states_give_minus_inf(tiny):
    wl, ds = tiny
    th = np.repeat(wl.theta[:1], 5, axis=0)
    kn = zero_knots(5, 4, kmax=3)
    kn["count"][:] = 2
    kn["x"][:, :, 0] = -3.0
    kn["x"][:, :, 1] = -2.5
    kn["count"][1, 0] = 4          # > kmax
    kn["x"][2, 1, 1] = -3.0        # duplicate
    kn["x"][3, 2, 0] = 0.5         # outside the band
    th[4, 2] = np.nan              # non-finite template parameter
    L, g, st = oracle.loglike_grad(ds, th, kn)
    assert st[0] == 0 and np.isfinite(L[0])
    assert list(st[1:]) == [1, 4, 2, 16]
    assert np.all(np.isneginf(L[1:]))
    assert np.all(g[1:] == 0)
