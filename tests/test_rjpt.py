"""The reversible-jump parallel-tempered sampler (paper_2507_06300_gb300.rjpt) on the CPU.

Pins: with a flat likelihood the chains must sample the Table I prior, including the uniform
knot-count prior that the birth/death acceptance ratio has to preserve (a dropped or inverted
move-selection term skews the count histogram); on a Gaussian likelihood MALA must recover the
closed-form posterior; the stepping-stone estimator must reproduce the closed-form evidence of a
conjugate Gaussian problem from exact tempered draws; the DIC's effective parameter count must be
the dimension for a Gaussian posterior; and with the oracle likelihood the sampler's cached log L
must equal a fresh evaluation of the states it ends in."""
import math

import numpy as np
import pytest
import torch
from scipy import stats

from paper_2507_06300_gb300 import rjpt

X_LO, X_HI = -4.0, -1.5


def flat_like(nsp, kmax):
    def like(st, with_grad=True):
        S = st.theta.shape[0]
        return np.zeros(S), np.zeros((S, rjpt.N_THETA + nsp * (2 * kmax + 2)))
    return like


def test_ladder_matches_the_papers_placement():
    b = rjpt.paper_ladder(20)
    assert b.shape == (20,) and b[0] == 1.0 and np.all(np.diff(b) < 0)
    lb = np.log10(b[::-1])
    assert np.allclose(lb[:5], np.linspace(-20, -12, 5, endpoint=False))
    assert np.allclose(lb[5:15], np.linspace(-12, -5, 10, endpoint=False))
    assert np.allclose(lb[15:], np.linspace(-5, 0, 5))


def test_flat_likelihood_recovers_the_prior_and_the_uniform_count_prior():
    nsp, kmax, kr, W = 2, 6, 4, 256
    s = rjpt.RJPTSampler(flat_like(nsp, kmax), betas=[1.0], n_walkers=W, n_splines=nsp, kmax=kmax, k_max_rj=kr,
                         x_lo=X_LO, x_hi=X_HI, sgwb_model=1, seed=3)
    s.init_from_prior(k0=0, w_sigma0=0.1)
    rec = s.run(400, n_adapt=100, record_every=5)
    counts = rec["count"][20:].reshape(-1)
    hist = np.bincount(counts, minlength=kr + 1)
    assert hist.size == kr + 1
    # uniform over 0..kr (the samples are correlated: a loose chi-square on thinned draws)
    chi2 = np.sum((hist - hist.mean()) ** 2 / hist.mean())
    assert chi2 < 3.0 * stats.chi2.ppf(0.999, kr), hist
    # knot positions uniform, amplitudes N(0, 0.1), theta uniform in Table I
    mx, mw = rjpt.knot_masks(s.st.count, kmax)
    xa = s.st.x[mx].numpy()
    assert stats.kstest((xa - X_LO) / (X_HI - X_LO), "uniform").pvalue > 1e-3
    wa = s.st.w[mw].numpy()
    assert abs(wa.mean()) < 0.02 and abs(wa.std() - rjpt.W_SIGMA) < 0.02
    th = rec["theta"][20:].reshape(-1, rjpt.N_THETA)
    mid = 0.5 * (rjpt.THETA_LO + rjpt.THETA_HI)
    half = 0.5 * (rjpt.THETA_HI - rjpt.THETA_LO)
    assert np.all(np.abs(th[:, :4].mean(axis=0) - mid[:4]) < 0.1 * half[:4])
    assert np.all(th >= rjpt.THETA_LO) and np.all(th <= rjpt.THETA_HI)
    assert np.array_equal(th[:, 4], th[:, 3])            # single power law: n2 mirrors n1


def test_mala_recovers_a_gaussian_posterior_and_tempering_widens_it():
    nsp, kmax = 1, 2
    mu = np.array([15.0, 3.0, -12.0, 0.5, 0.5])
    sig = np.array([0.05, 0.02, 0.01, 0.03, 0.03])

    def like(st, with_grad=True):
        th, w = st.theta.numpy(), st.w.numpy()
        S = th.shape[0]
        z = (th - mu) / sig
        L = -0.5 * np.sum(z[:, :4] ** 2, axis=1) - 0.5 * np.sum(w[:, :, [0, kmax + 1]] ** 2, axis=(1, 2)) / 0.01 ** 2
        g = np.zeros((S, rjpt.N_THETA + nsp * (2 * kmax + 2)))
        g[:, :4] = -(z / sig)[:, :4]
        g[:, rjpt.N_THETA + 0] = -w[:, 0, 0] / 0.01 ** 2
        g[:, rjpt.N_THETA + kmax + 1] = -w[:, 0, kmax + 1] / 0.01 ** 2
        return L, g

    betas = [1.0, 0.25]
    s = rjpt.RJPTSampler(like, betas=betas, n_walkers=128, n_splines=nsp, kmax=kmax, k_max_rj=0, x_lo=X_LO,
                         x_hi=X_HI, sgwb_model=1, seed=5)
    s.init_from_prior(theta_center=mu, rel=0.001, w_sigma0=0.001)
    rec = s.run(600, n_adapt=200, record_every=2)
    th = rec["theta"].reshape(-1, rjpt.N_THETA)[:, :4]
    assert np.allclose(th.mean(axis=0), mu[:4], atol=0.15 * sig[:4] * 4)
    assert np.allclose(th.std(axis=0), sig[:4], rtol=0.15)
    acc = s.acceptance()["mala"]
    assert 0.3 < acc[0] < 0.85
    # the beta = 1/4 chain samples N(mu, sig / sqrt(beta))
    hot = s.st.theta[128:, :4].numpy()
    assert np.allclose(hot.std(axis=0), sig[:4] * 2.0, rtol=0.35)


def test_swap_acceptance_follows_the_tempered_likelihood_ratio():
    nsp, kmax = 1, 0
    levels = {0: -10.0, 1: -12.0}

    def like(st, with_grad=True):
        S = st.theta.shape[0]
        L = np.where(st.theta[:, 0].numpy() < 50.0, levels[0], levels[1])
        return L, np.zeros((S, rjpt.N_THETA + nsp * 2))

    betas = [1.0, 0.3]
    s = rjpt.RJPTSampler(like, betas=betas, n_walkers=4000, n_splines=nsp, kmax=kmax, k_max_rj=0, x_lo=X_LO,
                         x_hi=X_HI, seed=7)
    s.init_from_prior()
    th = s.st.theta.clone()
    th[:4000, 0] = 10.0      # cold walkers at log L = -10, hot ones at -12
    th[4000:, 0] = 90.0
    s.set_state(rjpt.State(th, s.st.count, s.st.x, s.st.w))
    s.swap()
    # exchanging raises the cold chain's log L by -2: accepted with exp((1 - 0.3) * (-2))
    p = math.exp((1.0 - 0.3) * (-12.0 + 10.0))
    th1, L1 = s.st.theta.numpy(), s.logL.numpy()
    frac = np.mean(th1[:4000, 0] > 50.0)
    assert abs(frac - p) < 4.0 * math.sqrt(p * (1 - p) / 4000)
    # exchanged states keep their own log L
    assert np.all(L1[:4000][th1[:4000, 0] > 50.0] == -12.0)


def test_stepping_stone_matches_the_closed_form_evidence():
    # prior N(0, sp^2), likelihood N(d; theta, sl^2): the tempered posterior at beta is Gaussian
    # with precision 1/sp^2 + beta/sl^2, and Z = N(d; 0, sp^2 + sl^2)
    sp, sl, d, n = 1.0, 0.5, 0.3, 40000
    rng = np.random.default_rng(11)
    betas = rjpt.paper_ladder(20)
    logL = np.empty((n, betas.size))
    for k, b in enumerate(betas):
        prec = 1.0 / sp ** 2 + b / sl ** 2
        m = (b * d / sl ** 2) / prec
        th = m + rng.standard_normal(n) / math.sqrt(prec)
        logL[:, k] = stats.norm.logpdf(d, th, sl)
    lz, terms = rjpt.stepping_stone_log_z(betas, logL)
    assert terms.shape == (19,)
    assert abs(lz - stats.norm.logpdf(d, 0.0, math.hypot(sp, sl))) < 0.02


def test_dic_effective_parameters_equal_the_dimension_for_a_gaussian_posterior():
    rng = np.random.default_rng(2)
    k, sig, n = 3, 0.2, 200000
    dat = np.array([0.5, -1.0, 2.0])
    th = dat + sig * rng.standard_normal((n, k))          # flat prior: posterior N(d, sig^2)
    logL = -0.5 * np.sum(((th - dat) / sig) ** 2, axis=1)
    at_mean = -0.5 * np.sum(((th.mean(axis=0) - dat) / sig) ** 2)
    r = rjpt.dic(logL, at_mean)
    assert abs(r["pD"] - k) < 0.05
    assert abs(r["DIC"] - (r["Dbar"] + r["pD"])) < 1e-12


def test_sweeps_with_the_oracle_keep_log_l_consistent():
    import oracle
    from paper_2507_06300_gb300 import synth
    from tests._workloads import oracle_dataset
    wl = synth.workload("tiny", n_bins=200, n_states=4)
    ds = oracle_dataset(wl)
    nsp, kmax = wl.n_splines, 6

    def like(st, with_grad=True):
        kn = {"count": st.count.numpy(), "x": st.x.numpy(), "w": st.w.numpy(), "kmax": kmax, "kind": 0}
        L, g, status = oracle.loglike_grad(ds, st.theta.numpy(), kn)
        return np.where(status == 0, L, -np.inf), g

    x_lo, x_hi = float(ds["x_lo"]), float(ds["x_hi"])
    s = rjpt.RJPTSampler(like, betas=[1.0, 0.1], n_walkers=3, n_splines=nsp, kmax=kmax, k_max_rj=4, x_lo=x_lo,
                         x_hi=x_hi, sgwb_model=1, seed=1)
    s.init_from_prior(theta_center=wl.theta_true[0], rel=0.01, k0=1)
    s.run(6, n_adapt=3)
    kn = {"count": s.st.count.numpy(), "x": s.st.x.numpy(), "w": s.st.w.numpy(), "kmax": kmax, "kind": 0}
    L, _ = oracle.loglike(ds, s.st.theta.numpy(), kn)
    assert np.allclose(s.logL.numpy(), L, rtol=1e-12, atol=0)
    assert np.all(s.st.count.numpy() <= 4)
    assert np.all(np.isfinite(s.logL.numpy()))


def test_stepping_stone_of_a_constant_likelihood_is_exactly_its_value():
    # L = e^c everywhere: every tempered posterior is the prior and log Z = c exactly (a wrong
    # normaliser, e.g. log(n - 1) in place of log n, shifts it by K log(n / (n - 1)))
    betas = rjpt.paper_ladder(8)
    for n, c in ((2, 0.0), (5, -3.5)):
        lz, terms = rjpt.stepping_stone_log_z(betas, np.full((n, betas.size), c))
        assert abs(lz - c * (betas.max() - betas.min())) < 1e-12


def test_mala_proposal_mean_is_the_preconditioned_gradient_step():
    # with the noise switched off the proposal is z + (eps^2 / 2) s^2 grad log pi(z): a Gaussian
    # log L with a known gradient fixes its sign and scale
    nsp, kmax = 1, 0
    mu, sig = 20.0, 0.5

    def like(st, with_grad=True):
        th = st.theta.numpy()
        g = np.zeros((th.shape[0], rjpt.N_THETA + nsp * 2))
        g[:, 0] = -(th[:, 0] - mu) / sig ** 2
        return -0.5 * ((th[:, 0] - mu) / sig) ** 2, g

    s = rjpt.RJPTSampler(like, betas=[0.5], n_walkers=4, n_splines=nsp, kmax=kmax, k_max_rj=0, x_lo=X_LO,
                         x_hi=X_HI, sgwb_model=0, seed=0)
    s.init_from_prior(theta_center=[21.0, 3.0, -12.0, 0.0, 0.0], rel=0.0, w_sigma0=0.0)
    s.adapting = False
    s.eps[:] = 0.3
    s_th = np.ones((1, rjpt.N_THETA))
    s.scales = (s_th, np.array([0.1]), np.array([0.1]))
    seen = []

    def like_spy(st, with_grad=True):
        seen.append(st.theta.numpy().copy())
        return like(st, with_grad)

    s.like = like_spy
    s._normal = lambda shape: torch.zeros(shape, dtype=torch.float64)   # Gaussian draws switched off
    s.mala()
    z = 21.0
    expect = z + 0.5 * 0.3 ** 2 * (0.5 * -(z - mu) / sig ** 2)   # beta = 0.5, flat theta prior
    assert np.allclose(seen[0][:, 0], expect, rtol=0, atol=1e-12)
    assert np.allclose(seen[0][:, 1], 3.0)                     # a_tm moves only with its gradient
