"""Pins of the data-preparation oracle (oracle.prep): Sec. II.D synthesis and the Sec. III.C
averaged periodogram."""
import numpy as np
from scipy import stats

from oracle import prep


def test_constant_power_is_reproduced_exactly_and_nu_counts_samples():
    C, N = 3, 600
    phase = np.exp(1j * np.linspace(0.0, 7.0, N))
    amp = np.array([2.0, 0.5, 3.0])[:, None]
    d = amp * phase[None, :]                          # |d|^2 = amp^2 exactly up to rounding
    off = np.array([0, 1, 7, 64, 300, 600])
    P, f, nu = prep.averaged_periodogram(d, 1e-4, 1e-6, off)
    assert np.allclose(P, amp ** 2, rtol=1e-14)
    assert np.array_equal(nu, np.diff(off))


def test_single_sample_bins_are_the_plain_periodogram():
    rng = np.random.default_rng(0)
    d = rng.standard_normal((2, 50)) + 1j * rng.standard_normal((2, 50))
    P, _, nu = prep.averaged_periodogram(d, 0.0, 1.0, np.arange(51))
    assert np.allclose(P, np.abs(d) ** 2, rtol=1e-15)         # n_i = 1: the Whittle limit
    assert np.all(nu == 1)


def test_bin_centres_and_empty_bins():
    f0, df = 1e-4, 3.2e-8
    off = np.array([0, 4, 4, 11])
    d = np.ones((1, 11), dtype=complex)
    P, f, nu = prep.averaged_periodogram(d, f0, df, off)
    fk = f0 + df * np.arange(11)
    assert np.isclose(f[0], fk[0:4].mean(), rtol=1e-15) and np.isclose(f[2], fk[4:11].mean(), rtol=1e-15)
    assert np.isnan(P[0, 1]) and nu[1] == 0


def test_gaussian_data_give_the_gamma_law_of_the_wishart_likelihood():
    # nu P / S ~ Gamma(nu, 1) for stationary Gaussian data with E|d|^2 = S (S constant over a
    # bin): the 1x1 complex Wishart law behind the per-bin term -nu (P/S + ln S) of the likelihood
    rng = np.random.default_rng(7)
    C, nb, n = 2, 4000, 16
    S_bin = np.exp(rng.uniform(-2.0, 2.0, size=(C, nb)))
    S = np.repeat(S_bin, n, axis=1)
    d = prep.fd_synthesize(S, rng.standard_normal((C, nb * n, 2)))
    assert np.allclose(np.mean(np.abs(d) ** 2 / S), 1.0, atol=0.01)
    P, _, nu = prep.averaged_periodogram(d, 0.0, 1.0, np.arange(0, nb * n + 1, n))
    y = nu * P / S_bin
    assert stats.kstest(y.ravel(), stats.gamma(n).cdf).pvalue > 1e-3
    assert abs(y.mean() - n) < 0.1 and abs(y.var() / n - 1.0) < 0.06
