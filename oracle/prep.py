"""Plain numpy definitions of the data preparation, the inputs of the likelihood.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle``): used by the tests and by nothing in the
product package.

* ``fd_synthesize`` -- frequency-domain data of a stationary Gaussian process generated directly
  in the frequency domain (Sec. II.D), normalised so that the periodogram is comparable to the
  one-sided PSD (Sec. III.A): d = sqrt(S / 2) (z0 + i z1) with z0, z1 standard normal, so that
  E|d|^2 = S.
* ``averaged_periodogram`` -- Sec. III.C: the periodogram averaged over the n_i consecutive,
  non-overlapping frequency samples of bin i, P(f_i) = (1/n_i) sum_k |d(f_k)|^2 (the diagonal of
  d d^dagger: the A, E, T covariance is diagonal), nu_i = n_i degrees of freedom, and f_i the
  centre of the bin.

Parity status: pinned in tests/test_oracle_prep.py (constant power, the n_i = 1 Whittle limit,
the Gamma(nu) law of nu P / S for Gaussian data, bin centres).
"""
from __future__ import annotations

import numpy as np


def fd_synthesize(S, z):
    """S [C, N] one-sided PSD, z [C, N, 2] standard normal draws -> complex d [C, N]."""
    S = np.asarray(S, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    a = np.sqrt(S / 2.0)
    return a * z[..., 0] + 1j * (a * z[..., 1])


def averaged_periodogram(d, f0, df, bin_offset):
    """d complex [C, N]; bins [bin_offset[i], bin_offset[i+1]) of the uniform grid f_k = f0 + k df.
    Returns (P [C, n_bins], f [n_bins], nu [n_bins]); an empty bin gets P = NaN, nu = 0."""
    d = np.asarray(d)
    off = np.asarray(bin_offset, dtype=np.int64)
    C, N = d.shape
    nb = off.size - 1
    P = np.empty((C, nb))
    f = np.empty(nb)
    nu = np.empty(nb)
    for i in range(nb):
        b0 = min(max(int(off[i]), 0), N)
        b1 = min(max(int(off[i + 1]), b0), N)
        n = b1 - b0
        for c in range(C):
            seg = d[c, b0:b1]
            P[c, i] = np.sum(seg.real ** 2 + seg.imag ** 2) / n if n > 0 else np.nan
        f[i] = f0 + df * 0.5 * (b0 + b1 - 1)
        nu[i] = n
    return P, f, nu
