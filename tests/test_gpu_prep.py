"""Data preparation through the C ABI against the numpy oracle (oracle.prep): synthesis is
elementwise and must match bit for bit; the averaged periodogram sums in FP64 in a different
order, so 1e-14 relative.  Ragged bins of 0..600 samples cover the three lane layouts (one
thread, 4 lanes, 8 lanes per bin), empty bins and a tail that is not a multiple of anything."""
import numpy as np
import pytest

from oracle import prep

pytestmark = pytest.mark.gpu


def test_fd_synthesize_is_exact():
    import torch
    from paper_2507_06300_gb300 import binding as B
    rng = np.random.default_rng(1)
    C, N = 3, 100003
    S = np.exp(rng.uniform(-60.0, -40.0, size=(C, N)))
    z = rng.standard_normal((C, N, 2))
    d = B.fd_synthesize(torch.as_tensor(S, device="cuda"), torch.as_tensor(z, device="cuda")).cpu().numpy()
    ref = prep.fd_synthesize(S, z)
    assert np.array_equal(d[..., 0], ref.real) and np.array_equal(d[..., 1], ref.imag)


@pytest.mark.parametrize("C", [2, 3])
@pytest.mark.parametrize("mean_width", [3, 20, 64, 300])
def test_averaged_periodogram_matches_the_oracle(C, mean_width):
    import torch
    from paper_2507_06300_gb300 import binding as B
    rng = np.random.default_rng(10 * C + mean_width)
    nb = 2500
    widths = rng.integers(0, 2 * mean_width + 1, size=nb)
    widths[::97] = 0
    off = np.concatenate([[0], np.cumsum(widths)]).astype(np.int64)
    N = int(off[-1]) + 5                                   # samples past the last bin are ignored
    d = rng.standard_normal((C, N)) * np.exp(rng.uniform(-3, 3, (C, N))) + 1j * rng.standard_normal((C, N))
    dd = torch.as_tensor(np.stack([d.real, d.imag], axis=-1), device="cuda")
    f0, df = 1e-4, 3.17e-8
    P, f, nu = B.averaged_periodogram(dd, f0, df, torch.as_tensor(off, device="cuda"))
    Pr, fr, nur = prep.averaged_periodogram(d, f0, df, off)
    P, f, nu = P.cpu().numpy(), f.cpu().numpy(), nu.cpu().numpy()
    assert np.array_equal(nu, nur)
    assert np.array_equal(np.isnan(P), np.isnan(Pr))
    ok = ~np.isnan(Pr)
    np.testing.assert_allclose(P[ok], Pr[ok], rtol=1e-14, atol=0)
    np.testing.assert_allclose(f, fr, rtol=1e-15, atol=0)


def test_periodogram_of_synthesized_data_follows_the_gamma_law():
    import torch
    from scipy import stats
    from paper_2507_06300_gb300 import binding as B
    C, nb, n = 3, 20000, 64
    g = torch.Generator(device="cuda").manual_seed(5)
    S_bin = torch.exp(torch.empty((C, nb), dtype=torch.float64, device="cuda").uniform_(-3, 3, generator=g))
    S = S_bin.repeat_interleave(n, dim=1).contiguous()
    z = torch.randn((C, nb * n, 2), dtype=torch.float64, device="cuda", generator=g)
    d = B.fd_synthesize(S, z)
    off = torch.arange(0, nb * n + 1, n, dtype=torch.int64, device="cuda")
    P, f, nu = B.averaged_periodogram(d, 0.0, 1.0, off)
    y = (nu * P / S_bin).cpu().numpy()
    assert stats.kstest(y.ravel(), stats.gamma(n).cdf).pvalue > 1e-3
