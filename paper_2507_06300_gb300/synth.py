"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the likelihood or of the PSD model: it only draws random
numbers and lays out grids.  Both the CUDA path and the CPU oracle consume what it returns, so
it is the one module they share.  The periodogram itself (model PSD x Gamma(nu)/nu) is formed
by whichever side needs it, from its own model PSD and the multipliers drawn here.

Workload shapes follow Sec. II.D and Sec. III of arXiv:2507.06300: A/E/T channels, frequencies
uniform in [1e-4, 2.9e-2] Hz, averaged periodograms with nu degrees of freedom per bin, template
parameters in the units of Table I, knot positions uniform in log10 f, knot amplitudes
N(0, 0.1).  The SGWB response R_c(f) is a labelled STAND-IN: the paper evaluates it from an
external Mathematica code whose grids are not available.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED = 20250706
F_MIN = 1.0e-4
F_MAX = 2.9e-2
N_THETA = 5  # a_oms, a_tm, log10 A, n1, n2

# Injection used for the paper-scale workload: OMS 15 pm, TM 3 fm/s^2, log10 Omega = -12,
# n_t = 2/3 (power law, so n2 = n1).
THETA_INJ = (15.0, 3.0, -12.0, 2.0 / 3.0, 2.0 / 3.0)


def freq_grid(n_bins: int, f_min: float = F_MIN, f_max: float = F_MAX) -> np.ndarray:
    """Bin centre frequencies, uniform in [f_min, f_max] (Hz)."""
    return np.linspace(f_min, f_max, int(n_bins))


def response_standin(f: np.ndarray, n_channels: int) -> np.ndarray:
    """STAND-IN for the sky-averaged SGWB response R_c(f), shape [C, N].

    A smooth positive shape, not the paper's response (its grids are not available): a steep
    low-frequency rise that rolls over near 20 mHz, with the T channel suppressed below ~30 mHz.
    Its scale puts a log10 Omega = -12 background at a few per cent of the injected noise in
    A and E around 1-3 mHz under the default (as printed) TDI transfer reading."""
    f = np.asarray(f, dtype=np.float64)
    y = f / 1.0e-3
    r_ae = 1.5e-9 * y ** 6 / (1.0 + (f / 1.9e-2) ** 2)
    out = np.empty((n_channels, f.size))
    out[0] = r_ae
    out[1] = r_ae
    if n_channels == 3:
        z = (f / 3.0e-2) ** 6
        out[2] = r_ae * z / (1.0 + z)
    return out


def gamma_multipliers(rng: np.random.Generator, n_channels: int, nu: np.ndarray) -> np.ndarray:
    """Gamma(nu, 1)/nu draws, shape [C, N]: the averaged-periodogram scatter around the PSD
    (a chi^2 with 2 nu degrees of freedom, scaled to unit mean)."""
    nu = np.asarray(nu, dtype=np.float64)
    return rng.gamma(shape=np.broadcast_to(nu, (n_channels, nu.size)), scale=1.0) / nu


def complex_wishart_unit(rng: np.random.Generator, nu: np.ndarray) -> np.ndarray:
    """Per bin, W = A A^dagger / nu with A lower triangular (Bartlett decomposition of a 3x3
    complex Wishart matrix with nu degrees of freedom and unit covariance): |A_kk|^2 ~
    Gamma(nu - k, 1), A_jk (j > k) complex normal with unit variance.  E[W] = I, and for a
    covariance C = L L^T the averaged periodogram of nu Gaussian samples is distributed as
    L W L^T.  Returns [9, N]: W_AA, W_EE, W_TT, then real and imaginary parts of W_AE, W_AT, W_ET."""
    nu = np.asarray(nu, dtype=np.float64)
    n = nu.size
    diag = np.sqrt(np.stack([rng.gamma(np.maximum(nu - k, 1e-9), 1.0) for k in range(3)]))
    off = (rng.standard_normal((3, n)) + 1j * rng.standard_normal((3, n))) / np.sqrt(2.0)   # A10, A20, A21
    A = np.zeros((n, 3, 3), dtype=np.complex128)
    A[:, 0, 0], A[:, 1, 1], A[:, 2, 2] = diag
    A[:, 1, 0], A[:, 2, 0], A[:, 2, 1] = off
    W = A @ np.conj(np.transpose(A, (0, 2, 1))) / nu[:, None, None]
    out = np.empty((9, n))
    out[0], out[1], out[2] = W[:, 0, 0].real, W[:, 1, 1].real, W[:, 2, 2].real
    for k, (a, b) in enumerate(((0, 1), (0, 2), (1, 2))):
        out[3 + 2 * k] = W[:, a, b].real
        out[4 + 2 * k] = W[:, a, b].imag
    return out


@dataclasses.dataclass
class Knots:
    """Variable-knot perturbation splines for S states (plain arrays, caller layout).

    count [S, nsp] int32    in-between knots per spline (0..kmax)
    x     [S, nsp, kmax]    in-between positions, log10 f, any order (unused slots 0)
    w     [S, nsp, kmax+2]  slot 0 = w_0 (left edge), 1+j = knot j, kmax+1 = w_n (right edge)
    kind  0 = Akima, 1 = natural cubic
    """
    count: np.ndarray
    x: np.ndarray
    w: np.ndarray
    kmax: int
    kind: int = 0

    def as_dict(self):
        return {"count": self.count, "x": self.x, "w": self.w, "kmax": self.kmax, "kind": self.kind}

    @property
    def n_states(self):
        return self.count.shape[0]

    @property
    def n_splines(self):
        return self.count.shape[1]


def draw_knots(rng: np.random.Generator, n_states: int, n_splines: int, kmin, kmax_draw,
               x_lo: float, x_hi: float, kmax: int | None = None, w_sigma: float = 0.1,
               kind: int = 0) -> Knots:
    """Knot counts uniform in [kmin, kmax_draw] (per spline, or a per-spline sequence),
    positions uniform in (x_lo, x_hi), amplitudes N(0, w_sigma) (Table I prior)."""
    kmin_a = np.broadcast_to(np.asarray(kmin), (n_splines,))
    kmaxd_a = np.broadcast_to(np.asarray(kmax_draw), (n_splines,))
    kmax = int(max(kmaxd_a.max(), 0) if kmax is None else kmax)
    count = np.empty((n_states, n_splines), dtype=np.int32)
    for a in range(n_splines):
        count[:, a] = rng.integers(int(kmin_a[a]), int(kmaxd_a[a]) + 1, size=n_states)
    x = np.zeros((n_states, n_splines, max(kmax, 1)))
    u = rng.random((n_states, n_splines, max(kmax, 1)))
    x[:] = x_lo + (x_hi - x_lo) * u
    # keep positions strictly inside the open interval
    x = np.clip(x, np.nextafter(x_lo, x_hi), np.nextafter(x_hi, x_lo))
    mask = np.arange(max(kmax, 1))[None, None, :] < count[:, :, None]
    x = np.where(mask, x, 0.0)[:, :, :kmax] if kmax > 0 else np.zeros((n_states, n_splines, 0))
    w = rng.normal(0.0, w_sigma, size=(n_states, n_splines, kmax + 2))
    inner = np.arange(kmax + 2)[None, None, :]
    active = (inner == 0) | (inner == kmax + 1) | ((inner >= 1) & (inner <= count[:, :, None]))
    w = np.where(active, w, 0.0)
    return Knots(count=count, x=np.ascontiguousarray(x), w=np.ascontiguousarray(w), kmax=kmax,
                 kind=kind)


def draw_theta(rng: np.random.Generator, n_states: int, mode: str = "posterior",
               center=THETA_INJ, sgwb_model: int = 1, rel: float = 0.02) -> np.ndarray:
    """Template parameters [S, 5] = (a_oms, a_tm, log10 A, n1, n2).

    mode "prior":     Table I: a_oms, a_tm ~ U[1e-2, 1e2], log10 A ~ U[-20, -10], n ~ U[-5, 5];
    mode "posterior": a tight cloud around ``center`` (relative spread ``rel``), the regime of
                      the cold chains of a converged run."""
    th = np.empty((n_states, N_THETA))
    if mode == "prior":
        th[:, 0] = rng.uniform(1e-2, 1e2, n_states)
        th[:, 1] = rng.uniform(1e-2, 1e2, n_states)
        th[:, 2] = rng.uniform(-20.0, -10.0, n_states)
        th[:, 3] = rng.uniform(-5.0, 5.0, n_states)
        th[:, 4] = rng.uniform(-5.0, 5.0, n_states)
    else:
        c = np.asarray(center, dtype=np.float64)
        th[:, 0] = c[0] * (1.0 + rel * rng.standard_normal(n_states))
        th[:, 1] = c[1] * (1.0 + rel * rng.standard_normal(n_states))
        th[:, 2] = c[2] + rel * rng.standard_normal(n_states)
        th[:, 3] = c[3] + rel * rng.standard_normal(n_states)
        th[:, 4] = c[4] + rel * rng.standard_normal(n_states)
    if sgwb_model == 1:
        th[:, 4] = th[:, 3]
    return th


@dataclasses.dataclass
class Workload:
    """One dataset (or a batch of datasets) plus the states to evaluate on it.

    Per dataset d (bins b0:b1 = bin_offset[d]:bin_offset[d+1], states state_offset[d]:...):
      f [N_total], nu [N_total], R [C, N_total], gamma [C, N_total] multipliers,
      x_lo/x_hi/f_ref [D].  theta [S_total, 5], knots (Knots over S_total states).
    The periodogram is P = S_model(theta_true) * gamma, formed by the consumer."""
    name: str
    n_channels: int
    sgwb_model: int
    tdi_form: int
    f: np.ndarray
    nu: np.ndarray
    R: np.ndarray
    gamma: np.ndarray
    bin_offset: np.ndarray
    state_offset: np.ndarray
    x_lo: np.ndarray
    x_hi: np.ndarray
    f_ref: np.ndarray
    theta_true: np.ndarray      # [D, 5] injection per dataset
    theta: np.ndarray           # [S_total, 5]
    knots: Knots
    true_knots: Knots | None = None  # [D] injected perturbations (None = no perturbation)
    cov_model: int = 0          # 1: dense covariance, knots carry z_AE, z_AT, z_ET after the others
    wishart: np.ndarray | None = None  # cov_model 1: unit complex Wishart draws [9, N_total]

    @property
    def n_datasets(self):
        return int(self.bin_offset.size - 1)

    @property
    def n_bins(self):
        return int(self.bin_offset[-1])

    @property
    def n_states(self):
        return int(self.state_offset[-1])

    @property
    def n_splines(self):
        return self.n_channels + (1 if self.sgwb_model else 0) + (3 if self.cov_model else 0)

    def dataset(self, d: int) -> dict:
        """Plain dict view of dataset d (no periodogram: the consumer forms it)."""
        b0, b1 = int(self.bin_offset[d]), int(self.bin_offset[d + 1])
        return {"n_channels": self.n_channels, "sgwb_model": self.sgwb_model,
                "tdi_form": self.tdi_form, "f": self.f[b0:b1], "nu": self.nu[b0:b1],
                "R": self.R[:, b0:b1], "x_lo": float(self.x_lo[d]), "x_hi": float(self.x_hi[d]),
                "f_ref": float(self.f_ref[d])}

    def states(self, d: int):
        s0, s1 = int(self.state_offset[d]), int(self.state_offset[d + 1])
        k = self.knots
        return self.theta[s0:s1], Knots(count=k.count[s0:s1], x=k.x[s0:s1], w=k.w[s0:s1],
                                       kmax=k.kmax, kind=k.kind)


# Correlations injected into the dense-covariance workloads: constant z_AE, z_AT, z_ET (r ~ z,
# a few per cent, the size the paper quotes for cross-correlations of the noise)
Z_INJ = (0.05, 0.03, -0.04)


def _single(name, rng, n_bins, nu, n_channels, sgwb_model, n_states, kmin, kmax_draw, kmax=None,
            theta_mode="mixed", tdi_form=0, kind=0, f_min=F_MIN, f_max=F_MAX, theta_true=THETA_INJ, cov_model=0):
    f = freq_grid(n_bins, f_min, f_max)
    nu_a = np.full(n_bins, float(nu))
    R = response_standin(f, n_channels) if sgwb_model else np.zeros((n_channels, n_bins))
    gam = gamma_multipliers(rng, n_channels, nu_a)
    x_lo, x_hi = math.log10(f_min), math.log10(f_max)
    nsp = n_channels + (1 if sgwb_model else 0)
    if theta_mode == "mixed":
        # Tempered ensemble: the first half of the states near the injection (cold chains),
        # the second half drawn from the prior (hot chains).
        h = n_states // 2
        theta = np.concatenate([draw_theta(rng, h, "posterior", theta_true, sgwb_model),
                                draw_theta(rng, n_states - h, "prior", theta_true, sgwb_model)])
    else:
        theta = draw_theta(rng, n_states, theta_mode, theta_true, sgwb_model)
    if cov_model:
        if n_channels != 3:
            raise ValueError("the dense covariance needs the A, E, T channels")
        nsp += 3
        if not isinstance(kmin, (int, np.integer)):
            kmin = list(kmin) + [0, 0, 0]
        if not isinstance(kmax_draw, (int, np.integer)):
            kmax_draw = list(kmax_draw) + [max(kmax_draw)] * 3
    knots = draw_knots(rng, n_states, nsp, kmin, kmax_draw, x_lo, x_hi, kmax=kmax, kind=kind)
    true_knots, wishart = None, None
    if cov_model:
        km = knots.kmax
        true_knots = Knots(count=np.zeros((1, nsp), np.int32), x=np.zeros((1, nsp, km)),
                           w=np.zeros((1, nsp, km + 2)), kmax=km, kind=kind)
        for q in range(3):
            true_knots.w[0, nsp - 3 + q, :] = Z_INJ[q]
        wishart = complex_wishart_unit(rng, nu_a)
    return Workload(name=name, n_channels=n_channels, sgwb_model=sgwb_model, tdi_form=tdi_form,
                    f=f, nu=nu_a, R=R, gamma=gam, bin_offset=np.array([0, n_bins], np.int64),
                    state_offset=np.array([0, n_states], np.int64), x_lo=np.array([x_lo]),
                    x_hi=np.array([x_hi]), f_ref=np.array([1.0e-3]),
                    theta_true=np.array([theta_true], dtype=np.float64), theta=theta, knots=knots,
                    true_knots=true_knots, cov_model=cov_model, wishart=wishart)


def workload(name: str, seed: int = SEED, **over) -> Workload:
    """Named workloads (sizes of the five configurations this library is measured on).

    small_ae   A,E; 2,000 bins; nu=16; 32x4 = 128 states; noise splines 6 knots, SGWB 4 knots
               (totals incl. the 2 edges).
    paper      A,E,T; 131,072 bins; nu=64; 64x16 = 1,024 states; 0-20 in-between knots.
    batched    1,024 A,E,T datasets, 8k-262k bins each, log10 Omega in [-13,-11], n in [-1,3];
               4x4 = 16 states per dataset; 0-30 in-between knots.
    adjoint    A,E,T; 131,072 bins; 256x8 = 2,048 states; noise 12 knots, SGWB 8 knots.
    full       A,E,T; 524,288 bins; nu=128; 32x256 = 8,192 states; broken power law
               (knee 3 mHz, slopes 2/3 and -1); 0-40 in-between knots.
    tiny       A,E,T; 300 bins; nu=4; 6 states; 0-6 knots (unit tests).

    cov_model=1 (A,E,T workloads) adds the dense covariance: three more splines per state, the
    correlations z_AE, z_AT, z_ET (drawn like the others), constant correlations Z_INJ in the
    injection, and unit complex Wishart draws from which the consumer forms the averaged
    periodogram matrix around its own model covariance.
    """
    rng = np.random.default_rng(seed)
    if name == "small_ae":
        kw = dict(n_bins=2000, nu=16, n_channels=2, sgwb_model=1, n_states=128,
                  kmin=[4, 4, 2], kmax_draw=[4, 4, 2], kmax=4)
    elif name == "paper":
        kw = dict(n_bins=131072, nu=64, n_channels=3, sgwb_model=1, n_states=1024, kmin=0,
                  kmax_draw=20)
    elif name == "adjoint":
        kw = dict(n_bins=131072, nu=64, n_channels=3, sgwb_model=1, n_states=2048,
                  kmin=[10, 10, 10, 6], kmax_draw=[10, 10, 10, 6], kmax=10)
    elif name == "full":
        kw = dict(n_bins=524288, nu=128, n_channels=3, sgwb_model=2, n_states=8192, kmin=0,
                  kmax_draw=40, theta_true=(15.0, 3.0, -12.0, 2.0 / 3.0, -1.0))
    elif name == "tiny":
        kw = dict(n_bins=300, nu=4, n_channels=3, sgwb_model=1, n_states=6, kmin=0, kmax_draw=6)
    elif name == "batched":
        return _batched(rng, **over)
    else:
        raise ValueError(f"unknown workload {name!r}")
    kw.update(over)
    wl = _single(name, rng, **kw)
    if name == "full":
        wl.f_ref[:] = 3.0e-3
    return wl


def _batched(rng, n_datasets=1024, n_min=8192, n_max=262144, states_per=16, kmin=0, kmax_draw=30,
             nu=64, tdi_form=0, kind=0):
    C, sg = 3, 1
    lens = rng.integers(n_min, n_max + 1, size=n_datasets)
    bin_off = np.zeros(n_datasets + 1, np.int64)
    bin_off[1:] = np.cumsum(lens)
    fs, nus, Rs, gs = [], [], [], []
    x_lo = np.empty(n_datasets)
    x_hi = np.empty(n_datasets)
    th_true = np.empty((n_datasets, N_THETA))
    thetas = []
    for d in range(n_datasets):
        f = freq_grid(int(lens[d]))
        fs.append(f)
        nus.append(np.full(f.size, float(nu)))
        Rs.append(response_standin(f, C))
        gs.append(gamma_multipliers(rng, C, nus[-1]))
        x_lo[d], x_hi[d] = math.log10(F_MIN), math.log10(F_MAX)
        lA = rng.uniform(-13.0, -11.0)
        n = rng.uniform(-1.0, 3.0)
        th_true[d] = (15.0, 3.0, lA, n, n)
        thetas.append(draw_theta(rng, states_per, "posterior", th_true[d], sg))
    S = n_datasets * states_per
    knots = draw_knots(rng, S, C + 1, kmin, kmax_draw, x_lo[0], x_hi[0], kind=kind)
    return Workload(name="batched", n_channels=C, sgwb_model=sg, tdi_form=tdi_form,
                    f=np.concatenate(fs), nu=np.concatenate(nus), R=np.concatenate(Rs, axis=1),
                    gamma=np.concatenate(gs, axis=1), bin_offset=bin_off,
                    state_offset=np.arange(n_datasets + 1, dtype=np.int64) * states_per,
                    x_lo=x_lo, x_hi=x_hi, f_ref=np.full(n_datasets, 1.0e-3), theta_true=th_true,
                    theta=np.concatenate(thetas), knots=knots)
