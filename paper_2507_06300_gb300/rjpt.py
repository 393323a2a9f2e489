"""Reversible-jump parallel-tempered ensemble sampler over the batched likelihood.

The sampler of the paper's analysis (Sec. III.A knot scheme, Sec. III.C MCMC setup, Table I
priors), restated for a batched likelihood: every walker x temperature state is evaluated in
one library call per move.

* Model: template parameters theta = (a_oms, a_tm, log10 A, n1, n2) (a_oms = A_OMS / 1e-12,
  a_tm = A_TM / 1e-15; n2 is the slope above the knee of the broken power law) and, per
  perturbation spline, the two edge amplitudes plus k in-between knots (log10 f_k, w_k),
  0 <= k <= k_max (Sec. III.A; the paper uses 0..10).
* Priors (Table I): a_oms, a_tm ~ U[1e-2, 1e2], log10 A ~ U[-20, -10], n ~ U[-5, 5],
  log10 f_k ~ U[log10 f_min, log10 f_max], w ~ N(0, 0.1) for edges and in-between knots, and a
  uniform prior on each spline's knot count.
* Between-model move (Sec. III.A): per walker one spline is picked and a knot is added, with its
  position and amplitude drawn from the prior, or a uniformly chosen in-between knot is removed.
  With the prior as the proposal, the acceptance ratio reduces to the tempered likelihood ratio
  times p(k')/p(k) times the ratio of the move-selection probabilities.
* Within-model move: Metropolis-adjusted Langevin (MALA) on all continuous parameters of the
  current model, with the tempered log posterior's gradient from lisa_psd_loglike_grad (the
  hand-written adjoint) and a diagonal preconditioner from the spread of each temperature's
  ensemble; the step size of each temperature is adapted towards 57 % acceptance during burn-in
  and then frozen.
* Parallel tempering: adjacent temperatures exchange states with probability
  min(1, exp((beta_t - beta_t+1)(log L_t+1 - log L_t))), from the hottest pair to the coldest.
* Evidence (Eq. ss, stepping-stone) and the deviance information criterion (Sec. IV.A) from the
  stored log-likelihoods.

The sampler holds its state in host (numpy) arrays; the likelihood backend moves it to the device
once per move.  Random numbers come from one numpy Generator (seeded).
"""
from __future__ import annotations

import dataclasses
import math
import time

import numpy as np

N_THETA = 5
THETA_LO = np.array([1e-2, 1e-2, -20.0, -5.0, -5.0])
THETA_HI = np.array([1e2, 1e2, -10.0, 5.0, 5.0])
W_SIGMA = 0.1
MALA_TARGET = 0.574


def paper_ladder(n_temps: int = 20) -> np.ndarray:
    """Inverse temperatures, descending from beta = 1 (index 0 is the cold chain), placed as in
    Sec. III.C: a quarter of the chains log-spaced in [1e-20, 1e-12), half in [1e-12, 1e-5) and a
    quarter in [1e-5, 1] (5 + 10 + 5 for the paper's 20 temperatures)."""
    if n_temps < 1:
        raise ValueError("n_temps >= 1")
    if n_temps == 1:
        return np.ones(1)
    a = max(1, n_temps // 4)
    c = max(1, n_temps // 4)
    b = n_temps - a - c
    parts = [np.logspace(-20.0, -12.0, a, endpoint=False)]
    if b > 0:
        parts.append(np.logspace(-12.0, -5.0, b, endpoint=False))
    parts.append(np.logspace(-5.0, 0.0, c))
    return np.concatenate(parts)[::-1].copy()


def active_theta(sgwb_model: int) -> np.ndarray:
    """Indices of theta that the model uses: noise only (a_oms, a_tm), + power law (log10 A, n),
    + broken power law (n2)."""
    return np.arange({0: 2, 1: 4, 2: 5}[int(sgwb_model)])


@dataclasses.dataclass
class State:
    """Walker x temperature states, temperature-major (state s = t * n_walkers + i).

    theta [S, 5]; count [S, nsp] in-between knots; x [S, nsp, kmax] their log10 f (slots < count);
    w [S, nsp, kmax + 2] amplitudes (slot 0 left edge, 1 + j knot j, kmax + 1 right edge)."""
    theta: np.ndarray
    count: np.ndarray
    x: np.ndarray
    w: np.ndarray

    def copy(self):
        return State(self.theta.copy(), self.count.copy(), self.x.copy(), self.w.copy())

    def take(self, idx):
        return State(self.theta[idx], self.count[idx], self.x[idx], self.w[idx])

    def put(self, mask, other):
        self.theta[mask] = other.theta[mask]
        self.count[mask] = other.count[mask]
        self.x[mask] = other.x[mask]
        self.w[mask] = other.w[mask]


def knot_masks(count: np.ndarray, kmax: int):
    """Active slots: x [S, nsp, kmax] (j < count) and w [S, nsp, kmax + 2] (edges and 1..count)."""
    j = np.arange(kmax)
    mx = j[None, None, :] < count[:, :, None]
    jw = np.arange(kmax + 2)
    mw = (jw == 0) | (jw == kmax + 1) | ((jw >= 1) & (jw <= count[:, :, None]))
    return mx, np.broadcast_to(mw, count.shape + (kmax + 2,))


def log_prior(st: State, x_lo: float, x_hi: float, th_idx: np.ndarray, kmax: int) -> np.ndarray:
    """Table I log prior of each state (labelled knots, uniform count prior dropped: it is
    constant).  -inf outside the bounds."""
    S = st.theta.shape[0]
    th = st.theta[:, th_idx]
    inside = np.all((th >= THETA_LO[th_idx]) & (th <= THETA_HI[th_idx]), axis=1)
    lp = np.where(inside, -np.sum(np.log(THETA_HI[th_idx] - THETA_LO[th_idx])), -np.inf)
    mx, mw = knot_masks(st.count, kmax)
    xin = np.all(~mx | ((st.x > x_lo) & (st.x < x_hi)), axis=(1, 2))
    nk = st.count.sum(axis=1)
    lp = lp + np.where(xin, -nk * math.log(x_hi - x_lo), -np.inf)
    nw = mw.reshape(S, -1).sum(axis=1)
    lp = lp - 0.5 * np.sum(np.where(mw, st.w * st.w, 0.0), axis=(1, 2)) / W_SIGMA ** 2 \
        - nw * math.log(W_SIGMA * math.sqrt(2.0 * math.pi))
    return lp


class GpuLikelihood:
    """Likelihood backend over the library: log L and its gradient for all states in one call.

    ``dataset`` is a binding.Dataset whose state count is n_temps * n_walkers; ``kmax`` the knot
    capacity of the arrays; ``precision`` binding.FP32 or FP64.  Inputs and outputs are numpy."""

    def __init__(self, dataset, kmax: int, kind: int = 0, precision: int = 0):
        import torch

        from . import binding as B
        self.B, self.torch = B, torch
        self.ds, self.kmax, self.kind, self.precision = dataset, int(kmax), int(kind), int(precision)
        S, nsp = dataset.n_states, dataset.n_splines
        self.buf = torch.empty(dataset.spline_buf_bytes(kmax, precision), dtype=torch.uint8, device="cuda")
        self.ws = torch.empty(dataset.workspace_bytes(kmax, precision, True), dtype=torch.uint8, device="cuda")
        self.out = torch.empty(S, dtype=torch.float64, device="cuda")
        self.grad = torch.empty((S, N_THETA + nsp * (2 * self.kmax + 2)), dtype=torch.float64, device="cuda")
        self.seconds = 0.0   # wall time inside the calls (copies, library calls, synchronisation)
        self.calls = 0

    def __call__(self, st: State, with_grad: bool = True):
        t0 = time.perf_counter()
        try:
            return self._call(st, with_grad)
        finally:
            self.seconds += time.perf_counter() - t0
            self.calls += 1

    def _call(self, st: State, with_grad: bool):
        t = self.torch
        theta = t.as_tensor(np.ascontiguousarray(st.theta), device="cuda")
        count = t.as_tensor(np.ascontiguousarray(st.count, np.int32), device="cuda")
        x = t.as_tensor(np.ascontiguousarray(st.x), device="cuda")
        w = t.as_tensor(np.ascontiguousarray(st.w), device="cuda")
        self.ds.spline_setup(count, x, w, self.kmax, self.kind, self.precision, buf=self.buf)
        if not with_grad:
            L = self.ds.psd_loglike(theta, self.buf, self.kmax, self.precision, out=self.out, workspace=self.ws)
            return L.cpu().numpy(), None
        L, g = self.ds.psd_loglike_grad(theta, count, x, w, self.kmax, self.kind, self.buf, self.precision,
                                        out=self.out, grad=self.grad, workspace=self.ws)
        return L.cpu().numpy(), g.cpu().numpy()


def split_grad(g: np.ndarray, nsp: int, kmax: int):
    """(d/dtheta [S, 5], d/dw [S, nsp, kmax + 2], d/dx [S, nsp, kmax]) from the library layout."""
    S = g.shape[0]
    body = g[:, N_THETA:].reshape(S, nsp, 2 * kmax + 2)
    return g[:, :N_THETA], body[:, :, :kmax + 2], body[:, :, kmax + 2:]


class RJPTSampler:
    """Reversible-jump parallel-tempered ensemble sampler (see the module docstring).

    like(state, with_grad) -> (log L [S], grad [S, 5 + nsp (2 kmax + 2)] or None): a batched
    likelihood backend (GpuLikelihood, or any callable with that contract)."""

    def __init__(self, like, betas, n_walkers: int, n_splines: int, kmax: int, k_max_rj: int, x_lo: float,
                 x_hi: float, sgwb_model: int = 1, seed: int = 0, rj_every: int = 1):
        self.like = like
        self.betas = np.asarray(betas, dtype=np.float64)
        self.T, self.W, self.nsp = len(self.betas), int(n_walkers), int(n_splines)
        self.S = self.T * self.W
        self.kmax, self.kr = int(kmax), int(k_max_rj)
        if not 0 <= self.kr <= self.kmax:
            raise ValueError("0 <= k_max_rj <= kmax")
        self.x_lo, self.x_hi = float(x_lo), float(x_hi)
        self.sgwb_model = int(sgwb_model)
        self.th_idx = active_theta(sgwb_model)
        self.rng = np.random.default_rng(seed)
        self.rj_every = int(rj_every)
        self.beta_s = np.repeat(self.betas, self.W)
        self.eps = np.full(self.T, 0.5)
        self.scales = None
        self.adapting = True
        self.n_sweeps = 0
        self.acc = {"mala": np.zeros(self.T), "rj": np.zeros(self.T), "swap": np.zeros(max(self.T - 1, 1))}
        self.tries = {"mala": np.zeros(self.T), "rj": np.zeros(self.T), "swap": np.zeros(max(self.T - 1, 1))}

    # ---- initial state -------------------------------------------------------------------
    def init_from_prior(self, theta_center=None, rel=0.0, w_sigma0=1e-4, k0=0):
        """Walkers from the prior (theta uniform in Table I, or a cloud of relative spread rel
        around theta_center), knots as in Sec. III.C: k0 in-between knots at prior positions and
        amplitudes N(0, w_sigma0) (the paper's 1e-8 variance)."""
        S, nsp, kmax = self.S, self.nsp, self.kmax
        th = np.empty((S, N_THETA))
        if theta_center is None:
            th[:] = self.rng.uniform(THETA_LO, THETA_HI, size=(S, N_THETA))
        else:
            c = np.asarray(theta_center, dtype=np.float64)
            th[:] = c + rel * np.abs(c) * self.rng.standard_normal((S, N_THETA)) * (np.abs(c) > 0)
            th[:] = np.clip(th, THETA_LO, THETA_HI)
        if self.sgwb_model == 1:
            th[:, 4] = th[:, 3]
        count = np.full((S, nsp), int(k0), dtype=np.int32)
        x = np.zeros((S, nsp, kmax))
        if kmax:
            x[:] = self.rng.uniform(self.x_lo, self.x_hi, size=(S, nsp, kmax))
        w = w_sigma0 * self.rng.standard_normal((S, nsp, kmax + 2))
        mx, mw = knot_masks(count, kmax)
        self.set_state(State(th, count, np.where(mx, x, 0.0), np.where(mw, w, 0.0)))

    def set_state(self, st: State):
        self.st = st.copy()
        self.logL, self.grad = self.like(self.st, True)
        self.lp = log_prior(self.st, self.x_lo, self.x_hi, self.th_idx, self.kmax)

    # ---- within-model move: MALA ----------------------------------------------------------
    def _grad_logpost(self, st: State, g):
        gt, gw, gx = split_grad(g, self.nsp, self.kmax)
        b = self.beta_s
        gt = b[:, None] * gt
        gw = b[:, None, None] * gw - st.w / W_SIGMA ** 2
        gx = b[:, None, None] * gx
        return gt, gw, gx

    def _ensemble_scales(self):
        """Per temperature: spread of each theta coordinate, of the active amplitudes and of the
        active positions over the walkers (floored), the diagonal preconditioner."""
        T, W = self.T, self.W
        th = self.st.theta.reshape(T, W, N_THETA)
        s_th = th.std(axis=1)
        s_th = np.maximum(s_th, 1e-6 * (THETA_HI - THETA_LO)[None, :])
        mx, mw = knot_masks(self.st.count, self.kmax)
        s_w = np.empty(T)
        s_x = np.empty(T)
        for t in range(T):
            sl = slice(t * W, (t + 1) * W)
            wa = self.st.w[sl][mw[sl]]
            xa = self.st.x[sl][mx[sl]]
            s_w[t] = max(wa.std() if wa.size > 1 else W_SIGMA, 1e-5)
            s_x[t] = max(xa.std() if xa.size > 1 else 0.1 * (self.x_hi - self.x_lo), 1e-5)
        return s_th, s_w, s_x

    def mala(self):
        if self.scales is None or self.adapting:
            self.scales = self._ensemble_scales()
        s_th, s_w, s_x = self.scales
        T, W, S = self.T, self.W, self.S
        tix = np.repeat(np.arange(T), W)
        eps = self.eps[tix]
        mth = np.zeros((S, N_THETA), dtype=bool)
        mth[:, self.th_idx] = True
        mx, mw = knot_masks(self.st.count, self.kmax)
        sth = s_th[tix] * mth
        sw = s_w[tix][:, None, None] * mw
        sx = s_x[tix][:, None, None] * mx

        def drift(st, g):
            gt, gw, gx = self._grad_logpost(st, g)
            return (0.5 * (eps[:, None] * sth) ** 2 * gt, 0.5 * (eps[:, None, None] * sw) ** 2 * gw,
                    0.5 * (eps[:, None, None] * sx) ** 2 * gx)

        def logq(to: State, frm: State, d):
            r = 0.0
            for a, b, dd, sc, e in ((to.theta, frm.theta, d[0], sth, eps[:, None]),
                                    (to.w, frm.w, d[1], sw, eps[:, None, None]),
                                    (to.x, frm.x, d[2], sx, eps[:, None, None])):
                var = (e * sc) ** 2
                z = np.where(var > 0, (a - b - dd) ** 2 / np.where(var > 0, 2.0 * var, 1.0), 0.0)
                r = r - z.reshape(S, -1).sum(axis=1)
            return r

        ok0 = np.isfinite(self.logL) & np.isfinite(self.lp)
        g0 = np.where(ok0[:, None], self.grad, 0.0)
        d0 = drift(self.st, g0)
        new = self.st.copy()
        new.theta = self.st.theta + d0[0] + eps[:, None] * sth * self.rng.standard_normal((S, N_THETA))
        if self.sgwb_model == 1:
            new.theta[:, 4] = new.theta[:, 3]
        new.w = self.st.w + d0[1] + eps[:, None, None] * sw * self.rng.standard_normal(self.st.w.shape)
        new.x = self.st.x + d0[2] + eps[:, None, None] * sx * self.rng.standard_normal(self.st.x.shape)
        lp1 = log_prior(new, self.x_lo, self.x_hi, self.th_idx, self.kmax)
        L1, g1 = self.like(new, True)
        ok1 = np.isfinite(L1) & np.isfinite(lp1)
        d1 = drift(new, np.where(ok1[:, None], g1, 0.0))
        b = self.beta_s
        with np.errstate(invalid="ignore"):
            la = (b * L1 + lp1) - (b * self.logL + self.lp) + logq(self.st, new, d1) - logq(new, self.st, d0)
        la = np.where(ok1, la, -np.inf)
        la = np.where(ok0, la, np.where(ok1, np.inf, -np.inf))   # leave an invalid state at once
        acc = np.log(self.rng.random(S)) < la
        self._accept(acc, new, L1, g1, lp1)
        a_t = acc.reshape(T, W).mean(axis=1)
        self.acc["mala"] += a_t
        self.tries["mala"] += 1
        if self.adapting:
            self.eps *= np.exp((a_t - MALA_TARGET) / math.sqrt(self.n_sweeps + 1.0))
            self.eps = np.clip(self.eps, 1e-4, 5.0)
        return acc

    def _accept(self, acc, new: State, L1, g1, lp1):
        self.st.put(acc, new)
        self.logL = np.where(acc, L1, self.logL)
        self.grad = np.where(acc[:, None], g1, self.grad)
        self.lp = np.where(acc, lp1, self.lp)

    # ---- between-model move: knot birth / death --------------------------------------------
    def _p_birth(self, k):
        return np.where(k <= 0, 1.0, np.where(k >= self.kr, 0.0, 0.5))

    def rj(self):
        S, nsp, kmax = self.S, self.nsp, self.kmax
        if self.kr == 0:
            return np.zeros(S, dtype=bool)
        rows = np.arange(S)
        a = self.rng.integers(0, nsp, size=S)
        k = self.st.count[rows, a].astype(np.int64)
        pb = self._p_birth(k)
        birth = self.rng.random(S) < pb
        new = self.st.copy()
        # birth: a knot from the prior appended at slot k
        xb = self.rng.uniform(self.x_lo, self.x_hi, size=S)
        wb = W_SIGMA * self.rng.standard_normal(S)
        bi = rows[birth]
        new.x[bi, a[birth], k[birth]] = xb[birth]
        new.w[bi, a[birth], 1 + k[birth]] = wb[birth]
        new.count[bi, a[birth]] += 1
        # death: a uniformly chosen in-between knot, the last one moved into its slot
        de = ~birth
        di = rows[de]
        kd = k[de]
        jd = (self.rng.random(di.size) * kd).astype(np.int64)
        ad = a[de]
        new.x[di, ad, jd] = new.x[di, ad, kd - 1]
        new.w[di, ad, 1 + jd] = new.w[di, ad, kd]
        new.x[di, ad, kd - 1] = 0.0
        new.w[di, ad, kd] = 0.0
        new.count[di, ad] -= 1
        k1 = new.count[rows, a].astype(np.int64)
        # move-selection ratio q(reverse) / q(forward); the count prior is uniform and the new
        # knot's prior density cancels its proposal density
        lq = np.where(birth, np.log(np.maximum(1.0 - self._p_birth(k1), 1e-300)) - np.log(np.maximum(pb, 1e-300)),
                      np.log(np.maximum(self._p_birth(k1), 1e-300)) - np.log(np.maximum(1.0 - pb, 1e-300)))
        lp1 = log_prior(new, self.x_lo, self.x_hi, self.th_idx, self.kmax)
        L1, g1 = self.like(new, True)
        ok1 = np.isfinite(L1) & np.isfinite(lp1)
        with np.errstate(invalid="ignore"):
            la = self.beta_s * (L1 - self.logL) + lq
        la = np.where(ok1, la, -np.inf)
        la = np.where(np.isfinite(self.logL), la, np.where(ok1, np.inf, -np.inf))
        acc = np.log(self.rng.random(S)) < la
        self._accept(acc, new, L1, g1, lp1)
        self.acc["rj"] += acc.reshape(self.T, self.W).mean(axis=1)
        self.tries["rj"] += 1
        return acc

    # ---- parallel tempering ----------------------------------------------------------------
    def swap(self):
        """Adjacent-temperature exchanges, hottest pair first; walkers of the hotter temperature
        are paired with a random permutation of the colder one's."""
        T, W = self.T, self.W
        for t in range(T - 2, -1, -1):
            c = np.arange(t * W, (t + 1) * W)                       # colder (larger beta)
            h = (t + 1) * W + self.rng.permutation(W)               # hotter
            with np.errstate(invalid="ignore"):
                la = (self.betas[t] - self.betas[t + 1]) * (self.logL[h] - self.logL[c])
            la = np.where(np.isnan(la), -np.inf, la)
            acc = np.log(self.rng.random(W)) < la
            ci, hi = c[acc], h[acc]
            if ci.size:
                for arr in (self.st.theta, self.st.count, self.st.x, self.st.w):
                    tmp = arr[ci].copy()
                    arr[ci] = arr[hi]
                    arr[hi] = tmp
                for name in ("logL", "lp"):
                    v = getattr(self, name)
                    tmp = v[ci].copy()
                    v[ci] = v[hi]
                    v[hi] = tmp
                tmp = self.grad[ci].copy()
                self.grad[ci] = self.grad[hi]
                self.grad[hi] = tmp
            self.acc["swap"][t] += acc.mean()
            self.tries["swap"][t] += 1

    # ---- driver ------------------------------------------------------------------------------
    def sweep(self):
        self.mala()
        if self.n_sweeps % self.rj_every == 0:
            self.rj()
        if self.T > 1:
            self.swap()
        self.n_sweeps += 1

    def run(self, n_sweeps: int, n_adapt: int = 0, record_every: int = 1):
        """Runs n_sweeps sweeps (the first n_adapt adapt the MALA step sizes and preconditioner,
        then they are frozen).  Returns a dict of recorded arrays: log L of every state
        [n_rec, T, W], and the cold chain's theta [n_rec, W, 5] and knot counts [n_rec, W, nsp]."""
        rec_L, rec_th, rec_k = [], [], []
        for i in range(n_sweeps):
            self.adapting = i < n_adapt
            self.sweep()
            if i >= n_adapt and (i - n_adapt) % record_every == 0:
                rec_L.append(self.logL.reshape(self.T, self.W).copy())
                rec_th.append(self.st.theta[:self.W].copy())
                rec_k.append(self.st.count[:self.W].copy())
        self.adapting = False
        return {"logL": np.array(rec_L), "theta": np.array(rec_th), "count": np.array(rec_k)}

    def acceptance(self):
        return {k: self.acc[k] / np.maximum(self.tries[k], 1) for k in self.acc}


def stepping_stone_log_z(betas, logL) -> tuple:
    """Stepping-stone estimate of log Z (Eq. ss): with the inverse temperatures sorted ascending
    beta_1 < ... < beta_K and n draws theta^i from the tempered posterior at each,
      log Z = sum_k log sum_i L(theta^i at beta_k-1)^(beta_k - beta_k-1) - (K - 1) log n,
    over the K - 1 adjacent pairs (the stretch below the smallest beta, 1e-20 in the paper's
    ladder, contributes log E_prior[L^beta_min], taken as zero).  logL [n_samples, K] (columns in
    the order of ``betas``).  Returns (log Z, the per-pair terms)."""
    b = np.asarray(betas, dtype=np.float64)
    L = np.asarray(logL, dtype=np.float64)
    o = np.argsort(b)
    b, L = b[o], L[:, o]
    n = L.shape[0]
    terms = []
    for k in range(1, b.size):
        v = (b[k] - b[k - 1]) * L[:, k - 1]
        m = np.max(v)
        terms.append(m + math.log(np.sum(np.exp(v - m))) - math.log(n))
    return float(np.sum(terms)), np.array(terms)


def dic(logL_samples, logL_at_point) -> dict:
    """Deviance information criterion (Sec. IV.A): D = -2 log L, p_D = mean(D) - D(point),
    DIC = mean(D) + p_D, for posterior samples of log L and log L at the chosen point estimate
    (the posterior mean of the parameters for a fixed-dimension model)."""
    D = -2.0 * np.asarray(logL_samples, dtype=np.float64)
    Dbar = float(np.mean(D))
    pD = Dbar - (-2.0 * float(logL_at_point))
    return {"Dbar": Dbar, "pD": pD, "DIC": Dbar + pD}
