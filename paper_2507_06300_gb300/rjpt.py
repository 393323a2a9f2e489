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

The sampler holds its state in torch tensors on one device (the GPU for the library backend, the
CPU for host-side likelihoods): proposals, priors, acceptance tests and swaps are batched tensor
operations over all walkers x temperatures, with no host round trip inside a sweep.  Random
numbers come from one seeded torch Generator on that device.
"""
from __future__ import annotations

import dataclasses
import math
import time

import numpy as np
import torch

N_THETA = 5
THETA_LO = np.array([1e-2, 1e-2, -20.0, -5.0, -5.0])
THETA_HI = np.array([1e2, 1e2, -10.0, 5.0, 5.0])
W_SIGMA = 0.1
MALA_TARGET = 0.574
F64 = torch.float64


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
    """Walker x temperature states, temperature-major (state s = t * n_walkers + i), as tensors on
    one device.

    theta [S, 5] f64; count [S, nsp] int32 in-between knots; x [S, nsp, kmax] f64 their log10 f
    (slots < count); w [S, nsp, kmax + 2] f64 amplitudes (slot 0 left edge, 1 + j knot j,
    kmax + 1 right edge)."""
    theta: torch.Tensor
    count: torch.Tensor
    x: torch.Tensor
    w: torch.Tensor

    def copy(self):
        return State(self.theta.clone(), self.count.clone(), self.x.clone(), self.w.clone())

    def to(self, device):
        """The state on ``device`` with the library's dtypes (numpy arrays accepted)."""
        def t(a, dt):
            return torch.as_tensor(np.asarray(a) if not torch.is_tensor(a) else a, dtype=dt,
                                   device=device).contiguous()
        return State(t(self.theta, F64), t(self.count, torch.int32), t(self.x, F64), t(self.w, F64))

    def put(self, mask, other):
        """Takes ``other``'s values where ``mask`` [S] is true."""
        self.theta = torch.where(mask[:, None], other.theta, self.theta)
        self.count = torch.where(mask[:, None], other.count, self.count)
        self.x = torch.where(mask[:, None, None], other.x, self.x)
        self.w = torch.where(mask[:, None, None], other.w, self.w)

    def gather(self, idx):
        """The states reordered: slot i takes state idx[i]."""
        return State(self.theta[idx], self.count[idx], self.x[idx], self.w[idx])


def knot_masks(count: torch.Tensor, kmax: int):
    """Active slots: x [S, nsp, kmax] (j < count) and w [S, nsp, kmax + 2] (edges and 1..count)."""
    c = count[:, :, None]
    j = torch.arange(kmax, device=count.device)
    mx = j < c
    jw = torch.arange(kmax + 2, device=count.device)
    mw = (jw == 0) | (jw == kmax + 1) | ((jw >= 1) & (jw <= c))
    return mx, mw


def log_prior(st: State, x_lo: float, x_hi: float, th_idx: np.ndarray, kmax: int) -> torch.Tensor:
    """Table I log prior of each state (labelled knots, uniform count prior dropped: it is
    constant).  -inf outside the bounds."""
    S, dev = st.theta.shape[0], st.theta.device
    nth = len(th_idx)
    lo = torch.as_tensor(THETA_LO[:nth], dtype=F64, device=dev)
    hi = torch.as_tensor(THETA_HI[:nth], dtype=F64, device=dev)
    th = st.theta[:, :nth]
    inside = ((th >= lo) & (th <= hi)).all(dim=1)
    ninf = torch.tensor(-math.inf, dtype=F64, device=dev)
    lp = torch.where(inside, -float(np.sum(np.log(THETA_HI[:nth] - THETA_LO[:nth]))), ninf)
    mx, mw = knot_masks(st.count, kmax)
    xin = (~mx | ((st.x > x_lo) & (st.x < x_hi))).reshape(S, -1).all(dim=1)
    nk = st.count.sum(dim=1).to(F64)
    lp = lp + torch.where(xin, -nk * math.log(x_hi - x_lo), ninf)
    nw = mw.reshape(S, -1).sum(dim=1).to(F64)
    ww = torch.where(mw, st.w * st.w, torch.zeros((), dtype=F64, device=dev)).reshape(S, -1).sum(dim=1)
    return lp - 0.5 * ww / W_SIGMA ** 2 - nw * math.log(W_SIGMA * math.sqrt(2.0 * math.pi))


class GpuLikelihood:
    """Likelihood backend over the library: log L and its gradient for all states in one call.

    ``dataset`` is a binding.Dataset whose state count is n_temps * n_walkers; ``kmax`` the knot
    capacity of the arrays; ``precision`` binding.FP32 or FP64.  States come in as device tensors
    and log L [S] and the gradient come back as new device tensors (no host copies).  With
    ``sync`` set, each call waits for the device, so that ``seconds`` (the wall time spent in
    calls) is the calls' device time."""

    def __init__(self, dataset, kmax: int, kind: int = 0, precision: int = 0, sync: bool = False):
        from . import binding as B
        self.B = B
        self.ds, self.kmax, self.kind, self.precision = dataset, int(kmax), int(kind), int(precision)
        self.buf = torch.empty(dataset.spline_buf_bytes(kmax, precision), dtype=torch.uint8, device="cuda")
        self.ws = torch.empty(dataset.workspace_bytes(kmax, precision, True), dtype=torch.uint8, device="cuda")
        self.sync = bool(sync)
        self.seconds = 0.0
        self.calls = 0

    def __call__(self, st: State, with_grad: bool = True):
        t0 = time.perf_counter()
        try:
            return self._call(st.to("cuda"), with_grad)
        finally:
            if self.sync:
                torch.cuda.synchronize()
            self.seconds += time.perf_counter() - t0
            self.calls += 1

    def _call(self, st: State, with_grad: bool):
        self.ds.spline_setup(st.count, st.x, st.w, self.kmax, self.kind, self.precision, buf=self.buf)
        if not with_grad:
            return self.ds.psd_loglike(st.theta, self.buf, self.kmax, self.precision, workspace=self.ws), None
        return self.ds.psd_loglike_grad(st.theta, st.count, st.x, st.w, self.kmax, self.kind, self.buf,
                                        self.precision, workspace=self.ws)


def split_grad(g: torch.Tensor, nsp: int, kmax: int):
    """(d/dtheta [S, 5], d/dw [S, nsp, kmax + 2], d/dx [S, nsp, kmax]) from the library layout."""
    S = g.shape[0]
    body = g[:, N_THETA:].reshape(S, nsp, 2 * kmax + 2)
    return g[:, :N_THETA], body[:, :, :kmax + 2], body[:, :, kmax + 2:]


class RJPTSampler:
    """Reversible-jump parallel-tempered ensemble sampler (see the module docstring).

    like(state, with_grad) -> (log L [S], grad [S, 5 + nsp (2 kmax + 2)] or None): a batched
    likelihood backend (GpuLikelihood, or any callable with that contract; numpy results are
    accepted).  ``device``: where the sampler's tensors live ("cuda" with the library backend)."""

    def __init__(self, like, betas, n_walkers: int, n_splines: int, kmax: int, k_max_rj: int, x_lo: float,
                 x_hi: float, sgwb_model: int = 1, seed: int = 0, rj_every: int = 1, device="cpu"):
        self.like = like
        self.dev = torch.device(device)
        self.betas = np.asarray(betas, dtype=np.float64)
        self.T, self.W, self.nsp = len(self.betas), int(n_walkers), int(n_splines)
        self.S = self.T * self.W
        self.kmax, self.kr = int(kmax), int(k_max_rj)
        if not 0 <= self.kr <= self.kmax:
            raise ValueError("0 <= k_max_rj <= kmax")
        self.x_lo, self.x_hi = float(x_lo), float(x_hi)
        self.sgwb_model = int(sgwb_model)
        self.th_idx = active_theta(sgwb_model)
        self.gen = torch.Generator(device=self.dev)
        self.gen.manual_seed(int(seed))
        self.rj_every = int(rj_every)
        self._b = torch.as_tensor(self.betas, dtype=F64, device=self.dev)
        self.beta_s = self._b.repeat_interleave(self.W)
        self.eps = torch.full((self.T,), 0.5, dtype=F64, device=self.dev)
        self.scales = None
        self.adapting = True
        self.n_sweeps = 0
        z = lambda n: torch.zeros(n, dtype=F64, device=self.dev)
        self.acc = {"mala": z(self.T), "rj": z(self.T), "swap": z(max(self.T - 1, 1))}
        self.tries = {"mala": 0, "rj": 0, "swap": 0}

    # ---- random numbers and the backend ----------------------------------------------------
    def _normal(self, shape):
        return torch.randn(shape, generator=self.gen, dtype=F64, device=self.dev)

    def _uniform(self, shape):
        return torch.rand(shape, generator=self.gen, dtype=F64, device=self.dev)

    def _like(self, st: State, with_grad: bool):
        L, g = self.like(st, with_grad)
        L = torch.as_tensor(L, dtype=F64, device=self.dev)
        g = None if g is None else torch.as_tensor(g, dtype=F64, device=self.dev)
        return L, g

    # ---- initial state -------------------------------------------------------------------
    def init_from_prior(self, theta_center=None, rel=0.0, w_sigma0=1e-4, k0=0):
        """Walkers from the prior (theta uniform in Table I, or a cloud of relative spread rel
        around theta_center), knots as in Sec. III.C: k0 in-between knots at prior positions and
        amplitudes N(0, w_sigma0) (the paper's 1e-8 variance)."""
        S, nsp, kmax = self.S, self.nsp, self.kmax
        lo = torch.as_tensor(THETA_LO, dtype=F64, device=self.dev)
        hi = torch.as_tensor(THETA_HI, dtype=F64, device=self.dev)
        if theta_center is None:
            th = lo + (hi - lo) * self._uniform((S, N_THETA))
        else:
            c = torch.as_tensor(np.asarray(theta_center, dtype=np.float64), device=self.dev)
            th = c + rel * c.abs() * self._normal((S, N_THETA)) * (c.abs() > 0)
            th = torch.minimum(torch.maximum(th, lo), hi)
        if self.sgwb_model == 1:
            th[:, 4] = th[:, 3]
        count = torch.full((S, nsp), int(k0), dtype=torch.int32, device=self.dev)
        x = self.x_lo + (self.x_hi - self.x_lo) * self._uniform((S, nsp, kmax))
        w = w_sigma0 * self._normal((S, nsp, kmax + 2))
        mx, mw = knot_masks(count, kmax)
        zero = torch.zeros((), dtype=F64, device=self.dev)
        self.set_state(State(th, count, torch.where(mx, x, zero), torch.where(mw, w, zero)))

    def set_state(self, st: State):
        self.st = st.to(self.dev).copy()
        self.logL, self.grad = self._like(self.st, True)
        self.lp = log_prior(self.st, self.x_lo, self.x_hi, self.th_idx, self.kmax)

    # ---- within-model move: MALA ----------------------------------------------------------
    def _grad_logpost(self, st: State, g):
        gt, gw, gx = split_grad(g, self.nsp, self.kmax)
        b = self.beta_s
        return b[:, None] * gt, b[:, None, None] * gw - st.w / W_SIGMA ** 2, b[:, None, None] * gx

    def _ensemble_scales(self):
        """Per temperature: spread of each theta coordinate, of the active amplitudes and of the
        active positions over the walkers (floored), the diagonal preconditioner."""
        T, W = self.T, self.W
        th = self.st.theta.reshape(T, W, N_THETA)
        s_th = th.std(dim=1, correction=0)
        floor = torch.as_tensor(1e-6 * (THETA_HI - THETA_LO), dtype=F64, device=self.dev)
        s_th = torch.maximum(s_th, floor[None, :])
        mx, mw = knot_masks(self.st.count, self.kmax)

        def masked_std(v, m, fallback):
            # population spread of the active slots of each temperature (fallback below 2 slots)
            m = m.reshape(T, -1).to(F64)
            v = v.reshape(T, -1)
            n = m.sum(dim=1)
            mean = (v * m).sum(dim=1) / n.clamp(min=1.0)
            sd = torch.sqrt(((v - mean[:, None]) ** 2 * m).sum(dim=1) / n.clamp(min=1.0))
            return torch.clamp(torch.where(n > 1, sd, torch.full_like(sd, fallback)), min=1e-5)

        s_w = masked_std(self.st.w, mw, W_SIGMA)
        s_x = masked_std(self.st.x, mx, 0.1 * (self.x_hi - self.x_lo))
        return s_th, s_w, s_x

    def mala(self):
        if self.scales is None or self.adapting:
            self.scales = self._ensemble_scales()
        s_th, s_w, s_x = (torch.as_tensor(v, dtype=F64, device=self.dev) for v in self.scales)
        T, W, S = self.T, self.W, self.S
        tix = torch.arange(T, device=self.dev).repeat_interleave(W)
        eps = self.eps[tix]
        mth = torch.zeros((S, N_THETA), dtype=F64, device=self.dev)
        mth[:, :len(self.th_idx)] = 1.0
        mx, mw = knot_masks(self.st.count, self.kmax)
        sth = s_th[tix] * mth
        sw = s_w[tix][:, None, None] * mw
        sx = s_x[tix][:, None, None] * mx
        e1, e3 = eps[:, None], eps[:, None, None]

        def drift(st, g):
            gt, gw, gx = self._grad_logpost(st, g)
            return 0.5 * (e1 * sth) ** 2 * gt, 0.5 * (e3 * sw) ** 2 * gw, 0.5 * (e3 * sx) ** 2 * gx

        def logq(to: State, frm: State, d):
            r = torch.zeros(S, dtype=F64, device=self.dev)
            for a, b, dd, sc, e in ((to.theta, frm.theta, d[0], sth, e1), (to.w, frm.w, d[1], sw, e3),
                                    (to.x, frm.x, d[2], sx, e3)):
                var = (e * sc) ** 2
                z = torch.where(var > 0, (a - b - dd) ** 2 / torch.where(var > 0, 2.0 * var, 1.0), 0.0)
                r = r - z.reshape(S, -1).sum(dim=1)
            return r

        ok0 = torch.isfinite(self.logL) & torch.isfinite(self.lp)
        g0 = torch.where(ok0[:, None], self.grad, 0.0)
        d0 = drift(self.st, g0)
        new = self.st.copy()
        new.theta = self.st.theta + d0[0] + e1 * sth * self._normal((S, N_THETA))
        if self.sgwb_model == 1:
            new.theta[:, 4] = new.theta[:, 3]
        new.w = self.st.w + d0[1] + e3 * sw * self._normal(tuple(self.st.w.shape))
        new.x = self.st.x + d0[2] + e3 * sx * self._normal(tuple(self.st.x.shape))
        lp1 = log_prior(new, self.x_lo, self.x_hi, self.th_idx, self.kmax)
        L1, g1 = self._like(new, True)
        ok1 = torch.isfinite(L1) & torch.isfinite(lp1)
        d1 = drift(new, torch.where(ok1[:, None], g1, 0.0))
        b = self.beta_s
        la = (b * L1 + lp1) - (b * self.logL + self.lp) + logq(self.st, new, d1) - logq(new, self.st, d0)
        inf = torch.tensor(math.inf, dtype=F64, device=self.dev)
        la = torch.where(ok1, la, -inf)
        la = torch.where(ok0, la, torch.where(ok1, inf, -inf))   # leave an invalid state at once
        acc = torch.log(self._uniform(S)) < la
        self._accept(acc, new, L1, g1, lp1)
        a_t = acc.reshape(T, W).to(F64).mean(dim=1)
        self.acc["mala"] += a_t
        self.tries["mala"] += 1
        if self.adapting:
            self.eps = torch.clamp(self.eps * torch.exp((a_t - MALA_TARGET) / math.sqrt(self.n_sweeps + 1.0)),
                                   1e-4, 5.0)
        return acc

    def _accept(self, acc, new: State, L1, g1, lp1):
        self.st.put(acc, new)
        self.logL = torch.where(acc, L1, self.logL)
        self.grad = torch.where(acc[:, None], g1, self.grad)
        self.lp = torch.where(acc, lp1, self.lp)

    # ---- between-model move: knot birth / death --------------------------------------------
    def _p_birth(self, k):
        return torch.where(k <= 0, 1.0, torch.where(k >= self.kr, 0.0, 0.5)).to(F64)

    def rj(self):
        S, nsp, kmax = self.S, self.nsp, self.kmax
        if self.kr == 0:
            return torch.zeros(S, dtype=torch.bool, device=self.dev)
        rows = torch.arange(S, device=self.dev)
        a = torch.randint(0, nsp, (S,), generator=self.gen, device=self.dev)
        k = self.st.count[rows, a].long()
        pb = self._p_birth(k)
        birth = self._uniform(S) < pb
        death = ~birth                                   # k >= 1 there (p_birth = 1 at k = 0)
        new = self.st.copy()
        xb = self.x_lo + (self.x_hi - self.x_lo) * self._uniform(S)
        wb = W_SIGMA * self._normal(S)
        jd = torch.minimum((self._uniform(S) * k).long(), (k - 1).clamp(min=0))
        kl = (k - 1).clamp(min=0)                        # the last in-between slot
        # every row changes only its own spline a, at most at the slots below; rows that take the
        # other move write their current values back
        def setx(j, v, m):
            new.x[rows, a, j] = torch.where(m, v, new.x[rows, a, j])

        def setw(j, v, m):
            new.w[rows, a, j] = torch.where(m, v, new.w[rows, a, j])

        # birth: a knot from the prior appended at slot k (k < k_max_rj <= kmax there)
        kb = k.clamp(max=kmax - 1)
        setx(kb, xb, birth)
        setw(k + 1, wb, birth)
        # death: a uniformly chosen in-between knot removed, the last one moved into its slot
        setx(jd, new.x[rows, a, kl], death)
        setw(jd + 1, new.w[rows, a, k], death)
        setx(kl, torch.zeros_like(xb), death)
        setw(k, torch.zeros_like(xb), death)
        new.count[rows, a] = new.count[rows, a] + birth.to(torch.int32) - death.to(torch.int32)
        k1 = new.count[rows, a].long()
        # move-selection ratio q(reverse) / q(forward); the count prior is uniform and the new
        # knot's prior density cancels its proposal density
        tiny = 1e-300
        pb1 = self._p_birth(k1)
        lq = torch.where(birth, torch.log((1.0 - pb1).clamp(min=tiny)) - torch.log(pb.clamp(min=tiny)),
                         torch.log(pb1.clamp(min=tiny)) - torch.log((1.0 - pb).clamp(min=tiny)))
        lp1 = log_prior(new, self.x_lo, self.x_hi, self.th_idx, self.kmax)
        L1, g1 = self._like(new, True)
        ok1 = torch.isfinite(L1) & torch.isfinite(lp1)
        inf = torch.tensor(math.inf, dtype=F64, device=self.dev)
        la = self.beta_s * (L1 - self.logL) + lq
        la = torch.where(ok1, la, -inf)
        la = torch.where(torch.isfinite(self.logL), la, torch.where(ok1, inf, -inf))
        acc = torch.log(self._uniform(S)) < la
        self._accept(acc, new, L1, g1, lp1)
        self.acc["rj"] += acc.reshape(self.T, self.W).to(F64).mean(dim=1)
        self.tries["rj"] += 1
        return acc

    # ---- parallel tempering ----------------------------------------------------------------
    def swap(self):
        """Adjacent-temperature exchanges, hottest pair first; walkers of the hotter temperature
        are paired with a random permutation of the colder one's.  The exchanges are applied to a
        slot -> state index (and to log L), and the states are gathered once at the end."""
        T, W = self.T, self.W
        idx = torch.arange(self.S, device=self.dev)
        L = self.logL.clone()
        for t in range(T - 2, -1, -1):
            c = torch.arange(t * W, (t + 1) * W, device=self.dev)                        # colder
            h = (t + 1) * W + torch.randperm(W, generator=self.gen, device=self.dev)     # hotter
            la = float(self.betas[t] - self.betas[t + 1]) * (L[h] - L[c])
            la = torch.where(torch.isnan(la), -math.inf, la)
            acc = torch.log(self._uniform(W)) < la
            ic, ih = idx[c], idx[h]
            idx[c], idx[h] = torch.where(acc, ih, ic), torch.where(acc, ic, ih)
            Lc, Lh = L[c], L[h]
            L[c], L[h] = torch.where(acc, Lh, Lc), torch.where(acc, Lc, Lh)
            self.acc["swap"][t] += acc.to(F64).mean()
        self.tries["swap"] += 1
        self.st = self.st.gather(idx)
        self.logL, self.lp, self.grad = self.logL[idx], self.lp[idx], self.grad[idx]

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
        then they are frozen).  Returns a dict of recorded numpy arrays: log L of every state
        [n_rec, T, W], and the cold chain's theta [n_rec, W, 5] and knot counts [n_rec, W, nsp]."""
        rec_L, rec_th, rec_k = [], [], []
        for i in range(n_sweeps):
            self.adapting = i < n_adapt
            self.sweep()
            if i >= n_adapt and (i - n_adapt) % record_every == 0:
                rec_L.append(self.logL.reshape(self.T, self.W).clone())
                rec_th.append(self.st.theta[:self.W].clone())
                rec_k.append(self.st.count[:self.W].clone())
        self.adapting = False

        def stack(v):
            return torch.stack(v).cpu().numpy() if v else np.array([])
        return {"logL": stack(rec_L), "theta": stack(rec_th), "count": stack(rec_k)}

    def acceptance(self):
        return {k: (self.acc[k] / max(self.tries[k], 1)).cpu().numpy() for k in self.acc}


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
