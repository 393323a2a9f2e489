"""Pins for the oracle's gradient condition scale (``oracle.loglike_grad_scale``).

The scale of a gradient component is the sum of the absolute values of the terms its sum is
made of.  Every FP32 gradient bound of the GPU tests is a multiple of it, so a mistake in it (a
dropped absolute value, a wrong slope branch, a factor of two) would loosen those bounds without
any test failing.  The log-likelihood being differentiated is the per-bin Wishart term of
Sec. III.C, -nu sum_c (P_c/S_c + ln S_c), with S_c from Eq. (splines):

    d log L / d S_c,i = g_c,i = nu_i (P_c,i - S_c,i) / S_c,i^2.

Template parameters (a_oms, a_tm, log10 A, n1, n2) sum one term per (bin, channel):

    a_oms:   g 2 a_oms U_oms,c 10^{P_c}        U_oms = the noise template per unit a_oms
    a_tm:    g 2 a_tm  U_tm,c  10^{P_c}        U_tm  = the noise template per unit a_tm
    log10 A: g ln10 S_h,c 10^{P_h}
    n1, n2:  g ln(f / f_ref) S_h,c 10^{P_h}    below / at-and-above f_ref (broken power law)

Knot parameters sum one term per bin, q_a,i dP_a(x_i)/d(knot), with q the derivative of log L
with respect to the spline value: g_a ln10 S_n,a 10^{P_a} for the noise spline of channel a and
sum_c g_c ln10 S_h,c 10^{P_h} for the SGWB spline.

The pins rebuild those sums here from pieces pinned elsewhere (model PSD, templates, spline
values) and from central differences of the spline values, and check the two properties every
scale must have: |gradient| <= scale, with equality when all terms share one sign."""
import math

import numpy as np
import pytest

import oracle
from paper_2507_06300_gb300 import synth
from tests._workloads import oracle_dataset

LN10 = math.log(10.0)


def _spline_values(kind, kn, s, a, x_lo, x_hi, x, dw=None, dx=None):
    """P_a(x) of state s from the oracle's spline evaluator; dw = (slot, delta) perturbs one
    amplitude slot, dx = (j, delta) one in-between position."""
    kmax = kn["kmax"]
    k = int(kn["count"][s, a])
    xi = np.array(kn["x"][s, a, :k], dtype=np.float64)
    w = np.concatenate([kn["w"][s, a, :1 + k], kn["w"][s, a, kmax + 1:kmax + 2]]).astype(np.float64)
    if dw is not None:
        slot, h = dw
        w[slot if slot <= k else k + 1] += h
    if dx is not None:
        j, h = dx
        xi[j] += h
    st, v = oracle.spline_eval(kind, xi, w, x_lo, x_hi, x)
    assert st == 0
    return v


def _pieces(ds, th, kn, s):
    """Per-bin pieces of state s: g [C, N], noise templates and SGWB templates, the spline
    values, and q [nsp, N]."""
    f = ds["f"]
    C = int(ds["n_channels"])
    sg = int(ds.get("sgwb_model", 1))
    nsp = C + (1 if sg else 0)
    x = np.log10(f)
    kind = int(kn.get("kind", 0))
    one = {k: (v[s:s + 1] if isinstance(v, np.ndarray) else v) for k, v in kn.items()}
    S, st = oracle.model_psd(ds, th[s:s + 1], one)
    assert st[0] == 0
    S = S[0]
    g = ds["nu"] * (ds["P"] - S) / S ** 2
    U_o = oracle.noise_templates(f, 1.0, 0.0)[:C]
    U_t = oracle.noise_templates(f, 0.0, 1.0)[:C]
    Sn = th[s, 0] ** 2 * U_o + th[s, 1] ** 2 * U_t
    P = np.array([_spline_values(kind, kn, s, a, ds["x_lo"], ds["x_hi"], x) for a in range(nsp)])
    En = 10.0 ** P[:C]
    if sg:
        Sh = np.array([oracle.sgwb_template(f, ds["R"][c], th[s, 2], th[s, 3], th[s, 4], ds["f_ref"], sg)
                       for c in range(C)])
        Eh = 10.0 ** P[C]
    else:
        Sh, Eh = np.zeros((C, f.size)), np.zeros(f.size)
    q = np.empty((nsp, f.size))
    q[:C] = g * LN10 * Sn * En
    if sg:
        q[C] = np.sum(g * LN10 * Sh * Eh, axis=0)
    return dict(S=S, g=g, U_o=U_o, U_t=U_t, Sn=Sn, En=En, Sh=Sh, Eh=Eh, q=q, x=x, kind=kind, nsp=nsp, C=C, sg=sg)


def _template_scales(ds, th, s, pc):
    g, En = pc["g"], pc["En"]
    lnf = np.log(ds["f"] / ds["f_ref"])
    out = np.zeros(5)
    out[0] = np.abs(g * 2.0 * th[s, 0] * pc["U_o"] * En).sum()
    out[1] = np.abs(g * 2.0 * th[s, 1] * pc["U_t"] * En).sum()
    if pc["sg"]:
        H = g * pc["Sh"] * pc["Eh"]
        out[2] = np.abs(LN10 * H).sum()
        if pc["sg"] == 2:
            below = ds["f"] < ds["f_ref"]
            out[3] = np.abs(H * lnf)[:, below].sum()
            out[4] = np.abs(H * lnf)[:, ~below].sum()
        else:
            out[3] = np.abs(H * lnf).sum()
    return out


def _knot_scale_fd(ds, kn, s, a, pc, which, idx, h=1e-6):
    """sum_i |q_a,i dP_a(x_i)/d(knot)| with the derivative by central differences."""
    kw = dict(dw=(idx, h)) if which == "w" else dict(dx=(idx, h))
    km = dict(dw=(idx, -h)) if which == "w" else dict(dx=(idx, -h))
    vp = _spline_values(pc["kind"], kn, s, a, ds["x_lo"], ds["x_hi"], pc["x"], **kw)
    vm = _spline_values(pc["kind"], kn, s, a, ds["x_lo"], ds["x_hi"], pc["x"], **km)
    return np.abs(pc["q"][a] * (vp - vm) / (2 * h)).sum()


def _knots(rng, nsp, kmax, count, kind):
    count = np.asarray(count, np.int32).reshape(1, nsp)
    x = np.zeros((1, nsp, kmax))
    for a in range(nsp):
        x[0, a, :count[0, a]] = rng.permutation(np.sort(rng.uniform(-3.9, -1.6, count[0, a])))
    w = rng.normal(0.0, 0.1, (1, nsp, kmax + 2))
    for a in range(nsp):
        w[0, a, 1 + count[0, a]:kmax + 1] = 0.0
    return {"count": count, "x": x, "w": w, "kmax": kmax, "kind": kind}


@pytest.fixture(scope="module")
def tiny():
    wl = synth.workload("tiny")
    return wl, oracle_dataset(wl)


@pytest.mark.parametrize("sgwb_model, kind", [(1, 0), (2, 0), (1, 1)])
def test_scale_matches_rebuilt_sums(tiny, sgwb_model, kind):
    """Every component of the scale equals the same sum rebuilt from pinned pieces: template
    components from the closed-form dS/d(parameter), knot components from central differences
    of the spline values."""
    wl, ds = tiny
    ds = dict(ds, sgwb_model=sgwb_model, f_ref=3e-3)
    rng = np.random.default_rng(101 + sgwb_model + 10 * kind)
    nsp, kmax = 4, 5
    kn = _knots(rng, nsp, kmax, [4, 2, 0, 3], kind)
    th = np.array([[14.0, 3.2, -11.9, 0.5, -0.8]])
    L, G, scale, st = oracle.loglike_grad_scale(ds, th, kn)
    assert st[0] == 0
    pc = _pieces(ds, th, kn, 0)
    expect_t = _template_scales(ds, th, 0, pc)
    n_t = 5 if sgwb_model == 2 else 4
    np.testing.assert_allclose(scale[0, :n_t], expect_t[:n_t], rtol=1e-12)
    if sgwb_model != 2:
        assert scale[0, 4] == 0.0
    for a in range(nsp):
        base = 5 + a * (2 * kmax + 2)
        k = int(kn["count"][0, a])
        for slot in [0] + list(range(1, k + 1)) + [kmax + 1]:
            fd = _knot_scale_fd(ds, kn, 0, a, pc, "w", slot)
            assert scale[0, base + slot] == pytest.approx(fd, rel=1e-6), ("w", a, slot)
        for j in range(k):
            fd = _knot_scale_fd(ds, kn, 0, a, pc, "x", j)
            assert scale[0, base + kmax + 2 + j] == pytest.approx(fd, rel=1e-5), ("x", a, j)
        # inactive slots: no terms
        assert np.all(scale[0, base + 1 + k: base + kmax + 1] == 0)
        assert np.all(scale[0, base + kmax + 2 + k: base + 2 * kmax + 2] == 0)


def test_scale_bounds_gradient(tiny):
    """Triangle inequality, every component of every state of the tiny workload."""
    wl, ds = tiny
    th, kn = wl.states(0)
    L, G, scale, st = oracle.loglike_grad_scale(ds, th, kn.as_dict())
    ok = st == 0
    assert ok.sum() >= 3
    assert np.all(scale[ok] >= 0)
    assert np.all(np.abs(G[ok]) <= scale[ok] * (1 + 1e-12) + 1e-300)
    # a component with any nonzero term has a nonzero scale
    assert np.all(scale[ok][G[ok] != 0] > 0)


def test_scale_equals_gradient_when_terms_share_a_sign():
    """Noise-only model, P = 2 S: g = nu / S > 0 in every bin, so every a_oms and a_tm term is
    positive, and with 0 or 1 in-between knots (linear fallback, hat-function derivatives >= 0)
    every amplitude term is positive too: the scale is |gradient| exactly."""
    f = synth.freq_grid(400)
    C = 3
    ds = {"n_channels": C, "sgwb_model": 0, "f": f, "nu": np.full(f.size, 8.0), "x_lo": -4.0,
          "x_hi": math.log10(2.9e-2), "f_ref": 1e-3}
    kmax, nsp = 2, C
    rng = np.random.default_rng(7)
    count = np.array([[0, 1, 1]], np.int32)
    x = np.zeros((1, nsp, kmax))
    x[0, 1, 0], x[0, 2, 0] = -2.7, -3.3
    w = rng.normal(0.0, 0.1, (1, nsp, kmax + 2))
    w[0, 0, 1:kmax + 1] = 0.0
    w[0, 1:, 2:kmax + 1] = 0.0
    kn = {"count": count, "x": x, "w": w, "kmax": kmax, "kind": 0}
    th = np.array([[12.0, 4.0, 0.0, 0.0, 0.0]])
    S, st = oracle.model_psd(ds, th, kn)
    assert st[0] == 0
    ds["P"] = 2.0 * S[0]
    L, G, scale, st = oracle.loglike_grad_scale(ds, th, kn)
    assert st[0] == 0
    assert G[0, 0] > 0 and G[0, 1] > 0
    np.testing.assert_allclose(scale[0, :2], G[0, :2], rtol=1e-13)
    for a in range(nsp):
        base = 5 + a * (2 * kmax + 2)
        for slot in [0] + list(range(1, int(count[0, a]) + 1)) + [kmax + 1]:
            assert G[0, base + slot] > 0
            assert scale[0, base + slot] == pytest.approx(G[0, base + slot], rel=1e-13)


def test_scale_of_positions_sees_both_signs():
    """With P = 2 S the amplitude terms share a sign, but dP/dx_k changes sign across the knot
    (the hat moves right: its rising side drops, its falling side rises), so the position scale
    is strictly larger than |gradient| -- a scale computed as |sum| instead of sum |.| fails."""
    f = synth.freq_grid(400)
    ds = {"n_channels": 2, "sgwb_model": 0, "f": f, "nu": np.full(f.size, 8.0), "x_lo": -4.0,
          "x_hi": math.log10(2.9e-2), "f_ref": 1e-3}
    kmax = 1
    kn = {"count": np.array([[1, 0]], np.int32), "x": np.array([[[-2.5], [0.0]]]),
          "w": np.array([[[0.05, 0.3, -0.1], [0.0, 0.0, 0.02]]]), "kmax": kmax, "kind": 0}
    th = np.array([[12.0, 4.0, 0.0, 0.0, 0.0]])
    S, st = oracle.model_psd(ds, th, kn)
    ds["P"] = 2.0 * S[0]
    L, G, scale, st = oracle.loglike_grad_scale(ds, th, kn)
    assert st[0] == 0
    gx = 5 + kmax + 2           # d/dx of the one knot of spline 0
    assert scale[0, gx] > 1.05 * abs(G[0, gx])
    pc = _pieces(ds, th, kn, 0)
    assert scale[0, gx] == pytest.approx(_knot_scale_fd(ds, kn, 0, 0, pc, "x", 0), rel=1e-5)
