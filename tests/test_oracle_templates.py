"""Pins for the oracle's PSD templates (Sec. II.B, Eq. noise_tdi; Sec. II.C, Eq. pl, Eq. Sh).

The transfer functions are checked at phases u = 2 pi f L / c where sin and cos take exact
values (hand-derived closed forms), in the low-frequency limit (Taylor expansion), and the
SGWB template against the paper's printed Hubble constant and its power-law scaling."""
import math

import numpy as np
import pytest

import oracle

C_LIGHT = 299792458.0
L_ARM = 2.5e9


def f_at_phase(u):
    return u * C_LIGHT / (2.0 * math.pi * L_ARM)


def link(f, a_oms=15.0, a_tm=3.0):
    s = oracle.link_psds(np.atleast_1d(f), a_oms, a_tm)
    return s[0, 0], s[1, 0]


@pytest.mark.parametrize("u, pref0, pref1, cu", [
    (math.pi / 2, 1.0, 0.0, 0.0),            # sin u = 1, cos u = 0, sin 2u = 0
    (math.pi / 3, 27.0 / 64.0, 9.0 / 16.0, 0.5),
    (2 * math.pi / 3, 27.0 / 64.0, 9.0 / 16.0, -0.5),
])
def test_transfer_at_exact_phases(u, pref0, pref1, cu):
    f = f_at_phase(u)
    so, st = link(f)
    # hand-derived brackets: A/E: (2 + cos u) S_OMS + 4 (1 + cos u + cos^2 u) S_TM
    #                        T:   (1 - cos u) S_OMS + 2 (1 - cos u)^2 S_TM
    br_ae = (2 + cu) * so + 4 * (1 + cu + cu * cu) * st
    br_t = (1 - cu) * so + 2 * (1 - cu) ** 2 * st
    for form, pref in ((0, pref0), (1, pref1)):
        out = oracle.noise_templates(np.array([f]), 15.0, 3.0, form)[:, 0]
        scale = 32 * br_ae
        assert abs(out[0] - 32 * pref * br_ae) <= 1e-13 * scale
        assert out[1] == out[0]
        assert abs(out[2] - 64 * pref * br_t) <= 1e-13 * 64 * br_t


def test_low_frequency_limit_without_cancellation():
    # u ~ 5e-6: sin u = u (1 - u^2/6), 1 - cos u = u^2/2 (1 - u^2/12); corrections ~1e-11.
    f = 1.0e-7
    u = 2 * math.pi * f * L_ARM / C_LIGHT
    so, st = link(f)
    out0 = oracle.noise_templates(np.array([f]), 15.0, 3.0, 0)[:, 0]
    out1 = oracle.noise_templates(np.array([f]), 15.0, 3.0, 1)[:, 0]
    omc = u * u / 2
    assert out0[0] == pytest.approx(32 * u ** 6 * (3 * so + 12 * st), rel=1e-9, abs=0)
    assert out0[2] == pytest.approx(64 * u ** 6 * (omc * so + 2 * omc ** 2 * st), rel=1e-9, abs=0)
    assert out1[0] == pytest.approx(32 * u ** 2 * 4 * u ** 2 * (3 * so + 12 * st), rel=1e-9, abs=0)
    assert out1[2] == pytest.approx(64 * 4 * u ** 4 * (omc * so + 2 * omc ** 2 * st), rel=1e-9, abs=0)


def test_link_psd_corner_frequencies():
    # S_OMS / (A_OMS^2 (2 pi f / c)^2) = 1 + (2 mHz / f)^4 ; S_TM (2 pi f c)^2 / A_TM^2 =
    # [1 + (0.4 mHz/f)^2][1 + (f / 8 mHz)^4].  Values at the corner frequencies:
    for f, expect in ((2e-3, 2.0), (1e-3, 17.0), (4e-3, 1.0625)):
        so, _ = link(f, 7.9, 2.4)
        assert so / ((7.9e-12) ** 2 * (2 * math.pi * f / C_LIGHT) ** 2) == pytest.approx(expect, rel=1e-14, abs=0)
    for f, expect in ((0.4e-3, 2.0 * (1 + 0.05 ** 4)), (8e-3, 2.0 * (1 + 0.05 ** 2))):
        _, st = link(f, 7.9, 2.4)
        assert st * (2 * math.pi * f * C_LIGHT) ** 2 / (2.4e-15) ** 2 == pytest.approx(expect, rel=1e-14, abs=0)


def test_noise_scales_with_amplitudes_squared():
    f = np.geomspace(1e-4, 2.9e-2, 50)
    base = oracle.noise_templates(f, 1.0, 0.0)
    tm = oracle.noise_templates(f, 0.0, 1.0)
    both = oracle.noise_templates(f, 7.0, 0.5)
    np.testing.assert_allclose(both, 49 * base + 0.25 * tm, rtol=1e-14)


def test_sgwb_hubble_constant_matches_paper():
    # Sec. II.C: H0 = h x 100 km/s/Mpc ~ h x 3.24e-18 Hz.  At f = f_ref, h^2 Omega = A.
    f = np.array([1e-3])
    R = np.array([1.0])
    sh = oracle.sgwb_template(f, R, 0.0, 0.0, f_ref=1e-3)[0]
    H = math.sqrt(sh * 4 * math.pi ** 2 * f[0] ** 3 / 3.0)
    assert abs(H - 3.24e-18) / 3.24e-18 < 5e-4


@pytest.mark.parametrize("n", [-1.0, 0.0, 2.0 / 3.0, 3.0])
def test_sgwb_power_law_scaling(n):
    f = np.array([2e-3, 4e-3])
    R = np.array([0.7, 0.7])
    sh = oracle.sgwb_template(f, R, -12.0, n, f_ref=1e-3)
    assert sh[1] / sh[0] == pytest.approx(2.0 ** (n - 3.0), rel=1e-13, abs=0)
    sh2 = oracle.sgwb_template(f, 2 * R, -11.0, n, f_ref=1e-3)
    np.testing.assert_allclose(sh2, 20 * sh, rtol=1e-13)


def test_broken_power_law_slopes_and_continuity():
    fk = 3e-3
    f = np.array([fk / 2, fk, 2 * fk, np.nextafter(fk, 0)])
    R = np.ones(4)
    sh = oracle.sgwb_template(f, R, -12.0, 2.0 / 3.0, -1.0, f_ref=fk, sgwb_model=2)
    assert sh[0] / (sh[1] * 8) == pytest.approx(2.0 ** (-2.0 / 3.0), rel=1e-13, abs=0)  # below: n1
    assert sh[2] * 8 / sh[1] == pytest.approx(2.0 ** (-1.0), rel=1e-13, abs=0)         # above: n2
    assert sh[3] == pytest.approx(sh[1], rel=1e-12, abs=0)                               # continuous
