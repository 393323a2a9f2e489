"""Pins for the oracle's perturbation splines (Sec. III.A knot scheme, Appendix A Akima).

Independent library routines: scipy.interpolate.Akima1DInterpolator (whose end conditions
Appendix A says it follows), CubicSpline(bc_type='natural') and numpy.interp; plus exact
interpolation, exact reproduction of linear data, the paper's worked example and the knot
validation rules."""
import os

import numpy as np
import pytest
from scipy.interpolate import Akima1DInterpolator, CubicSpline

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "perturbed_noise_spline.txt")
X_LO, X_HI = -4.0, np.log10(2.9e-2)


def random_knots(rng, k, x_lo=X_LO, x_hi=X_HI):
    xi = rng.uniform(x_lo, x_hi, k)
    w = rng.normal(0, 0.1, k + 2)
    return xi, w


def sorted_points(xi, w, x_lo, x_hi):
    order = np.argsort(xi)
    xs = np.concatenate([[x_lo], xi[order], [x_hi]])
    ys = np.concatenate([[w[0]], w[1:-1][order], [w[-1]]])
    return xs, ys


@pytest.mark.parametrize("seed", range(12))
def test_akima_matches_scipy(seed):
    rng = np.random.default_rng(seed)
    k = int(rng.integers(2, 31))
    xi, w = random_knots(rng, k)
    xs, ys = sorted_points(xi, w, X_LO, X_HI)
    ref = Akima1DInterpolator(xs, ys, extrapolate=True)
    x = np.concatenate([rng.uniform(X_LO - 0.3, X_HI + 0.3, 400), xs])
    st, val = oracle.spline_eval(0, xi, w, X_LO, X_HI, x)
    assert st == 0
    np.testing.assert_allclose(val, ref(x), rtol=1e-13, atol=1e-12)
    st, xs_o, ys_o, coef = oracle.spline_coeffs(0, xi, w, X_LO, X_HI)
    np.testing.assert_array_equal(xs_o, xs)
    # SciPy PPoly stores the highest power first: c[0] = d, c[1] = c, c[2] = b, c[3] = a.
    np.testing.assert_allclose(coef[:, ::-1].T, ref.c, rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("ys", [
    [0.0, 0.0, 0.0, 1.0, 2.0, 2.0, 2.0, 5.0],     # flat run, ramp, flat run: exact weight ties
    [0.0, 1.0, 2.0, 3.0, 3.0, 3.0, 2.0, 1.0],
    [1.0, 1.0, 1.0, 1.0, 1.0, 1.0],
    [0.0, 1.0, 0.0, 1.0, 0.0, 1.0, 0.0],
])
def test_akima_exact_ties_match_scipy(ys):
    ys = np.asarray(ys, dtype=float)
    n = ys.size
    xs = np.arange(n, dtype=float)            # exact arithmetic: ties are exact zeros
    xi, w = xs[1:-1], np.concatenate([[ys[0]], ys[1:-1], [ys[-1]]])
    ref = Akima1DInterpolator(xs, ys, extrapolate=True)
    x = np.linspace(-0.5, n - 0.5, 301)
    st, val = oracle.spline_eval(0, xi, w, xs[0], xs[-1], x)
    assert st == 0
    np.testing.assert_allclose(val, ref(x), rtol=0, atol=1e-13)


@pytest.mark.parametrize("kind", [0, 1])
def test_interpolates_knots_exactly_and_reproduces_lines(kind):
    rng = np.random.default_rng(5)
    for k in (0, 1, 2, 3, 7, 20):
        xi, w = random_knots(rng, k)
        xs, ys = sorted_points(xi, w, X_LO, X_HI)
        st, val = oracle.spline_eval(kind, xi, w, X_LO, X_HI, xs)
        assert st == 0
        np.testing.assert_allclose(val, ys, rtol=0, atol=2e-16)
        # linear data y = 0.3 x - 0.1 is reproduced up to rounding (all slopes equal)
        wl = 0.3 * np.concatenate([[X_LO], xi, [X_HI]]) - 0.1
        x = rng.uniform(X_LO - 0.2, X_HI + 0.2, 100)
        st, val = oracle.spline_eval(kind, xi, wl, X_LO, X_HI, x)
        np.testing.assert_allclose(val, 0.3 * x - 0.1, rtol=0, atol=1e-12)


@pytest.mark.parametrize("k", [0, 1])
def test_linear_fallback_matches_numpy_interp(k):
    rng = np.random.default_rng(11 + k)
    for _ in range(5):
        xi, w = random_knots(rng, k)
        xs, ys = sorted_points(xi, w, X_LO, X_HI)
        x = rng.uniform(X_LO, X_HI, 200)
        for kind in (0, 1):
            st, val = oracle.spline_eval(kind, xi, w, X_LO, X_HI, x)
            np.testing.assert_allclose(val, np.interp(x, xs, ys), rtol=0, atol=1e-15)
        # outside the edges: the end segments extended
        st, val = oracle.spline_eval(0, xi, w, X_LO, X_HI, np.array([X_LO - 0.5, X_HI + 0.5]))
        s0 = (ys[1] - ys[0]) / (xs[1] - xs[0])
        s1 = (ys[-1] - ys[-2]) / (xs[-1] - xs[-2])
        np.testing.assert_allclose(val, [ys[0] - 0.5 * s0, ys[-1] + 0.5 * s1], atol=1e-14)


@pytest.mark.parametrize("seed", range(8))
def test_natural_cubic_matches_scipy(seed):
    rng = np.random.default_rng(100 + seed)
    k = int(rng.integers(2, 41))
    xi, w = random_knots(rng, k)
    xs, ys = sorted_points(xi, w, X_LO, X_HI)
    ref = CubicSpline(xs, ys, bc_type="natural", extrapolate=True)
    x = np.concatenate([rng.uniform(X_LO - 0.3, X_HI + 0.3, 400), xs])
    st, val = oracle.spline_eval(1, xi, w, X_LO, X_HI, x)
    assert st == 0
    np.testing.assert_allclose(val, ref(x), rtol=1e-12, atol=1e-11 * max(1.0, np.abs(ref.c).max()))


def test_worked_example_perturbed_noise():
    data = np.loadtxt(GOLDEN)
    xk, wk = data[:, 0], data[:, 1]
    x_lo, x_hi = xk[0], xk[-1]
    xi = xk[1:-1]
    st, xs, ys, coef = oracle.spline_coeffs(0, xi, wk, x_lo, x_hi)
    assert st == 0 and xs.size == 6            # 4 in-between knots: the Akima branch
    assert np.any(coef[:, 3] != 0.0)           # genuinely cubic, not the linear fallback
    st, val = oracle.spline_eval(0, xi, wk, x_lo, x_hi, xk)
    np.testing.assert_allclose(10.0 ** val, 10.0 ** wk, rtol=1e-15)
    assert val[0] == 0.0 and abs(val[-1]) < 1e-15     # the last knot closes the last interval
    ref = Akima1DInterpolator(xk, wk)
    x = np.linspace(x_lo, x_hi, 1001)
    st, val = oracle.spline_eval(0, xi, wk, x_lo, x_hi, x)
    np.testing.assert_allclose(val, ref(x), atol=1e-13)


def test_knot_order_does_not_matter():
    rng = np.random.default_rng(3)
    xi, w = random_knots(rng, 9)
    perm = rng.permutation(9)
    w2 = np.concatenate([[w[0]], w[1:-1][perm], [w[-1]]])
    for kind in (0, 1):
        a = oracle.spline_coeffs(kind, xi, w, X_LO, X_HI)
        b = oracle.spline_coeffs(kind, xi[perm], w2, X_LO, X_HI)
        np.testing.assert_array_equal(a[3], b[3])


def test_knot_validation_status_bits():
    w = np.zeros(5)
    assert oracle.spline_coeffs(0, [-3.0, -3.0, -2.0], w, X_LO, X_HI)[0] == 4      # duplicate
    assert oracle.spline_coeffs(0, [-3.0, X_LO, -2.0], w, X_LO, X_HI)[0] == 2      # on the edge
    assert oracle.spline_coeffs(0, [-3.0, -5.0, -2.0], w, X_LO, X_HI)[0] == 2      # outside
    assert oracle.spline_coeffs(0, [-3.0, np.nan, -2.0], w, X_LO, X_HI)[0] == 2
    bad_w = np.array([0.0, np.inf, 0.0, 0.0, 0.0])
    assert oracle.spline_coeffs(0, [-3.0, -2.5, -2.0], bad_w, X_LO, X_HI)[0] == 8
