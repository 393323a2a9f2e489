"""Pins for the oracle's full-covariance log-likelihood (reading R16 of the dense 3x3 covariance the
paper names as the complete analysis, Sec. III.A; the Wishart term of Sec. III.C).

* The construction C = D^{1/2} R D^{1/2} + H is rebuilt here from pieces pinned elsewhere (noise
  and SGWB templates, spline values) with numpy, and R checked to be a correlation matrix.
* log L against numpy.linalg (solve, slogdet) on the complex Hermitian periodogram, bin by bin.
* Zero correlation splines reproduce the diagonal model's log L exactly, whatever the data's
  off-diagonal entries are.
* Basis changes: the XYZ basis (A, E, T are an orthogonal transform of X, Y, Z) leaves log L
  unchanged; any invertible real M shifts it by -sum(nu) ln det(M)^2 exactly.
* P = C gives log L = -sum nu (3 + ln det C) (tr(C^-1 C) = 3).
* Imaginary parts of the periodogram's off-diagonal entries cancel in the trace.
* Extreme correlation values keep C positive definite."""
import math

import numpy as np
import pytest

import oracle
from paper_2507_06300_gb300 import synth
from tests._workloads import colour_wishart, hermitian, oracle_dataset

NU = 8.0


def _knots(rng, S, nsp, kmax, kind=0, zscale=0.3, kmin=0):
    count = rng.integers(kmin, kmax + 1, size=(S, nsp)).astype(np.int32)
    x = np.zeros((S, nsp, kmax))
    for s in range(S):
        for a in range(nsp):
            x[s, a, :count[s, a]] = rng.uniform(-3.95, -1.6, count[s, a])
    w = rng.normal(0.0, 0.1, (S, nsp, kmax + 2))
    w[:, nsp - 3:, :] = rng.normal(0.0, zscale, (S, 3, kmax + 2))    # correlation splines
    for s in range(S):
        for a in range(nsp):
            w[s, a, 1 + count[s, a]:kmax + 1] = 0.0
    return {"count": count, "x": x, "w": w, "kmax": kmax, "kind": kind}


def _cov_matrix(c6):
    N = c6.shape[1]
    C = np.empty((N, 3, 3))
    C[:, 0, 0], C[:, 1, 1], C[:, 2, 2] = c6[0], c6[1], c6[2]
    C[:, 0, 1] = C[:, 1, 0] = c6[3]
    C[:, 0, 2] = C[:, 2, 0] = c6[4]
    C[:, 1, 2] = C[:, 2, 1] = c6[5]
    return C


@pytest.fixture(scope="module")
def full():
    """A 300-bin A,E,T dataset whose averaged periodogram is a complex Wishart draw around a
    covariance with correlations of a few per cent, and states with random correlation splines."""
    wl = synth.workload("tiny")
    ds = wl.dataset(0)
    ds["nu"] = np.full(wl.n_bins, NU)
    nsp = oracle.n_splines_full(ds)
    rng = np.random.default_rng(11)
    kmax = 4
    kn_true = {"count": np.zeros((1, nsp), np.int32), "x": np.zeros((1, nsp, kmax)),
               "w": np.zeros((1, nsp, kmax + 2)), "kmax": kmax, "kind": 0}
    kn_true["w"][0, nsp - 3:, :] = [[0.1, 0, 0, 0, 0, 0.1], [0.05, 0, 0, 0, 0, 0.05], [-0.08, 0, 0, 0, 0, -0.08]]
    C_true, st = oracle.model_cov_full(ds, wl.theta_true, kn_true)
    assert st[0] == 0
    W = synth.complex_wishart_unit(rng, ds["nu"])
    ds["P9"] = colour_wishart(C_true[0], W)
    th = np.concatenate([wl.theta_true, wl.theta[:5]])
    kn = _knots(rng, 6, nsp, kmax)
    return ds, th, kn


def test_covariance_construction(full):
    ds, th, kn = full
    C6, st = oracle.model_cov_full(ds, th, kn)
    assert not st.any()
    nsp = oracle.n_splines_full(ds)
    f, x = ds["f"], np.log10(ds["f"])
    for s in range(th.shape[0]):
        k = kn["count"][s]
        P = []
        for a in range(nsp):
            w = np.concatenate([kn["w"][s, a, :1 + k[a]], kn["w"][s, a, kn["kmax"] + 1:]])
            st_a, v = oracle.spline_eval(0, kn["x"][s, a, :k[a]], w, ds["x_lo"], ds["x_hi"], x)
            assert st_a == 0
            P.append(v)
        sn = oracle.noise_templates(f, th[s, 0], th[s, 1])
        D = sn * 10.0 ** np.array(P[:3])
        H = np.array([oracle.sgwb_template(f, ds["R"][c], th[s, 2], th[s, 3], th[s, 4], ds["f_ref"], 1)
                      for c in range(3)]) * 10.0 ** P[3]
        z = np.array(P[4:7])
        r = z / np.sqrt(1 + z * z)
        q = 1 / np.sqrt(1 + z * z)
        Lam = np.zeros((f.size, 3, 3))
        Lam[:, 0, 0] = 1
        Lam[:, 1, 0], Lam[:, 1, 1] = r[0], q[0]
        Lam[:, 2, 0], Lam[:, 2, 1], Lam[:, 2, 2] = r[1], r[2] * q[1], q[1] * q[2]
        R = Lam @ np.transpose(Lam, (0, 2, 1))
        np.testing.assert_allclose(np.diagonal(R, axis1=1, axis2=2), 1.0, rtol=1e-14)
        assert np.all(np.abs(R) <= 1 + 1e-14)
        sd = np.sqrt(D.T)
        C = sd[:, :, None] * R * sd[:, None, :]
        C[:, [0, 1, 2], [0, 1, 2]] += H.T
        # diagonal relative; off-diagonal relative to sqrt(C_aa C_bb) (a correlation near its zero
        # crossing has no relative accuracy: here and in the oracle x = log10 f is rounded apart)
        Co = _cov_matrix(C6[s])
        dg = np.sqrt(np.diagonal(C, axis1=1, axis2=2))
        np.testing.assert_allclose(np.diagonal(Co, axis1=1, axis2=2), np.diagonal(C, axis1=1, axis2=2), rtol=1e-13)
        np.testing.assert_allclose(Co / (dg[:, :, None] * dg[:, None, :]), C / (dg[:, :, None] * dg[:, None, :]),
                                   rtol=0, atol=1e-13)
        assert np.all(np.linalg.eigvalsh(C / np.sqrt(D.T[:, :, None] * D.T[:, None, :])) > 0)


def test_loglike_against_numpy_linalg(full):
    ds, th, kn = full
    L, st = oracle.loglike_full(ds, th, kn)
    C6, _ = oracle.model_cov_full(ds, th, kn)
    P = hermitian(ds["P9"])
    for s in range(th.shape[0]):
        C = _cov_matrix(C6[s]).astype(np.complex128)
        tr = np.trace(np.linalg.solve(C, P), axis1=1, axis2=2)
        sign, ld = np.linalg.slogdet(C)
        assert np.all(sign.real > 0)
        ref = -np.sum(ds["nu"] * (tr.real + ld))
        assert np.max(np.abs(tr.imag)) < 1e-10 * np.max(np.abs(tr.real))
        assert L[s] == pytest.approx(ref, rel=1e-11, abs=0)


def test_zero_correlations_reduce_to_the_diagonal_model(full):
    ds, th, kn = full
    nsp = oracle.n_splines_full(ds)
    kn0 = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in kn.items()}
    kn0["count"][:, nsp - 3:] = 0
    kn0["w"][:, nsp - 3:, :] = 0.0
    L_full, st = oracle.loglike_full(ds, th, kn0)
    dsd = dict(ds, P=ds["P9"][:3])
    knd = {"count": kn0["count"][:, :4], "x": kn0["x"][:, :4], "w": kn0["w"][:, :4], "kmax": kn0["kmax"],
           "kind": kn0["kind"]}
    L_diag, st_d = oracle.loglike(dsd, th, knd)
    np.testing.assert_array_equal(st, st_d)
    np.testing.assert_allclose(L_full, L_diag, rtol=1e-13, atol=0)


def _wishart_numpy(C, P, nu):
    tr = np.trace(np.linalg.solve(C, P), axis1=1, axis2=2).real
    return -np.sum(nu * (tr + np.linalg.slogdet(C)[1]))


def test_basis_change(full):
    """A change of basis d' = M d multiplies det C by det(M)^2 and leaves tr(C^-1 P) alone, so
    log L shifts by -sum(nu) ln det(M)^2 exactly (zero for an orthogonal M, such as XYZ from
    A, E, T: A = (Z - X)/sqrt2, E = (X - 2Y + Z)/sqrt6, T = (X + Y + Z)/sqrt3, Sec. II.A).  The
    per-bin scaling by 1/sqrt(P_cc) (a diagonal M) is applied first, which keeps the matrices
    numpy solves well conditioned; the general M is then applied on top."""
    ds, th, kn = full
    L, st = oracle.loglike_full(ds, th, kn)
    C6, _ = oracle.model_cov_full(ds, th, kn)
    P = hermitian(ds["P9"])
    sd = 1.0 / np.sqrt(ds["P9"][:3].T)                       # [N, 3]
    scale_shift = np.sum(ds["nu"] * np.log(ds["P9"][:3]).sum(axis=0))
    M_aet = np.array([[-1, 0, 1], [1, -2, 1], [1, 1, 1]], float) / np.array([[math.sqrt(2)], [math.sqrt(6)], [math.sqrt(3)]])
    np.testing.assert_allclose(M_aet @ M_aet.T, np.eye(3), atol=1e-15)
    M_gen = np.array([[1.3, 0.2, -0.4], [0.1, 0.9, 0.3], [-0.2, 0.5, 1.7]])
    for s in range(th.shape[0]):
        C = _cov_matrix(C6[s])
        Cs = sd[:, :, None] * C * sd[:, None, :]
        Ps = sd[:, :, None] * P * sd[:, None, :]
        assert _wishart_numpy(Cs, Ps, ds["nu"]) == pytest.approx(L[s] + scale_shift, rel=1e-12, abs=0)
        for M in (M_aet.T, M_gen):      # data in the new basis: d' = M d
            Cx = M @ Cs @ M.T
            Px = M @ Ps @ M.T
            assert np.max(np.linalg.cond(Cx)) < 1e4
            shift = -np.sum(ds["nu"]) * math.log(np.linalg.det(M) ** 2)
            assert _wishart_numpy(Cx, Px, ds["nu"]) == pytest.approx(L[s] + scale_shift + shift, rel=1e-12, abs=0)


def test_periodogram_equal_to_model_closed_form(full):
    ds, th, kn = full
    C6, _ = oracle.model_cov_full(ds, th[:1], {k: (v[:1] if isinstance(v, np.ndarray) else v) for k, v in kn.items()})
    c = C6[0]
    P9 = np.zeros((9, c.shape[1]))
    P9[0], P9[1], P9[2], P9[3], P9[5], P9[7] = c[0], c[1], c[2], c[3], c[4], c[5]
    L, st = oracle.loglike_full(dict(ds, P9=P9), th[:1], {k: (v[:1] if isinstance(v, np.ndarray) else v)
                                                          for k, v in kn.items()})
    det = np.linalg.det(_cov_matrix(c))
    assert L[0] == pytest.approx(-np.sum(ds["nu"] * (3.0 + np.log(det))), rel=1e-13)


def test_imaginary_parts_cancel(full):
    ds, th, kn = full
    L1, st1, im1 = oracle.loglike_full(ds, th, kn, return_im=True)
    P9 = ds["P9"].copy()
    P9[[4, 6, 8]] *= -3.7                      # other imaginary parts, same real parts
    L2, st2, im2 = oracle.loglike_full(dict(ds, P9=P9), th, kn, return_im=True)
    np.testing.assert_allclose(L1, L2, rtol=1e-14, atol=0)
    assert np.all(im1 < 1e-13) and np.all(im2 < 1e-13)


def test_extreme_correlations_stay_positive_definite(full):
    ds, th, kn = full
    nsp = oracle.n_splines_full(ds)
    kx = {k: (v[:2].copy() if isinstance(v, np.ndarray) else v) for k, v in kn.items()}
    kx["count"][:, nsp - 3:] = 0
    kx["w"][0, nsp - 3:, :] = 1e3              # |r| -> 1 - 5e-7
    kx["w"][1, nsp - 3:, :] = np.array([[-1e2], [1e2], [-1e2]])
    C6, st = oracle.model_cov_full(ds, th[:2], kx)
    L, st2 = oracle.loglike_full(ds, th[:2], kx)
    assert not st.any() and not st2.any() and np.all(np.isfinite(L))
    for s in range(2):
        C = _cov_matrix(C6[s])
        D = np.sqrt(np.diagonal(C, axis1=1, axis2=2))
        assert np.all(np.linalg.det(C / (D[:, :, None] * D[:, None, :])) > 0)
