"""Plain FP64 CPU oracle for the spline-perturbed Whittle/Wishart log-likelihood.

TEST INFRASTRUCTURE ONLY: this package checks the CUDA library and is used by the test suite,
by ``__graft_entry__.smoke()`` and by the CPU-baseline leg of ``bench.py``.  Nothing in the
product package imports it, and it imports nothing from the product package.

The arithmetic lives in ``lisa_oracle.cpp`` (a single-threaded C++17 translation of the paper's
definitions, each function citing its section / equation); this module only compiles it with
g++ and marshals numpy arrays through ctypes.

Parity status: every oracle function is pinned in ``tests/test_oracle_*.py`` against closed
forms, special values, SciPy / numpy library routines, brute force or the paper's worked example.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lisa_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "liblisa_oracle.so")
_lock = threading.Lock()
_lib = None

N_THETA = 5


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liblisa_oracle.so`` (plain -O2, no fast-math)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-std=c++17", "-O2", "-fno-fast-math", "-ffp-contract=off", "-shared", "-fPIC",
           "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            D = ctypes.POINTER(ctypes.c_double)
            I = ctypes.POINTER(ctypes.c_int)
            i64, c_int, c_double = ctypes.c_int64, ctypes.c_int, ctypes.c_double
            lib.lo_noise_templates.argtypes = [c_int, i64, D, c_double, c_double, D]
            lib.lo_noise_templates.restype = None
            lib.lo_link_psds.argtypes = [i64, D, c_double, c_double, D]
            lib.lo_link_psds.restype = None
            lib.lo_sgwb_template.argtypes = [c_int, i64, D, D, c_double, c_double, c_double,
                                             c_double, D]
            lib.lo_sgwb_template.restype = None
            lib.lo_spline_coeffs.argtypes = [c_int, c_int, c_int, D, D, c_double, c_double, D, D, D]
            lib.lo_spline_coeffs.restype = c_int
            lib.lo_spline_eval.argtypes = [c_int, c_int, c_int, D, D, c_double, c_double, i64, D, D]
            lib.lo_spline_eval.restype = c_int
            common = [c_int, c_int, c_int, i64, D]
            lib.lo_model_psd.argtypes = common + [D, c_double, c_double, c_double, c_int, c_int,
                                                  c_int, D, I, D, D, D, I]
            lib.lo_model_psd.restype = None
            lib.lo_loglike.argtypes = common + [D, D, D, c_double, c_double, c_double, c_int, c_int,
                                                c_int, D, I, D, D, D, I]
            lib.lo_loglike.restype = None
            lib.lo_loglike_grad.argtypes = common + [D, D, D, c_double, c_double, c_double, c_int,
                                                     c_int, c_int, D, I, D, D, D, D, I]
            lib.lo_loglike_grad.restype = None
            lib.lo_loglike_grad_scaled.argtypes = common + [D, D, D, c_double, c_double, c_double, c_int,
                                                            c_int, c_int, D, I, D, D, D, D, D, I]
            lib.lo_loglike_grad_scaled.restype = None
            full = [c_int, c_int, i64, D]
            lib.lo_model_cov_full.argtypes = full + [D, c_double, c_double, c_double, c_int, c_int, c_int, D, I, D, D,
                                                     D, I]
            lib.lo_model_cov_full.restype = None
            lib.lo_loglike_full.argtypes = full + [D, D, D, c_double, c_double, c_double, c_int, c_int, c_int, D, I,
                                                   D, D, D, D, I]
            lib.lo_loglike_full.restype = None
            _lib = lib
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def noise_templates(f, a_oms, a_tm, tdi_form=0):
    """Eq. (noise_tdi): A, E, T noise PSDs, shape [3, N]."""
    f, pf = _d(f)
    out = np.empty((3, f.size))
    _, po = _d(out)
    _load().lo_noise_templates(int(tdi_form), f.size, pf, float(a_oms), float(a_tm), po)
    return out


def link_psds(f, a_oms, a_tm):
    """Sec. II.B single-link PSDs, shape [2, N]: S_OMS, S_TM."""
    f, pf = _d(f)
    out = np.empty((2, f.size))
    _, po = _d(out)
    _load().lo_link_psds(f.size, pf, float(a_oms), float(a_tm), po)
    return out


def sgwb_template(f, R, log10A, n1, n2=None, f_ref=1e-3, sgwb_model=1):
    """Eq. (pl) and Eq. (Sh) for one response row R(f), shape [N]."""
    f, pf = _d(f)
    R, pR = _d(R)
    out = np.empty(f.size)
    _, po = _d(out)
    n2 = n1 if n2 is None else n2
    _load().lo_sgwb_template(int(sgwb_model), f.size, pf, pR, float(log10A), float(n1), float(n2),
                             float(f_ref), po)
    return out


def spline_coeffs(kind, x_int, w, x_lo, x_hi):
    """One spline: returns (status, xs[k+2], ys[k+2], coef[k+1, 4]).

    ``x_int`` holds the k in-between positions (any order); ``w`` the k+2 amplitudes in the
    slot layout (w_0, knots..., w_n)."""
    x_int = np.asarray(x_int, dtype=np.float64).ravel()
    k = x_int.size
    kmax = max(k, 0)
    kx = np.zeros(max(kmax, 1))
    kx[:k] = x_int
    w = np.asarray(w, dtype=np.float64).ravel()
    kw = np.zeros(kmax + 2)
    kw[0] = w[0]
    kw[1:1 + k] = w[1:1 + k]
    kw[kmax + 1] = w[k + 1]
    _, pkx = _d(kx)
    _, pkw = _d(kw)
    xs, ys, coef = np.zeros(k + 2), np.zeros(k + 2), np.zeros((k + 1, 4))
    _, px = _d(xs)
    _, py = _d(ys)
    _, pc = _d(coef)
    st = _load().lo_spline_coeffs(int(kind), k, kmax, pkx, pkw, float(x_lo), float(x_hi), px, py, pc)
    return st, xs, ys, coef


def spline_eval(kind, x_int, w, x_lo, x_hi, x):
    """Evaluates one spline at the abscissae ``x``; returns (status, values)."""
    x_int = np.asarray(x_int, dtype=np.float64).ravel()
    k = x_int.size
    kx = np.zeros(max(k, 1))
    kx[:k] = x_int
    w = np.asarray(w, dtype=np.float64).ravel()
    kw = np.zeros(k + 2)
    kw[:] = w[:k + 2]
    x, pxx = _d(np.atleast_1d(x))
    out = np.empty(x.size)
    _, po = _d(out)
    _, pkx = _d(kx)
    _, pkw = _d(kw)
    st = _load().lo_spline_eval(int(kind), k, k, pkx, pkw, float(x_lo), float(x_hi), x.size, pxx, po)
    return st, out


def _problem_args(ds):
    C = int(ds["n_channels"])
    f, pf = _d(ds["f"])
    N = f.size
    nu = np.ascontiguousarray(np.broadcast_to(np.asarray(ds.get("nu", 1.0), dtype=np.float64), (N,)))
    nu, pnu = _d(nu)
    P = ds.get("P")
    P = np.ones((C, N)) if P is None else P
    P, pP = _d(np.asarray(P).reshape(C, N))
    R = ds.get("R")
    R = np.zeros((C, N)) if R is None else R
    R, pR = _d(np.asarray(R).reshape(C, N))
    keep = (f, nu, P, R)
    return keep, (C, int(ds.get("sgwb_model", 1)), int(ds.get("tdi_form", 0)), N, pf, pnu, pP, pR,
                  float(ds["x_lo"]), float(ds["x_hi"]), float(ds.get("f_ref", 1e-3)))


def _state_args(theta, knots):
    theta, pt = _d(np.asarray(theta).reshape(-1, N_THETA))
    S = theta.shape[0]
    kmax = int(knots["kmax"])
    count, pc = _i(np.asarray(knots["count"]).reshape(S, -1))
    nsp = count.shape[1]
    kx, pkx = _d(np.asarray(knots["x"]).reshape(S, nsp, max(kmax, 0)) if kmax > 0
                 else np.zeros((S, nsp, 1)))
    kw, pkw = _d(np.asarray(knots["w"]).reshape(S, nsp, kmax + 2))
    keep = (theta, count, kx, kw)
    return keep, S, nsp, kmax, int(knots.get("kind", 0)), (pt, pc, pkx, pkw)


def n_splines(ds):
    return int(ds["n_channels"]) + (1 if int(ds.get("sgwb_model", 1)) != 0 else 0)


def model_psd(ds, theta, knots):
    """Model PSD S_c(f_i) for every state: returns (S [S, C, N], status [S])."""
    keep1, pa = _problem_args(ds)
    keep2, S, nsp, kmax, kind, sa = _state_args(theta, knots)
    C, sg, tf, N, pf, pnu, pP, pR, xlo, xhi, fref = pa
    out = np.empty((S, C, N))
    st = np.zeros(S, dtype=np.int32)
    _, po = _d(out)
    _, pst = _i(st)
    _load().lo_model_psd(C, sg, tf, N, pf, pR, xlo, xhi, fref, kind, kmax, S, *sa, po, pst)
    return out, st


def loglike(ds, theta, knots):
    """Sec. III.C log-likelihood for every state: returns (logL [S], status [S])."""
    keep1, pa = _problem_args(ds)
    keep2, S, nsp, kmax, kind, sa = _state_args(theta, knots)
    out = np.empty(S)
    st = np.zeros(S, dtype=np.int32)
    _, po = _d(out)
    _, pst = _i(st)
    _load().lo_loglike(*pa, kind, kmax, S, *sa, po, pst)
    return out, st


def grad_size(nsp, kmax):
    return N_THETA + nsp * (2 * kmax + 2)


def loglike_grad(ds, theta, knots):
    """log-likelihood and analytic gradient: returns (logL [S], grad [S, G], status [S])."""
    keep1, pa = _problem_args(ds)
    keep2, S, nsp, kmax, kind, sa = _state_args(theta, knots)
    out = np.empty(S)
    g = np.zeros((S, grad_size(nsp, kmax)))
    st = np.zeros(S, dtype=np.int32)
    _, po = _d(out)
    _, pg = _d(g)
    _, pst = _i(st)
    _load().lo_loglike_grad(*pa, kind, kmax, S, *sa, po, pg, pst)
    return out, g, st


def loglike_grad_scale(ds, theta, knots):
    """As loglike_grad, plus per gradient component the sum over bins of the absolute values of
    its per-bin contributions: returns (logL, grad, scale, status)."""
    keep1, pa = _problem_args(ds)
    keep2, S, nsp, kmax, kind, sa = _state_args(theta, knots)
    out = np.empty(S)
    g = np.zeros((S, grad_size(nsp, kmax)))
    sc = np.zeros_like(g)
    st = np.zeros(S, dtype=np.int32)
    _, po = _d(out)
    _, pg = _d(g)
    _, ps = _d(sc)
    _, pst = _i(st)
    _load().lo_loglike_grad_scaled(*pa, kind, kmax, S, *sa, po, pg, ps, pst)
    return out, g, sc, st


# ---- full covariance (reading R16: the dense 3x3 covariance of Sec. III.A) -------------------------

def n_splines_full(ds):
    """3 noise splines, the SGWB spline if present, then z_AE, z_AT, z_ET."""
    return 3 + (1 if int(ds.get("sgwb_model", 1)) != 0 else 0) + 3


def _full_args(ds):
    f, pf = _d(ds["f"])
    N = f.size
    nu = np.ascontiguousarray(np.broadcast_to(np.asarray(ds.get("nu", 1.0), dtype=np.float64), (N,)))
    nu, pnu = _d(nu)
    P9 = ds.get("P9")
    P9 = np.zeros((9, N)) if P9 is None else P9
    P9, pP = _d(np.asarray(P9).reshape(9, N))
    R = ds.get("R")
    R = np.zeros((3, N)) if R is None else R
    R, pR = _d(np.asarray(R).reshape(3, N))
    keep = (f, nu, P9, R)
    return keep, N, pf, pnu, pP, pR


def model_cov_full(ds, theta, knots):
    """Full-covariance model C for every state: returns (cov [S, 6, N] = C00, C11, C22, C01, C02,
    C12 in physical units, status [S])."""
    keep1, N, pf, pnu, pP, pR = _full_args(ds)
    keep2, S, nsp, kmax, kind, sa = _state_args(theta, knots)
    assert nsp == n_splines_full(ds)
    out = np.empty((S, 6, N))
    st = np.zeros(S, dtype=np.int32)
    _, po = _d(out)
    _, pst = _i(st)
    _load().lo_model_cov_full(int(ds.get("sgwb_model", 1)), int(ds.get("tdi_form", 0)), N, pf, pR,
                              float(ds["x_lo"]), float(ds["x_hi"]), float(ds.get("f_ref", 1e-3)), kind, kmax, S,
                              *sa, po, pst)
    return out, st


def loglike_full(ds, theta, knots, return_im=False):
    """Sec. III.C log-likelihood with the dense covariance, every state: returns (logL [S], status
    [S]) (and, with return_im, the largest |Im tr(C^-1 P)| / |Re tr| over bins).  ds["P9"] [9, N]:
    P_AA, P_EE, P_TT, Re/Im P_AE, Re/Im P_AT, Re/Im P_ET."""
    keep1, N, pf, pnu, pP, pR = _full_args(ds)
    keep2, S, nsp, kmax, kind, sa = _state_args(theta, knots)
    assert nsp == n_splines_full(ds)
    out = np.empty(S)
    im = np.zeros(S)
    st = np.zeros(S, dtype=np.int32)
    _, po = _d(out)
    _, pim = _d(im)
    _, pst = _i(st)
    _load().lo_loglike_full(int(ds.get("sgwb_model", 1)), int(ds.get("tdi_form", 0)), N, pf, pnu, pP, pR,
                            float(ds["x_lo"]), float(ds["x_hi"]), float(ds.get("f_ref", 1e-3)), kind, kmax, S,
                            *sa, po, pim, pst)
    return (out, st, im) if return_im else (out, st)
