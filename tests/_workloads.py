"""Test helpers: oracle-side datasets built from the seeded synthetic workloads."""
import numpy as np

import oracle
from paper_2507_06300_gb300 import synth


def zero_knots(n_states, nsp, kmax=0):
    return {"count": np.zeros((n_states, nsp), np.int32), "x": np.zeros((n_states, nsp, max(kmax, 1))),
            "w": np.zeros((n_states, nsp, kmax + 2)), "kmax": kmax, "kind": 0}


def oracle_dataset(wl, d=0):
    """Dataset d of a workload with its periodogram P = S_model(theta_true) * Gamma(nu)/nu,
    the model PSD taken from the oracle."""
    ds = wl.dataset(d)
    b0, b1 = int(wl.bin_offset[d]), int(wl.bin_offset[d + 1])
    nsp = wl.n_splines
    if wl.true_knots is None:
        kn = zero_knots(1, nsp)
    else:
        tk = wl.true_knots
        kn = {"count": tk.count[d:d + 1], "x": tk.x[d:d + 1], "w": tk.w[d:d + 1], "kmax": tk.kmax,
              "kind": tk.kind}
    S, st = oracle.model_psd(ds, wl.theta_true[d:d + 1], kn)
    assert st[0] == 0
    ds["P"] = S[0] * wl.gamma[:, b0:b1]
    return ds


def gpu_eval(wl, P, precision, kind=None, tiling=None, theta=None, knots=None):
    """Runs spline setup + log-likelihood through the C ABI; returns (logL, status) as numpy."""
    import torch
    from paper_2507_06300_gb300 import binding as B
    ds = B.Dataset.from_workload(wl, P)
    if tiling:
        ds.set_tiling(**tiling)
    kn = wl.knots if knots is None else knots
    th = wl.theta if theta is None else theta
    count, x, w, kmax, kd = B.knots_to_device(kn)
    if kind is not None:
        kd = kind
    theta_d = torch.as_tensor(np.ascontiguousarray(th), device="cuda")
    buf, st = ds.spline_setup(count, x, w, kmax, kd, precision)
    out = ds.psd_loglike(theta_d, buf, kmax, precision)
    torch.cuda.synchronize()
    res = out.cpu().numpy(), st.cpu().numpy()
    ds.close()
    return res


def oracle_batched(wl):
    """Per-dataset oracle periodograms [C, N_total] and log-likelihoods [S_total]."""
    P = np.empty((wl.n_channels, wl.n_bins))
    L = np.empty(wl.n_states)
    St = np.empty(wl.n_states, np.int32)
    for d in range(wl.n_datasets):
        ds = oracle_dataset(wl, d)
        b0, b1 = int(wl.bin_offset[d]), int(wl.bin_offset[d + 1])
        P[:, b0:b1] = ds["P"]
        th, kn = wl.states(d)
        s0, s1 = int(wl.state_offset[d]), int(wl.state_offset[d + 1])
        if s1 > s0:
            L[s0:s1], St[s0:s1] = oracle.loglike(ds, th, kn.as_dict())
    return P, L, St


def fp32_tolerance(L_ref, wl, P):
    """FP32-bulk bound: 1e-6 of the normalised log-likelihood's scale, max(|log L - K|, C sum nu)
    with K = -sum nu sum_c ln P (the part of log L that does not depend on the state)."""
    tol = np.empty_like(L_ref)
    for d in range(wl.n_datasets):
        b0, b1 = int(wl.bin_offset[d]), int(wl.bin_offset[d + 1])
        s0, s1 = int(wl.state_offset[d]), int(wl.state_offset[d + 1])
        K = -np.sum(wl.nu[b0:b1] * np.log(P[:, b0:b1]).sum(axis=0))
        scale = wl.n_channels * wl.nu[b0:b1].sum()
        tol[s0:s1] = 1e-6 * np.maximum(np.abs(L_ref[s0:s1] - K), scale)
    return tol


def colour_wishart(cov6, W9):
    """P = L W L^T per bin, with L the Cholesky factor of the model covariance (cov6 [6, N]:
    C00, C11, C22, C01, C02, C12) and W the unit complex Wishart draws (W9 [9, N]): the averaged
    periodogram of data with covariance C.  Returns P9 [9, N] in the oracle's layout."""
    N = cov6.shape[1]
    C = np.empty((N, 3, 3))
    C[:, 0, 0], C[:, 1, 1], C[:, 2, 2] = cov6[0], cov6[1], cov6[2]
    C[:, 0, 1] = C[:, 1, 0] = cov6[3]
    C[:, 0, 2] = C[:, 2, 0] = cov6[4]
    C[:, 1, 2] = C[:, 2, 1] = cov6[5]
    L = np.linalg.cholesky(C)
    W = np.zeros((N, 3, 3), dtype=np.complex128)
    W[:, 0, 0], W[:, 1, 1], W[:, 2, 2] = W9[0], W9[1], W9[2]
    for k, (a, b) in enumerate(((0, 1), (0, 2), (1, 2))):
        W[:, a, b] = W9[3 + 2 * k] + 1j * W9[4 + 2 * k]
        W[:, b, a] = np.conj(W[:, a, b])
    P = L @ W @ np.transpose(L, (0, 2, 1))
    out = np.empty((9, N))
    out[0], out[1], out[2] = P[:, 0, 0].real, P[:, 1, 1].real, P[:, 2, 2].real
    for k, (a, b) in enumerate(((0, 1), (0, 2), (1, 2))):
        out[3 + 2 * k] = P[:, a, b].real
        out[4 + 2 * k] = P[:, a, b].imag
    return out


def hermitian(P9):
    """[N, 3, 3] complex Hermitian matrices from the oracle's P9 layout."""
    N = P9.shape[1]
    P = np.zeros((N, 3, 3), dtype=np.complex128)
    P[:, 0, 0], P[:, 1, 1], P[:, 2, 2] = P9[0], P9[1], P9[2]
    for k, (a, b) in enumerate(((0, 1), (0, 2), (1, 2))):
        P[:, a, b] = P9[3 + 2 * k] + 1j * P9[4 + 2 * k]
        P[:, b, a] = np.conj(P[:, a, b])
    return P


def oracle_dataset_full(wl):
    """Dense-covariance dataset of a cov_model=1 workload: the averaged periodogram matrix P9
    [9, N] = L W L^T around the oracle's model covariance of the injection (constant
    correlations), W the workload's unit complex Wishart draws."""
    ds = wl.dataset(0)
    tk = wl.true_knots
    C6, st = oracle.model_cov_full(ds, wl.theta_true[:1], tk.as_dict())
    assert st[0] == 0
    ds["P9"] = colour_wishart(C6[0], wl.wishart)
    return ds


def fp32_tolerance_full(L_ref, wl, P9):
    """The FP32-bulk bound for the dense covariance: 1e-6 of max(|log L - K|, 3 sum nu), with
    K = -sum nu sum_c ln P_cc."""
    K = -np.sum(wl.nu * np.log(P9[:3]).sum(axis=0))
    return 1e-6 * np.maximum(np.abs(L_ref - K), 3 * wl.nu.sum())
