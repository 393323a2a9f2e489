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
