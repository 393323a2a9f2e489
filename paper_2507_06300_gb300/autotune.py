"""Tile-shape autotuner for the fused FP32 likelihood.

Times ``lisa_psd_loglike`` (the setup is not affected by the tiling) on the caller's own inputs
for a grid of tilings -- bins staged per work item, state lanes per item, bins between interval
checks -- with CUDA events after a warm-up, and leaves the fastest applied to the dataset.  The
L2 cache is flushed (a 256 MB buffer written, more than GB300's 129 MB L2) before every timed
call, and each call is timed on its own, so tilings are compared in the regime a sampler step
meets: bin tables and spline records read from HBM, not left resident by the previous call.
Shared-memory limits are handled by the library: a tiling whose staging does not fit is
rejected by ``lisa_data_set_tiling`` or by the launch and simply skipped here.
"""
from __future__ import annotations

import itertools

from . import binding as B

DEFAULT_TILES = (256, 320, 384, 448, 512, 768, 1024)
DEFAULT_STATES = (64, 128)
DEFAULT_GROUPS = (2, 4, 8)


FLUSH_BYTES = 256 * 1024 * 1024


def autotune(dataset, theta, count, x, w, kmax, kind=B.AKIMA, precision=B.FP32, tiles=DEFAULT_TILES,
             states=DEFAULT_STATES, groups=DEFAULT_GROUPS, reps=5):
    """Returns (best tiling dict, list of (tiling dict, ms) for every candidate that ran); ms is
    the mean over ``reps`` calls, each timed alone after an L2 flush."""
    import torch

    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    buf, _ = dataset.spline_setup(count, x, w, kmax, kind, precision)
    ws = torch.empty(max(dataset.workspace_bytes(kmax, precision), 1), dtype=torch.uint8, device="cuda")
    out = torch.empty(dataset.n_states, dtype=torch.float64, device="cuda")
    results = []
    for tb, sc, g in itertools.product(tiles, states, groups):
        t = dict(tile_bins=tb, states_per_cta=sc, group=g, ctas_per_sm=0)
        try:
            dataset.set_tiling(**t)
            need = dataset.workspace_bytes(kmax, precision)
            if need > ws.numel():
                ws = torch.empty(need, dtype=torch.uint8, device="cuda")
            for _ in range(2):
                dataset.psd_loglike(theta, buf, kmax, precision, out=out, workspace=ws)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
            for k in range(reps):
                flush.fill_(float(k))
                ev[k][0].record()
                dataset.psd_loglike(theta, buf, kmax, precision, out=out, workspace=ws)
                ev[k][1].record()
            torch.cuda.synchronize()
            results.append((t, sum(a.elapsed_time(b) for a, b in ev) / reps))
        except B.LisaError:
            continue
    if not results:
        raise B.LisaError("autotune: no tiling could be launched")
    best = min(results, key=lambda r: r[1])[0]
    dataset.set_tiling(**best)
    return best, results
