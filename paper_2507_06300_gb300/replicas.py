"""Multi-GPU layout: independent replicas, one process per GPU.

The states of a tempered ensemble, and the datasets of a batch, are independent: the
log-likelihood of one needs nothing from another (Sec. III.C sums over the bins of one
dataset for one parameter point).  The path therefore shards with no exchange step: each rank
evaluates a contiguous block of datasets (or, for a single dataset, of states) on its own GPU
through the same C ABI.  The only collectives are host-side bookkeeping -- the maximum over
ranks of a timing (the slowest replica sets the job's time) and, when the caller wants every
log-likelihood in one place, a gather of the per-rank results in rank order.  Nothing here
touches the device.
"""
from __future__ import annotations

import dataclasses

import numpy as np


def shard_range(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous block [lo, hi) of n units for `rank` of `world`; sizes differ by at most one
    and the blocks tile [0, n) in rank order."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError(f"bad shard request n={n} rank={rank} world={world}")
    q, r = divmod(n, world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def shard_workload(wl, rank: int, world: int):
    """The part of a synth.Workload that `rank` evaluates: a block of whole datasets when there
    are several (bins, states and offsets re-based), else a block of the single dataset's
    states.  The periodogram formed from the part equals the corresponding slice of the whole's,
    since each dataset keeps its own injection and noise draws."""
    k = wl.knots
    if wl.n_datasets > 1:
        d0, d1 = shard_range(wl.n_datasets, rank, world)
        b0, b1 = int(wl.bin_offset[d0]), int(wl.bin_offset[d1])
        s0, s1 = int(wl.state_offset[d0]), int(wl.state_offset[d1])
        sl = slice(s0, s1)
        return dataclasses.replace(
            wl, f=wl.f[b0:b1], nu=wl.nu[b0:b1], R=wl.R[:, b0:b1], gamma=wl.gamma[:, b0:b1],
            bin_offset=wl.bin_offset[d0:d1 + 1] - b0, state_offset=wl.state_offset[d0:d1 + 1] - s0,
            x_lo=wl.x_lo[d0:d1], x_hi=wl.x_hi[d0:d1], f_ref=wl.f_ref[d0:d1], theta_true=wl.theta_true[d0:d1],
            theta=wl.theta[sl], knots=dataclasses.replace(k, count=k.count[sl], x=k.x[sl], w=k.w[sl]),
            true_knots=None if wl.true_knots is None else dataclasses.replace(
                wl.true_knots, count=wl.true_knots.count[d0:d1], x=wl.true_knots.x[d0:d1],
                w=wl.true_knots.w[d0:d1]))
    s0, s1 = shard_range(wl.n_states, rank, world)
    sl = slice(s0, s1)
    return dataclasses.replace(wl, state_offset=np.array([0, s1 - s0], np.int64), theta=wl.theta[sl],
                               knots=dataclasses.replace(k, count=k.count[sl], x=k.x[sl], w=k.w[sl]))


def _reduce(values, dist, device, op):
    vals = [float(v) for v in values]
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return vals
    import torch
    t = torch.tensor(vals, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=getattr(dist.ReduceOp, op))
    return t.tolist()


def max_over_ranks(values, dist=None, device="cpu"):
    """Element-wise maximum over ranks of a list of floats (identity without a process group)."""
    return _reduce(values, dist, device, "MAX")


def sum_over_ranks(values, dist=None, device="cpu"):
    """Element-wise sum over ranks of a list of floats (identity without a process group)."""
    return _reduce(values, dist, device, "SUM")


def gather_rows(local, dist=None):
    """Concatenation, in rank order, of every rank's 1-D or 2-D numpy block (on every rank)."""
    local = np.asarray(local)
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return local
    parts = [None] * dist.get_world_size()
    dist.all_gather_object(parts, local)
    return np.concatenate(parts, axis=0)
