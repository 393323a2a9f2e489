"""Multi-rank (replica) layout on CPU: gloo process groups of world size 2, the oracle standing in
for each rank's GPU evaluation.  Sharding by states and by datasets must reproduce the single
process result exactly after the gather, and timings reduce to the maximum over ranks."""
import os
import socket

import numpy as np
import pytest

from paper_2507_06300_gb300 import replicas, synth
from tests._workloads import oracle_batched


def test_shard_range_tiles_in_rank_order():
    for n in (0, 1, 5, 6, 7, 1024):
        for world in (1, 2, 3, 8):
            blocks = [replicas.shard_range(n, r, world) for r in range(world)]
            assert blocks[0][0] == 0 and blocks[-1][1] == n
            for (a, b), (c, d) in zip(blocks, blocks[1:]):
                assert b == c
            sizes = [b - a for a, b in blocks]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        replicas.shard_range(4, 2, 2)


def test_shard_workload_by_datasets_keeps_each_dataset_whole():
    wl = synth.workload("batched", n_datasets=5, n_min=40, n_max=90, states_per=3, kmax_draw=4)
    parts = [replicas.shard_workload(wl, r, 2) for r in range(2)]
    assert sum(p.n_datasets for p in parts) == 5
    assert np.array_equal(np.concatenate([p.f for p in parts]), wl.f)
    assert np.array_equal(np.concatenate([p.theta for p in parts]), wl.theta)
    for p in parts:
        assert p.bin_offset[0] == 0 and p.state_offset[0] == 0
        assert p.bin_offset[-1] == p.f.size and p.state_offset[-1] == p.theta.shape[0]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, name, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl = (synth.workload("tiny") if name == "tiny" else
              synth.workload("batched", n_datasets=5, n_min=40, n_max=90, states_per=3, kmax_draw=4))
        part = replicas.shard_workload(wl, rank, world)
        _, L, St = oracle_batched(part)
        L_all = replicas.gather_rows(L, dist)
        St_all = replicas.gather_rows(St, dist)
        t = replicas.max_over_ranks([1.0 + rank, 5.0 - rank], dist)
        n = replicas.sum_over_ranks([part.n_states], dist)
        q.put((rank, L_all, St_all, t + n))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name", ["tiny", "batched"])
def test_two_ranks_gather_the_single_process_result(name):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, name, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get() for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    wl = (synth.workload("tiny") if name == "tiny" else
          synth.workload("batched", n_datasets=5, n_min=40, n_max=90, states_per=3, kmax_draw=4))
    _, L, St = oracle_batched(wl)
    for rank, L_all, St_all, t in res:
        np.testing.assert_array_equal(St_all, St)
        np.testing.assert_array_equal(L_all, L)
        assert t == [2.0, 5.0, float(wl.n_states)]
