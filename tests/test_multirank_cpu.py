"""The multi-rank form of bench.py on CPU (gloo, world size 2): each rank
takes a disjoint set of 128-path prefixes, and the job time is the slowest
rank's (no collective touches the data path)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, first_ids, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        pre = bench.rank_prefixes(first_ids, world, rank, 5)
        t = bench.max_over_ranks(1.0 + rank, "cpu")
        out.put((rank, pre, t))
    finally:
        dist.destroy_process_group()


def test_ranks_take_disjoint_prefixes_and_max_time():
    ids = np.arange(128 * 12, dtype=np.uint64) * 3  # 12 prefixes
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, ids, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, pre0, t0), (r1, pre1, t1) = res
    assert not set(pre0) & set(pre1)
    assert sorted(pre0 + pre1) == [int(ids[128 * i]) for i in range(10)]
    assert t0 == t1 == 2.0


def test_single_rank_is_identity():
    import bench
    ids = np.arange(128 * 3, dtype=np.uint64)
    assert bench.rank_prefixes(ids, 1, 0, 3) == [0, 128, 256]
    assert bench.max_over_ranks(3.5) == 3.5


def test_amplitude_rates():
    import bench
    r = bench.amplitude_rates(3000.0, 1_000_000, 171_798_912)
    assert r["path_amplitudes_per_s"] == 3e9
    assert abs(r["request_seconds"] - 171_798_912 / 3000.0) < 1e-6
    assert abs(r["request_amplitudes_per_s"] * r["request_seconds"] - 1_000_000) < 1e-3
