"""bench.py's replica aggregation across ranks (the N-GPU path is replicas only:
no collective on the data path, only the timing max and pose counts), run as
two gloo processes on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(WORLD_SIZE=str(world), RANK=str(rank), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench
    d = bench.Dist()
    try:
        assert d.world == world and d.rank == rank
        d.barrier()
        t_max = d.max(10.0 + rank)            # per-rank step time in ms
        poses = d.sum(16)                     # poses each replica solved
        out[rank] = (t_max, poses, 1e3 * poses / t_max)
    finally:
        d.close()


def test_two_replicas_aggregate_with_gloo():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]
    t_max, poses, value = res[0]
    assert t_max == 11.0 and poses == 32
    assert value == pytest.approx(32 / 0.011)     # whole-job throughput over the slowest rank


def test_single_process_needs_no_process_group(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    import bench
    d = bench.Dist()
    assert d.world == 1 and d.pg is None
    assert d.max(3.0) == 3.0 and d.sum(5) == 5
