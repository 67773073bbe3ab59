"""The multi-rank bookkeeping of bench.py on CPU ranks (gloo, world size 2):
every rank compresses its own field (no collective on the data path), the
job's time is the slowest rank's, and the job's GB/s counts every rank's
values over that time (weak scaling)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_local = 10.0 + 5.0 * rank          # rank 1 is the slow one
        ms = bench.max_over_ranks(ms_local, dist, "cpu")
        out[rank] = (bench.rank_field_seed(rank), ms, bench.job_gbps(world, 1000, ms))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_to_the_slowest_rank():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:  # no fork of a process that may hold threads
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    seeds = {r: v[0] for r, v in res.items()}
    assert seeds[0] != seeds[1]                       # distinct fields per rank
    assert res[0][1] == res[1][1] == 15.0             # max over ranks
    assert res[0][2] == pytest.approx(2 * 1000 * 4 / 15e-3 / 1e9)


def test_single_rank_is_the_identity():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
