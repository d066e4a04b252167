"""The N > 1 host path of bench.py on CPU: world_size 2 over gloo.

Each rank runs an independent replica; the job time is the slowest rank's
time (max over ranks) and the whole-job rate counts every rank's units.
"""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as tdist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ws, r, local = bench._dist()
    assert (ws, r, local) == (world, rank, rank)
    bench._barrier(ws)
    ms_local = [1.5, 4.0][rank]
    ms, rate = bench.aggregate(ws, ms_local, 1000)
    out[rank] = (ms, rate)
    tdist.destroy_process_group()


def test_two_ranks_gloo_max_time_and_total_rate():
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True,
                       start_method="spawn")
    for rank in range(2):
        ms, rate = out[rank]
        assert ms == pytest.approx(4.0)
        assert rate == pytest.approx(2 * 1000 / 4.0e-3)
