"""The replica path of `bench.py --gpus N` on the CPU: two gloo ranks.

Each rank joins its own instance of the workload (weak scaling); the job's
step time is the max over ranks and its work the sum.  The GPU runs of this
pool have one GPU, so the host logic is checked here with world_size 2."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        times = [10.0 + rank, 20.0 - rank, 5.0 * (rank + 1)]
        cells = 1000 * (rank + 1)
        red_t, red_c = bench.reduce_over_ranks(times, cells, torch.device("cpu"))
        out[rank] = (red_t, red_c, bench.replica_seed(2, rank))
    finally:
        dist.barrier()
        dist.destroy_process_group()


def test_two_ranks_max_time_sum_work():
    world, port = 2, _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        got = dict(out)
    assert sorted(got) == [0, 1]
    for rank in (0, 1):
        red_t, red_c, _ = got[rank]
        assert red_t == [11.0, 20.0, 10.0]   # element-wise max over the ranks
        assert red_c == 3000.0                # the ranks' work summed
    assert got[0][2] == 2 and got[1][2] != got[0][2]   # rank 0 joins the workload itself, rank 1 another instance


def test_one_process_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    torch = pytest.importorskip("torch")
    t, c = bench.reduce_over_ranks([1.5, 2.5], 7, torch.device("cpu"))
    assert t == [1.5, 2.5] and c == 7.0
