"""The N>1 path of bench.py on the CPU: ranks read their identity from the
torchrun environment and the timing is the maximum over ranks (two gloo
ranks, world size 2). The benchmark's replicas share no data: this max and a
barrier are its only collectives."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "RANK": str(rank), "WORLD_SIZE": str(ws), "LOCAL_RANK": str(rank)})
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        got_ws, got_rank, got_local = bench.dist_env()
        t = bench.reduce_max(1.5 + rank, ws, "cpu")
        dist.barrier()
        out[rank] = (got_ws, got_rank, got_local, t)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time():
    ws = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(ws, _free_port(), out), nprocs=ws, join=True,
                       start_method="spawn")
    for r in range(ws):
        assert out[r] == (ws, r, r, 1.5 + ws - 1)


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_max(3.25, 1, "cpu") == 3.25
