"""The multi-GPU form of the benchmark runs independent replicas (the step has no exchange
between grids): whole-job throughput = all ranks' cell-updates / the slowest rank's time.
Tested here with two gloo ranks on the CPU, through the same function bench.py uses."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    ms_local = [10.0, 25.0][rank]            # rank 1 is the slow one
    units_local = [1.0e9, 1.0e9][rank]       # equal work per replica (weak scaling)
    value, ms = bench.aggregate_replicas(ms_local, units_local)
    out[rank] = (value, ms)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_benchmark():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for r in (0, 1):
        value, ms = res[r]
        assert ms == 25.0
        assert value == pytest.approx(2.0e9 / 25e-3)


def test_single_process_aggregate():
    import bench
    value, ms = bench.aggregate_replicas(10.0, 5.0e8)
    assert ms == 10.0 and value == pytest.approx(5.0e10)
