"""Multi-GPU is replicas only: independent pairs per rank, no data-path
collective, a barrier and a max over ranks around the timed region.

The host logic of bench.py's replica timing runs here as two gloo ranks on
the CPU, with a fake step whose duration differs per rank."""
import os
import socket
import time

import pytest
import torch.distributed as dist
import torch.multiprocessing as tmp

import bench


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    done = []

    def step():
        time.sleep(0.01 * (rank + 1))  # rank 1 is the slow replica
        done.append(1)

    def start_timer():
        t0 = time.perf_counter()
        return lambda: 1000.0 * (time.perf_counter() - t0)

    def reduce_max(x):
        t = torch.tensor([x], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    ms = bench.timed_replicas(step, 5, 2, dist.barrier, start_timer, reduce_max)
    rate = bench.aggregate_rate(world, 64, 5, ms)
    out[rank] = (ms, rate, len(done), tuple(bench.replica_seeds(rank, 8)))
    dist.destroy_process_group()


def test_two_gloo_replicas_take_the_slowest_rank_and_sum_the_pairs():
    world = 2
    mgr = tmp.get_context("spawn").Manager()
    out = mgr.dict()
    tmp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    (ms0, rate0, n0, s0), (ms1, rate1, n1, s1) = out[0], out[1]
    # every rank ran warm-up + timed steps and reports the same (max) time
    assert n0 == n1 == 7
    assert ms0 == ms1
    # the slow rank's five 20 ms steps bound the region from below
    assert ms0 >= 5 * 20.0 * 0.95
    # value = pairs of all ranks / slowest time
    assert rate0 == pytest.approx(2 * 64 * 5 / (ms0 / 1000.0))
    assert rate0 == rate1
    # replicas work on distinct synthetic pairs
    assert not set(s0) & set(s1)
