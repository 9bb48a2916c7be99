"""The N-GPU form of the benchmark is replicas (pairs are independent; no data-path collective): every rank
matches its own pairs, the step time is the maximum over ranks and the value counts the pixels of all ranks.
Checked here with two gloo ranks on the CPU (rendezvous on 127.0.0.1)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [3.0, 5.0][rank]  # rank 1 is the slower replica
    ms, value = bench.aggregate_ranks(torch, dist, torch.device("cpu"), local_ms, 465750, world)
    dist.barrier()
    out.put((rank, ms, value))
    dist.destroy_process_group()


def test_two_rank_aggregation_takes_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in res:
        assert ms == 5.0
        assert value == pytest.approx(2 * 465750 / 5e-3 / 1e6)


def test_single_process_aggregation():
    import bench

    ms, value = bench.aggregate_ranks(torch, None, torch.device("cpu"), 2.0, 1000000, 1)
    assert ms == 2.0 and value == pytest.approx(500.0)
