"""The multi-GPU path of the benchmark is independent replicas (a solve does
not shard): its only cross-rank steps are the timing barrier and the maximum
of the elapsed times.  Checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        dist.barrier()
        t = bench.max_over_ranks([1.0 + rank, 10.0 * (ws - rank)], ws, "cpu")
        out[rank] = t
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_two_gloo_ranks():
    ws = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(ws, port, out), nprocs=ws, start_method="spawn", join=True)
        got = dict(out)
    assert got[0] == got[1] == [2.0, 20.0]          # every rank sees the slowest rank's times


def test_single_rank_and_throughput():
    assert bench.max_over_ranks([0.5, 0.7], 1, "cpu") == [0.5, 0.7]
    # two replicas of 120 projections, slowest rank 0.3 s: 800 projections/s for the job
    assert bench.replica_throughput(2, 120, 0.3) == pytest.approx(800.0)
    assert bench.replica_throughput(1, 120, 0.3) == pytest.approx(400.0)
