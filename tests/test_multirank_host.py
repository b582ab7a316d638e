"""The multi-rank host logic of bench.py on CPU (gloo, world size 2): the
whole-job throughput of a weak-scaling run takes the slowest rank's time and
counts every rank's units; the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    local_ms = [120.0, 200.0][rank]              # rank 1 is the slow one
    value, ms = bench.job_throughput(local_ms, 1000, ws, "cpu")
    # the reference arm does its work on rank 0 only; the others return 0 at once
    class A:
        grid, steps, warmup = 4, 1, 0
    rc = bench.run_reference(A()) if rank == 1 else None
    out[rank] = (value, ms, rc, bench.dist_env())
    dist.barrier()
    dist.destroy_process_group()


def test_job_throughput_and_reference_rank_gating_gloo():
    ws, port = 2, _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank_main, args=(ws, port, out), nprocs=ws, join=True)
    for r in range(ws):
        value, ms, _, env = out[r]
        assert ms == pytest.approx(200.0)                  # max over ranks
        assert value == pytest.approx(2 * 1000 / 0.2)      # units of all ranks / slowest time
        assert env == (ws, r, r)
    assert out[1][2] == 0                                  # reference arm: non-zero rank does no work


def test_job_throughput_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    value, ms = bench.job_throughput(250.0, 500, 1, "cpu")
    assert ms == 250.0 and value == pytest.approx(2000.0)
