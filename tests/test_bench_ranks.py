"""Multi-rank logic of bench.py on CPU: two gloo ranks (one replica each, no
data-path collective), the maximum of the measured times over ranks, distinct
replica seeds, and the reference arm doing its work on rank 0 only."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    r = bench.Ranks("gloo")
    r.barrier()
    out[rank] = (r.max(1.5 + rank), r.seed(7), r.world)
    r.barrier()
    r.close()


def test_two_gloo_ranks_max_and_seeds():
    world, port = 2, _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, start_method="spawn")
    assert out[0][0] == out[1][0] == 2.5          # the slowest rank's time
    assert out[0][1] != out[1][1]                 # one Philox seed per replica
    assert out[0][2] == out[1][2] == 2


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    args = type("A", (), dict(steps=1, warmup=0))()
    bench.run_reference(args)                     # rank 1: returns at once, prints nothing
    assert capsys.readouterr().out == ""
