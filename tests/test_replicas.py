"""Multi-rank bench aggregation (replicas, no data-path collective) with two gloo ranks on CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as tdist
import torch.multiprocessing as mp

from paper_2606_27134_b300.replicas import job_throughput, max_over_ranks


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        step_ms = 2.0 + 3.0 * rank                # ranks finish at different times
        value, t = job_throughput(1000, step_ms, tdist)
        mx = max_over_ranks(-rank, tdist)
        out[rank] = (value, t, mx)
    finally:
        tdist.destroy_process_group()


def test_single_rank_is_identity():
    value, t = job_throughput(1000, 4.0)
    assert t == 4.0 and value == pytest.approx(1000 / 4e-3)
    assert max_over_ranks(3.5) == 3.5


def test_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    assert sorted(out.keys()) == [0, 1]
    for rank in range(world):
        value, t, mx = out[rank]
        assert t == 5.0                            # the slower rank's step time
        assert value == pytest.approx(world * 1000 / 5e-3)
        assert mx == 0.0
