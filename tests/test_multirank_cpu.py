"""The N > 1 path of bench.py on CPU: world-size-2 gloo ranks, each an independent replica; the
whole-job rate uses the slowest rank's span and the units of every rank."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, local_ms, units, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    value, span = bench.whole_job_rate(local_ms[rank], units, world)
    out[rank] = (value, span)
    dist.barrier()
    dist.destroy_process_group()


def test_whole_job_rate_two_gloo_ranks():
    world, units = 2, 1_000_000
    local_ms = [120.0, 150.0]
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, local_ms, units, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        value, span = res[rank]
        assert span == 150.0
        assert abs(value - world * units / 0.150) < 1e-6 * value


def test_single_rank_rate():
    import bench
    value, span = bench.whole_job_rate(200.0, 5_000, 1)
    assert span == 200.0 and abs(value - 25_000.0) < 1e-9
