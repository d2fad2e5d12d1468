"""The multi-GPU path of bench.py on CPU: two gloo ranks, each with its own
replica time; both see the slowest rank's time and the whole-job throughput
(all ranks' particle-steps over it), as the torchrun launch computes it."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.dist_env()
    ms_max, value = bench.aggregate_throughput(100.0 + 50.0 * rank, 1_000_000, w, dist)
    q.put((r, w, local, ms_max, value))
    dist.destroy_process_group()


def test_two_rank_aggregation_over_gloo():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[:3] for o in out] == [(0, 2, 0), (1, 2, 1)]
    for _, _, _, ms_max, value in out:
        assert ms_max == 150.0
        assert value == pytest.approx(2 * 1_000_000 / 0.150)
