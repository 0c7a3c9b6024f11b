"""The multi-rank part of bench.py on CPU: replicas on world-size-2 gloo
ranks meet only in the reduction of the timed region (max over ranks) and
of the work (sum over ranks)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert bench.dist_env() == (rank, rank, world)
        # rank r: 10 + 5 r ms for 1e9 (r + 1) point-windows
        v = bench.combine_ranks(10.0 + 5.0 * rank, 1e9 * (rank + 1), torch.device("cpu"))
        out[rank] = v
    finally:
        dist.destroy_process_group()


def test_replica_reduction_two_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    expect = (1e9 + 2e9) / (15.0 * 1e-3) / 1e9   # all work / the slowest rank's time
    assert out[0] == pytest.approx(expect) and out[1] == pytest.approx(expect)


def test_single_rank_is_plain_ratio():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks(20.0, 4e9, torch.device("cpu")) == pytest.approx(200.0)
