"""Window sharding on CPU ranks (gloo, world size 2): the window ranges cover
every window exactly once, and the sum over ranks of each rank's share of
Gamma_full v (its windows' direct sums, normalised by the count of all
windows; Sec. 3, the ANOVA kernel as a mean of per-window Gauss transforms)
equals the oracle's Gamma_full v over all windows.  The shares are the
oracle's direct sums; the reduction is the library's reduce callback
(shard.allreduce_sum) on CPU tensors."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2407_06834_gb300 import shard  # noqa: E402


@pytest.mark.parametrize("L", [1, 3, 9, 13])
def test_window_ranges_cover_every_window_once(L):
    for world in range(1, L + 1):
        ranges = [shard.window_range(L, world, r) for r in range(world)]
        covered = [w for f, c in ranges for w in range(f, f + c)]
        assert covered == list(range(L)), (L, world, ranges)
        counts = [c for _, c in ranges]
        assert min(counts) >= 1 and max(counts) - min(counts) <= 1
        assert counts == sorted(counts, reverse=True)
    with pytest.raises(ValueError):
        shard.window_range(9, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    from oracle import oracle as orc
    from paper_2407_06834_gb300 import shard as sh
    from paper_2407_06834_gb300.inputs import random_vector, raster_windows, synthetic_image
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        img = synthetic_image(14, 12, 7)[1]
        win = raster_windows(2)                         # 5x5 patches: L = 9
        coords = orc.image_coords(img, 2, win)
        L = coords.shape[0]
        v = random_vector(img.size, 8)
        first, count = sh.window_range(L, world, rank)
        # this rank's share: mean over its windows times count / L
        share = orc.gamma_full_matvec(coords[first:first + count], 0.2, v) * (count / L)
        buf = torch.as_tensor(share.copy())
        sh.allreduce_sum(buf)
        out[rank] = (buf.numpy().copy(), (first, count))
        # the sharded solve's timing: one job's work over the slowest rank
        out["t%d" % rank] = bench.combine_ranks(10.0 + 5.0 * rank, 2e9, torch.device("cpu"),
                                                sum_work=False)
    finally:
        dist.destroy_process_group()


def test_shares_sum_to_the_full_operator_two_ranks():
    from oracle import oracle as orc
    from paper_2407_06834_gb300.inputs import random_vector, raster_windows, synthetic_image
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    img = synthetic_image(14, 12, 7)[1]
    coords = orc.image_coords(img, 2, raster_windows(2))
    full = orc.gamma_full_matvec(coords, 0.2, random_vector(img.size, 8))
    (y0, r0), (y1, r1) = out[0], out[1]
    assert r0 == (0, 5) and r1 == (5, 4)
    np.testing.assert_array_equal(y0, y1)              # every rank holds the same sum
    assert np.max(np.abs(y0 - full)) <= 1e-13 * np.max(np.abs(full))
    expect = 2e9 / (15.0 * 1e-3) / 1e9                 # work counted once, slowest rank
    assert out["t0"] == pytest.approx(expect) and out["t1"] == pytest.approx(expect)
