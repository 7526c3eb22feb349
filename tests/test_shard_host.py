"""Pixel sharding's host logic without a GPU: the row partition, and the all-gather that
assembles one field from each rank's slab (gloo, world sizes 2 and 3, uneven slabs and an
empty one).  Each rank's slab comes from a stand-in slab function that writes a known
complex value per detector pixel, so the assembled field shows every row in its place."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2404_12454_gb300 import shard  # noqa: E402


def test_partition_covers_every_row_once_in_order():
    for ny in (0, 1, 7, 512, 1000, 1024):
        for world in (1, 2, 3, 5, 8):
            s = shard.all_slabs(ny, world)
            assert s[0][0] == 0 and s[-1][1] == ny
            assert all(a <= b for a, b in s)
            assert all(s[k][1] == s[k + 1][0] for k in range(world - 1))
            sizes = [b - a for a, b in s]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.slab_bounds(10, 2, 2)
    with pytest.raises(ValueError):
        shard.slab_bounds(10, 0, 0)


class _Det:
    def __init__(self, nx, ny):
        self.nx, self.ny = nx, ny


def _pixel_value(i, j):
    return complex(1000.0 * j + i, -0.5 * i + 0.25 * j)


def _rank_main(rank, world, port, ny, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from paper_2404_12454_gb300 import shard as S
    dist.init_process_group("gloo", rank=rank, world_size=world)
    calls = []

    def slab_fn(b, lam, det, r0, r1, prec, stream):
        calls.append((r0, r1))
        out = torch.empty((r1 - r0, det.nx), dtype=torch.complex64)
        for j in range(r0, r1):
            for i in range(det.nx):
                out[j - r0, i] = _pixel_value(i, j)
        return out

    E = S.field_sharded(None, 1e-6, _Det(5, ny), 1, slab_fn=slab_fn)
    q.put((rank, calls, E.numpy().tolist()))
    dist.destroy_process_group()


@pytest.mark.parametrize("world,ny", [(2, 9), (3, 7), (3, 2)])
def test_sharded_field_is_gathered_in_row_order(world, ny):
    import multiprocessing as mp
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, ny, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want = [[_pixel_value(i, j) for i in range(5)] for j in range(ny)]
    for rank, calls, E in res:
        # each rank evaluated its own slab once, and holds the whole field
        assert calls == [shard.slab_bounds(ny, world, rank)]
        assert E == want
