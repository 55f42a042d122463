"""Multi-rank sharding of the grid run, on CPU with gloo (world size 2 and 3).

Each rank owns `ny` rows of a (world*ny)-row grid plus one halo row on each side
that has a neighbour; no data-path collective is needed.  The ranks check, with
the same all-gathers the bench's timing reductions use, that the owned rows tile
the global grid exactly once, that each slab's cell centres are those of the
global grid, and that the halo rows make every owned cell's LD stencil complete."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
import oracle as O


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, ny, npy, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        y0, y1, p0, p1 = bench.grid_box(1.0 / 6.0)
        sy0, sy1, rows, hlo = bench.slab_bounds(y0, y1, ny, rank, world)
        first, _, _, hhi = bench.shard_rows(ny, rank, world)
        ics, st = O.grid_ics(1.0 / 6.0, sy0, sy1, rows, p0, p1, npy)
        gics, gst = O.grid_ics(1.0 / 6.0, y0, y1, ny * world, p0, p1, npy)
        g = gics.reshape(4, ny * world, npy)[:, first:first + rows]
        mine = ics.reshape(4, rows, npy)
        same_status = np.array_equal(gst.reshape(ny * world, npy)[first:first + rows],
                                     st.reshape(rows, npy))
        fin = np.isfinite(g)
        ok_centres = (same_status and np.array_equal(fin, np.isfinite(mine))
                      and np.abs(g[fin] - mine[fin]).max() < 1e-13)
        owned = torch.zeros(ny * world, dtype=torch.int64)
        owned[first + hlo:first + hlo + ny] = 1
        dist.all_reduce(owned)
        # LD stencil completeness: every owned interior row has both neighbours in the slab
        own_lo, own_hi = hlo, hlo + ny
        complete = all((r - 1 >= 0 or first + r == 0) and (r + 1 < rows or first + r == ny * world - 1)
                       for r in range(own_lo, own_hi))
        cnt = torch.tensor([ny * npy], dtype=torch.int64)
        dist.all_reduce(cnt)
        t = torch.tensor([float(rank + 1)], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        q.put((rank, bool(ok_centres), owned.tolist(), complete, int(cnt), float(t), hhi))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_shards_tile_grid_without_exchange(world):
    ny, npy = 16, 8
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, ny, npy, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ok_centres, owned, complete, cnt, tmax, hhi in res:
        assert ok_centres and complete
        assert owned == [1] * (ny * world)
        assert cnt == world * ny * npy
        assert tmax == float(world)
        assert hhi == (1 if rank < world - 1 else 0)
