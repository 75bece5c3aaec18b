"""Host logic of the row-partitioned domain (swe_multi), on the CPU: the
partition of rows into strips, and the per-stage exchange of three halo rows
and the maximum of the wave speeds across strips, run as two gloo ranks that
each hold one strip -- the layout the GPU path uses within one device."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def swe():
    import __graft_entry__
    b = __graft_entry__._build_module()
    if not b.up_to_date():
        b.build()
    import paper_2301_12010_gb300 as m
    return m


@pytest.mark.parametrize("ny,nparts", [(4096, 2), (4096, 3), (1000, 7), (100, 3), (40, 2), (12, 4), (3, 1)])
def test_strips_cover_the_rows_in_order(swe, ny, nparts):
    b = swe.strip_bounds(ny, nparts)
    assert len(b) == nparts and b[0][0] == 0 and b[-1][0] + b[-1][1] == ny
    for (r0, n), (r1, _) in zip(b, b[1:]):
        assert r0 + n == r1
    assert all(n >= 3 for _, n in b)
    if ny >= 64 * nparts:
        assert all(r0 % 32 == 0 for r0, _ in b)
        assert max(n for _, n in b) - min(n for _, n in b) <= 32


@pytest.mark.parametrize("ny,nparts", [(8, 3), (5, 2), (2, 1), (100, 0)])
def test_too_many_strips_are_rejected(swe, ny, nparts):
    import ctypes
    r0, n = ctypes.c_int32(), ctypes.c_int32()
    assert swe.lib.swe_strip_bounds(ny, nparts, 0, ctypes.byref(r0), ctypes.byref(n)) == swe.EINVAL


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, ny, nx, q):
    import torch.distributed as dist
    import paper_2301_12010_gb300 as swe
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rng = np.random.default_rng(7)
        full = rng.normal(size=(ny, nx))       # every rank can rebuild the global field
        speeds = rng.uniform(0.5, 9.0, size=(ny, nx))
        r0, n = swe.strip_bounds(ny, world)[rank]
        H = 3
        # the strip with its halo rows; halo rows start as NaN and must be filled
        local = np.full((n + 2 * H, nx), np.nan)
        local[H:H + n] = full[r0:r0 + n]
        t = torch.from_numpy(local)
        reqs = []
        if rank > 0:      # my bottom rows to the lower neighbour, its top rows into my low halo
            reqs.append(dist.isend(t[H:2 * H].clone(), rank - 1))
            lo = torch.empty((H, nx), dtype=torch.float64)
            reqs.append(dist.irecv(lo, rank - 1))
        if rank + 1 < world:
            reqs.append(dist.isend(t[n:n + H].clone(), rank + 1))
            hi = torch.empty((H, nx), dtype=torch.float64)
            reqs.append(dist.irecv(hi, rank + 1))
        for r in reqs:
            r.wait()
        if rank > 0:
            t[:H] = lo
        if rank + 1 < world:
            t[n + H:] = hi
        # the halo rows are the neighbours' rows of the global field, bit for bit
        ok = True
        if rank > 0:
            ok &= np.array_equal(t[:H].numpy(), full[r0 - H:r0])
        if rank + 1 < world:
            ok &= np.array_equal(t[n + H:].numpy(), full[r0 + n:r0 + n + H])
        # the stage's wave speed: a maximum over all strips
        a = torch.tensor([speeds[r0:r0 + n].max()], dtype=torch.float64)
        dist.all_reduce(a, op=dist.ReduceOp.MAX)
        ok &= float(a.item()) == float(speeds.max())
        q.put((rank, bool(ok)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ny", [96, 131])
def test_two_gloo_ranks_exchange_halo_rows_and_reduce_the_wave_speed(swe, ny):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, ny, 17, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    assert res == {0: True, 1: True}
