"""Host logic of the slab decomposition: the split of the axis, the
neighbour ranks, the exchange schedule between ranks (two and three gloo
processes on the CPU, the same torch.distributed point-to-point calls that
move the halo messages between GPUs over NCCL), and the validation of
lbm_create_slab before any device work."""
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

import paper_2302_04741_gb300 as lbm
from paper_2302_04741_gb300 import build as lbm_build
from paper_2302_04741_gb300 import slabs as SL


def test_split_covers_the_axis():
    for n, k in ((512, 2), (512, 3), (10, 3), (9, 3), (37, 5)):
        r = SL.split(n, k)
        assert r[0][0] == 0 and r[-1][1] == n and len(r) == k
        assert all(a1 == b0 for (_, a1), (b0, _) in zip(r, r[1:]))
        sizes = [b - a for a, b in r]
        assert min(sizes) >= 3 and max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        SL.split(8, 3)


def test_halo_peers():
    assert SL.halo_peers(0, 3, False) == (None, 1)
    assert SL.halo_peers(1, 3, False) == (0, 2)
    assert SL.halo_peers(2, 3, False) == (1, None)
    assert SL.halo_peers(0, 3, True) == (2, 1)
    assert SL.halo_peers(2, 3, True) == (1, 0)
    assert SL.halo_peers(0, 1, True) == (0, 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, periodic, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        below, above = SL.halo_peers(rank, world, periodic)
        n = 5
        # each message carries (sender, side) so the receiver can check its origin
        mk = lambda side: torch.tensor([rank, side] + [rank * 10 + side] * (n - 2), dtype=torch.float64)
        send_b = mk(0) if below is not None else None
        send_a = mk(1) if above is not None else None
        recv_b = torch.full((n,), -1.0, dtype=torch.float64) if below is not None else None
        recv_a = torch.full((n,), -1.0, dtype=torch.float64) if above is not None else None
        SL.exchange_halos(send_b, send_a, recv_b, recv_a, rank, world, periodic)
        out = {"below": None if recv_b is None else recv_b.tolist(),
               "above": None if recv_a is None else recv_a.tolist()}
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,periodic", [(2, False), (2, True), (3, False), (3, True)])
def test_exchange_schedule_gloo(world, periodic):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, periodic, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        below, above = SL.halo_peers(r, world, periodic)
        if below is None:
            assert res[r]["below"] is None
        else:  # the neighbour below sent its upward message (side 1)
            assert res[r]["below"][:2] == [below, 1]
        if above is None:
            assert res[r]["above"] is None
        else:  # the neighbour above sent its downward message (side 0)
            assert res[r]["above"][:2] == [above, 0]


def test_create_slab_validation():
    lbm_build.build()
    o = lbm.options(bc=(0, 2, 0))
    for a, b in ((-1, 5), (0, 2), (5, 5), (10, 30), (24, 26)):
        with pytest.raises(lbm.LbmError) as ei:
            lbm.lbm_create_slab(0, 16, 24, 1, a, b, 0.8, None, o)
        assert ei.value.status == lbm.LBM_EINVAL
    for kw in (dict(graph_steps=2), dict(kernel=lbm.LBM_KERNEL_TMA), dict(storage_probe=1)):
        o = lbm.options(bc=(0, 2, 0), **kw)
        with pytest.raises(lbm.LbmError) as ei:
            lbm.lbm_create_slab(0, 16, 24, 1, 0, 12, 0.8, None, o)
        assert ei.value.status == lbm.LBM_EINVAL
