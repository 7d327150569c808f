"""One grid split into slabs along its last axis (y on D2Q37, z on D3Q39).

Eq. lbm is local (Sec. 2): a site pulls f*_i(x - e_i) with |e_ia| <= 3, so
each slab steps on its own once the three layers beyond each cut hold its
neighbours' post-collision populations.  Every step is: the fused step on
every slab, then one halo exchange per cut (lbm_slab_exchange on one device,
or lbm_slab_halo_pack -> transport -> lbm_slab_halo_unpack between devices
or processes).  The slabs reproduce the undivided grid bit for bit.

``SlabGrid`` holds all slabs of a grid on the current device (one stream);
``exchange_halos`` is the per-step message schedule between ranks that each
hold one slab (torch.distributed point-to-point: NCCL between GPUs, gloo
between CPU processes), and ``DistributedSlab`` steps one rank's slab with
it.  Nothing here computes any part of the method: the binding only moves
arguments and messages.
"""
import math

import numpy as np

import paper_2302_04741_gb300 as lbm
from paper_2302_04741_gb300 import workloads as W

GHOST = 3  # layers a step reaches along each axis (max |e_ia| of both lattices)


def split(n_axis, k):
    """k contiguous ranges [a, b) covering [0, n_axis), sizes differing by at
    most one, each at least GHOST layers."""
    if k < 1 or n_axis < GHOST * k:
        raise ValueError(f"cannot cut {n_axis} layers into {k} slabs of >= {GHOST}")
    base, extra = divmod(n_axis, k)
    out, a = [], 0
    for r in range(k):
        b = a + base + (1 if r < extra else 0)
        out.append((a, b))
        a = b
    return out


def layer_sites(w):
    nx, ny, nz = w["shape"]
    return nx if W.dims(w["lattice"]) == 2 else nx * ny


def axis_length(w):
    nx, ny, nz = w["shape"]
    return ny if W.dims(w["lattice"]) == 2 else nz


def own_part(w, a, b):
    """The fields of layers [a, b) of workload w (rho, u, T, and a FIELD
    force), in the slab's layout."""
    S = layer_sites(w)
    rho = np.ascontiguousarray(w["rho"][a * S:b * S])
    u = np.ascontiguousarray(np.asarray(w["u"])[:, a * S:b * S])
    T = np.ascontiguousarray(w["T"][a * S:b * S])
    g = w.get("g")
    if g is not None and g["kind"] == W.G_FIELD:
        g = dict(g, field=np.ascontiguousarray(np.asarray(g["field"])[:, a * S:b * S]))
    return rho, u, T, g


def periodic_axis(w):
    return w.get("bc", (0, 0, 0))[W.dims(w["lattice"]) - 1] == W.PERIODIC


class SlabGrid:
    """All slabs of workload ``w`` on the current device, one stream.

    ``cuts``: the number of slabs (split evenly) or explicit [(a, b), ...]."""

    def __init__(self, w, cuts, stream=None, block_x=0):
        self.w = w
        self.lat = w["lattice"]
        self.D = W.dims(self.lat)
        n = axis_length(w)
        self.ranges = split(n, cuts) if isinstance(cuts, int) else list(cuts)
        self.periodic = periodic_axis(w)
        self.opt = lbm.options(w.get("precision", W.FP64), w.get("force_order", 2), w.get("bc", (0, 0, 0)),
                               w.get("T_lo", (1.0,) * 3), w.get("T_hi", (1.0,) * 3), stream, block_x, 0,
                               lbm.LBM_KERNEL_AUTO, 0, w.get("mu", 0.0), w.get("include_sigma", False))
        self.ctx = []
        for a, b in self.ranges:
            g = own_part(w, a, b)[3]
            self.ctx.append(lbm.lbm_create_slab(self.lat, *w["shape"], a, b, w["tau"], g, self.opt))
        # cuts: (lower, upper) slab pairs, with the wrap-around cut of a periodic axis
        k = len(self.ctx)
        self.cuts = [(r, r + 1) for r in range(k - 1)] + ([(k - 1, 0)] if self.periodic else [])

    def init(self):
        for (a, b), c in zip(self.ranges, self.ctx):
            rho, u, T, _ = own_part(self.w, a, b)
            lbm.lbm_init(c, rho, u, T)
        if self.w.get("precision", W.FP64) == W.FP16_SCALED:
            # one scale for all slabs: the undivided grid's, the smallest
            scale = min(lbm.lbm_fp16_scale(c) for c in self.ctx)
            for c in self.ctx:
                lbm.lbm_set_fp16_scale(c, scale)
        return self

    def exchange(self):
        for lo, hi in self.cuts:
            lbm.lbm_slab_exchange(self.ctx[lo], self.ctx[hi])

    def step(self, n=1):
        for _ in range(int(n)):
            for c in self.ctx:
                lbm.lbm_step(c, 1)
            self.exchange()

    def moments(self):
        """rho, u, T, q of the whole grid (the slabs' own layers, in order)."""
        parts = []
        S = layer_sites(self.w)
        for (a, b), c in zip(self.ranges, self.ctx):
            m = (b - a) * S
            rho, T = np.zeros(m), np.zeros(m)
            u, q = np.zeros((self.D, m)), np.zeros((self.D, m))
            lbm.lbm_moments(c, rho, u, T, q)
            parts.append((rho, u, T, q))
        return (np.concatenate([p[0] for p in parts]), np.concatenate([p[1] for p in parts], axis=1),
                np.concatenate([p[2] for p in parts]), np.concatenate([p[3] for p in parts], axis=1))

    def conserved(self):
        """(mass, momentum[D], energy) of the whole grid: the slabs' sums
        added with math.fsum (exactly rounded)."""
        res = [lbm.lbm_conserved(c, self.D) for c in self.ctx]
        mass = math.fsum(r[1] for r in res)
        mom = np.array([math.fsum(r[2][a] for r in res) for a in range(self.D)])
        energy = math.fsum(r[3] for r in res)
        return mass, mom, energy

    def close(self):
        for c in self.ctx:
            lbm.lbm_destroy(c)
        self.ctx = []

    def __del__(self):
        self.close()


# ------------------------------------------------ one slab per rank
def halo_peers(rank, world, periodic):
    """(rank below, rank above) along the split axis, None at a wall."""
    below = rank - 1 if rank > 0 else (world - 1 if periodic else None)
    above = rank + 1 if rank < world - 1 else (0 if periodic else None)
    return below, above


def exchange_halos(send_below, send_above, recv_below, recv_above, rank, world, periodic, group=None):
    """One halo exchange between ranks holding consecutive slabs: this rank's
    message for the neighbour below (send_below) and above (send_above) go
    out, the neighbours' messages arrive in recv_below / recv_above (tensors
    of the same size; None on a wall side).  All four transfers are posted
    together (torch.distributed.batch_isend_irecv), so no rank waits on
    another's order; a single periodic rank sends to itself.

    Messages between one pair of ranks are matched in the order they are
    posted (NCCL and gloo point-to-point carry no usable tag), and with two
    ranks on a periodic axis the neighbour below is also the one above.
    Every rank therefore posts its sends as (below, above) and its receives
    as (above, below): the peer's first message to this rank, its downward
    one, lands in recv_above, its upward one in recv_below."""
    import torch.distributed as dist

    below, above = halo_peers(rank, world, periodic)
    if world == 1:
        if periodic:
            recv_below.copy_(send_above)
            recv_above.copy_(send_below)
        return
    ops = []
    if below is not None:
        ops.append(dist.P2POp(dist.isend, send_below, below, group))
    if above is not None:
        ops.append(dist.P2POp(dist.isend, send_above, above, group))
    if above is not None:
        ops.append(dist.P2POp(dist.irecv, recv_above, above, group))
    if below is not None:
        ops.append(dist.P2POp(dist.irecv, recv_below, below, group))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()


class DistributedSlab:
    """The slab of one rank (rank r of world holds split(n_axis, world)[r]) on
    the current device, stepped with halo messages through torch.distributed
    (NCCL); the message buffers are device tensors."""

    def __init__(self, w, rank, world, stream=None, group=None):
        import torch

        self.w, self.rank, self.world, self.group = w, rank, world, group
        self.D = W.dims(w["lattice"])
        self.a, self.b = split(axis_length(w), world)[rank]
        self.periodic = periodic_axis(w)
        opt = lbm.options(w.get("precision", W.FP64), w.get("force_order", 2), w.get("bc", (0, 0, 0)),
                          w.get("T_lo", (1.0,) * 3), w.get("T_hi", (1.0,) * 3), stream, 0, 0,
                          lbm.LBM_KERNEL_AUTO, 0, w.get("mu", 0.0), w.get("include_sigma", False))
        self.ctx = lbm.lbm_create_slab(w["lattice"], *w["shape"], self.a, self.b, w["tau"],
                                       own_part(w, self.a, self.b)[3], opt)
        nbytes = lbm.lbm_slab_halo_bytes(self.ctx)
        below, above = halo_peers(rank, world, self.periodic)
        mk = lambda: torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        self.send = [mk() if below is not None else None, mk() if above is not None else None]
        self.recv = [mk() if below is not None else None, mk() if above is not None else None]

    def init(self):
        rho, u, T, _ = own_part(self.w, self.a, self.b)
        lbm.lbm_init(self.ctx, rho, u, T)
        return self

    def step(self, n=1):
        import torch

        for _ in range(int(n)):
            lbm.lbm_step(self.ctx, 1)
            for side in (0, 1):
                if self.send[side] is not None:
                    lbm.lbm_slab_halo_pack(self.ctx, side, self.send[side])
            torch.cuda.synchronize()
            exchange_halos(self.send[0], self.send[1], self.recv[0], self.recv[1], self.rank, self.world,
                           self.periodic, self.group)
            torch.cuda.synchronize()  # the messages have arrived before the unpack reads them
            for side in (0, 1):
                if self.recv[side] is not None:
                    lbm.lbm_slab_halo_unpack(self.ctx, side, self.recv[side])

    def close(self):
        if self.ctx:
            lbm.lbm_destroy(self.ctx)
            self.ctx = None
