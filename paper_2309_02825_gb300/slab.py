"""One grid over several processes (one GPU each): slab decomposition along
the slowest axis with a ghost-layer exchange before every sweep.

The streaming of Eq. (distribution-f) moves each population one node along
its velocity, so between two steps the only data a slab needs from outside
are the populations that cross its two cuts (include/lb_slab.h).
``halo_exchange`` moves the packed buffers of every part to its neighbours
with point-to-point messages of ``torch.distributed`` (NCCL between GPUs;
any backend whose tensors live where the buffers do).  Parts are numbered
along the slowest axis, periodically: part p sends "up" to p+1 and "down" to
p-1, and receives from p-1 what it sent up and from p+1 what it sent down.
With one part the buffers wrap onto the part itself.
"""

from __future__ import annotations

import torch
import torch.distributed as dist

from . import lb

TAG_UP, TAG_DOWN = 1, 2


def halo_exchange(send_down, send_up, recv_down, recv_up, rank, world, group=None):
    """recv_down <- send_up of part rank-1, recv_up <- send_down of part
    rank+1 (periodic).  Messages between one pair are posted in the same order
    on both sides (up first), so backends that match by order (NCCL) and by
    tag agree; two parts are each other's upper and lower neighbour."""
    if world == 1:
        recv_down.copy_(send_up)
        recv_up.copy_(send_down)
        return
    up, down = (rank + 1) % world, (rank - 1) % world
    ops = [dist.P2POp(dist.isend, send_up, up, group, TAG_UP),
           dist.P2POp(dist.irecv, recv_down, down, group, TAG_UP),
           dist.P2POp(dist.isend, send_down, down, group, TAG_DOWN),
           dist.P2POp(dist.irecv, recv_up, up, group, TAG_DOWN)]
    for req in dist.batch_isend_irecv(ops):
        req.wait()


def slab_layers(N, part, nparts):
    """(first layer, layers) of part `part`: N layers on the slowest axis cut
    into nparts slabs, the first N mod nparts taking one more."""
    base, extra = N // nparts, N % nparts
    return part * base + min(part, extra), base + (1 if part < extra else 0)


def with_ghost_layers(field, z0, nz, vector=False):
    """The owned layers z0 .. z0+nz-1 of a whole-grid field (slowest axis
    first, or second for a vector field) plus one layer on each side,
    periodic."""
    ax = 1 if vector else 0
    n = field.shape[ax]
    idx = torch.tensor([(z0 - 1 + k) % n for k in range(nz + 2)], device=field.device)
    return field.index_select(ax, idx).contiguous()


class SlabRunner:
    """This process's part of the grid on its current CUDA device."""

    def __init__(self, d, N, nu, dx, dt, precision="fx64", theta_ref=0.0, rank=None, world=None, group=None,
                 stream=None):
        self.rank = dist.get_rank(group) if rank is None else int(rank)
        self.world = dist.get_world_size(group) if world is None else int(world)
        self.group = group
        self.slab = lb.Slab(d, N, self.rank, self.world, nu, dx, dt, precision, theta_ref, stream)
        self.send = self.slab.halo_buffers(2)
        self.recv = self.slab.halo_buffers(2)
        self.steps = 0

    def set_theta0(self, theta0, grad0):
        """theta0 / grad theta0 of the whole grid (any device); every rank
        passes the same fields."""
        s = self.slab
        th = with_ghost_layers(theta0, s.z0, s.nz).to("cuda", torch.float64)
        g = with_ghost_layers(grad0, s.z0, s.nz, vector=True).to("cuda", torch.float64)
        s.set_theta0(th, g, float(theta0.abs().max()))
        self.steps = 0

    def exchange(self):
        """Pack, move, unpack.  The part's kernels and copies run on the CUDA
        stream that was current when the runner was made; torch.distributed
        orders its messages after the current stream's work and the current
        stream after their completion, so keep that stream current."""
        s = self.slab
        s.pack(self.send[0], self.send[1])
        halo_exchange(self.send[0], self.send[1], self.recv[0], self.recv[1], self.rank, self.world, self.group)
        s.unpack(self.recv[0], self.recv[1])

    def step(self, n):
        for _ in range(int(n)):
            self.exchange()
            self.slab.step()
            self.steps += 1

    def macros(self):
        self.exchange()
        return self.slab.macros()

    def sum_theta(self):
        """The whole grid's total (all-reduced)."""
        v = torch.tensor([self.slab.sum_theta()], dtype=torch.float64, device="cuda")
        if self.world > 1:
            dist.all_reduce(v, group=self.group)
        return float(v.item())
