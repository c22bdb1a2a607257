"""The slab decomposition's exchange (paper_2309_02825_gb300/slab.py) with
gloo ranks on the CPU.  Each rank steps its part of the grid, its owned
layers plus one ghost layer on each side, with the oracle (pre-collision
form: the ghost layers must hold the neighbours' boundary layers, all
populations, before every step), and the ghost layers are refreshed through
the same ``halo_exchange``, ``slab_layers`` and ``with_ghost_layers`` the
GPU runner uses.  The gathered owned layers must equal one oracle run of the
whole grid bit for bit: every owned node then saw the inputs of the whole
grid.  2 and 3 ranks (2: each part is both neighbours of the other)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as O
from paper_2309_02825_gb300 import slab as SL
from paper_2309_02825_gb300 import workloads as W


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case(d, N):
    nu = 0.02
    prob = W.FourierProblem.random(d, nu, 6, 3, 0.1, 1.5, 5 + d)
    dx = 1.0 / max(N)
    dt = 0.2 * dx * dx / nu
    return prob, nu, dx, dt


def _worker(rank, world, port, d, N, T, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    O.set_threads(1)
    prob, nu, dx, dt = _case(d, N)
    th0 = torch.from_numpy(prob.theta(N, dx))
    g0 = torch.from_numpy(np.ascontiguousarray(prob.grad(N, dx)))
    z0, nz = SL.slab_layers(N[-1], rank, world)
    th_ext = SL.with_ghost_layers(th0, z0, nz).numpy()
    g_ext = SL.with_ghost_layers(g0, z0, nz, vector=True).numpy()
    Nl = tuple(N[:-1]) + (nz + 2,)
    m = O.Model(d, Nl, nu, dx, dt)
    f = m.initialize(th_ext, g_ext)  # pre-collision f on owned and ghost layers
    send = [torch.empty((m.q,) + f.shape[2:], dtype=torch.float64) for _ in range(2)]
    recv = [torch.empty_like(send[0]) for _ in range(2)]
    for _ in range(T):
        # the ghost layers take the neighbours' boundary layers (all populations)
        send[0].copy_(torch.from_numpy(f[:, 1]))
        send[1].copy_(torch.from_numpy(f[:, nz]))
        SL.halo_exchange(send[0], send[1], recv[0], recv[1], rank, world)
        f[:, 0] = recv[0].numpy()
        f[:, nz + 1] = recv[1].numpy()
        f = m.step(f)
    out[rank] = (z0, nz, np.ascontiguousarray(f[:, 1:nz + 1]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,d,N,T", [(2, 2, (24, 10), 9), (3, 2, (17, 11), 7), (3, 3, (8, 6, 7), 5),
                                         (2, 3, (6, 5, 2), 4)])
def test_gloo_slabs_equal_one_grid(world, d, N, T):
    port = _free_port()
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, d, N, T, out), nprocs=world, join=True)
        parts = dict(out)
    prob, nu, dx, dt = _case(d, N)
    m = O.Model(d, N, nu, dx, dt)
    ref = m.run(m.initialize(prob.theta(N, dx), prob.grad(N, dx)), T)
    covered = 0
    for rank in range(world):
        z0, nz, fpart = parts[rank]
        assert np.array_equal(fpart, ref[:, z0:z0 + nz]), rank
        covered += nz
    assert covered == N[-1]


def test_slab_layers_cover_the_axis():
    for n in (1, 2, 7, 10, 64):
        for parts in range(1, n + 1):
            spans = [SL.slab_layers(n, p, parts) for p in range(parts)]
            assert spans[0][0] == 0 and all(nz >= 1 for _, nz in spans)
            assert all(spans[p][0] + spans[p][1] == spans[p + 1][0] for p in range(parts - 1))
            assert spans[-1][0] + spans[-1][1] == n
            assert max(nz for _, nz in spans) - min(nz for _, nz in spans) <= 1
