"""A periodic box split into z-slabs across gloo ranks on the CPU (the
cross-rank level synchronisation of Sec. III): before every RK4 stage each
rank fills its x/y ghosts periodically and exchanges its z halos with its
neighbours (decomp.exchange_z_halos); the stages run in the oracle.  Every
rank's slab after several steps must equal, bit for bit, the same slab of the
undecomposed box stepped with periodic ghosts: a right-hand side depends only
on its stencil's values, so a correct exchange reproduces it exactly."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle
from paper_1806_04182_gb300 import decomp, inputs

G = 3


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rk4(U, dx, dt, system, fill, steps):
    """RK4 steps (Sec. II.C) of a ghosted array with the oracle's RHS;
    `fill` fills the ghost shell of a ghosted array before each stage."""
    def L(V):
        fill(V)
        return oracle.rhs(system, V, dx)
    g = G
    inner = (slice(None), slice(g, -g), slice(g, -g), slice(g, -g))
    for _ in range(steps):
        u = U[inner].copy()
        k1 = dt * L(U)
        V = U.copy()
        V[inner] = u + 0.5 * k1
        k2 = dt * L(V)
        V[inner] = u + 0.5 * k2
        k3 = dt * L(V)
        V[inner] = u + k3
        k4 = dt * L(V)
        U[inner] = u + (k1 + 2.0 * k2 + 2.0 * k3 + k4) / 6.0
    return U


def data(system, n):
    if system == oracle.Z4:
        return inputs.z4_perturbed(n, seed=5, amp=0.04)
    return inputs.wave_plane(n, seed=2)


def _worker(rank, world, port, system, n, steps, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        U0, dx = data(system, n)
        dt = 0.25 * min(dx)
        z0, nzl = decomp.slab_bounds(n[2], rank, world)
        local = oracle.ghosted(np.ascontiguousarray(U0[:, z0:z0 + nzl]))

        def fill(V):
            oracle.fill_ghosts(V, G)               # x, y (and z, overwritten next)
            t = torch.from_numpy(V)
            decomp.exchange_z_halos(t, G)          # z from the neighbours

        rk4(local, dx, dt, system, fill, steps)
        whole = rk4(oracle.ghosted(U0.copy()), dx, dt, system, lambda V: oracle.fill_ghosts(V, G),
                    steps)
        want = oracle.interior(whole)[:, z0:z0 + nzl]
        q.put((rank, bool(np.array_equal(oracle.interior(local), want)),
               float(np.abs(oracle.interior(local) - want).max())))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("system,n,world", [
    (oracle.WAVE, (10, 8, 12), 2),
    (oracle.WAVE, (9, 7, 10), 3),    # slabs of 4, 3, 3 planes
    (oracle.Z4, (8, 7, 12), 2),
])
def test_slab_decomposition_equals_undecomposed_box(system, n, world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, system, n, 2, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == list(range(world))
    assert all(o[1] for o in out), out


def test_slab_bounds_cover_the_box():
    for nz, world in ((12, 2), (10, 3), (7, 7), (96, 5)):
        spans = [decomp.slab_bounds(nz, r, world) for r in range(world)]
        assert spans[0][0] == 0
        assert all(a + b == c for (a, b), (c, _) in zip(spans, spans[1:]))
        assert spans[-1][0] + spans[-1][1] == nz
        assert max(s[1] for s in spans) - min(s[1] for s in spans) <= 1
    with pytest.raises(ValueError):
        decomp.slab_bounds(8, 2, 2)


def test_single_rank_wraps_its_own_slab():
    # no process group: the z ghosts are the slab's own periodic images,
    # exactly the oracle's periodic fill
    U0, _ = data(oracle.WAVE, (6, 5, 7))
    V = oracle.ghosted(U0.copy())
    W = V.copy()
    W[:, :G] = 0.0
    W[:, -G:] = 0.0
    decomp.exchange_z_halos(torch.from_numpy(W), G)
    assert np.array_equal(W, V)
