"""A periodic box split across ranks into z-slabs: the level synchronisation
of Sec. III between processors.

Each rank holds one slab of the box as a ghosted array (fields, z, y, x;
x fastest), with the same ghost width g in every direction.  Before every
RK stage the slab's ghost shell must hold its neighbours' values:

* in x and y the slab is its own periodic neighbour, so those ghosts are
  filled locally (``sf_fill_ghosts_periodic`` on the device, or any periodic
  fill), which also fills the x/y ghost columns of the slab's own planes;
* in z the g planes below the slab are the top g interior planes of the
  rank below (periodically: rank 0's lower neighbour is the last rank) and
  the g planes above are the bottom g interior planes of the rank above.
  ``exchange_z_halos`` sends those whole planes (x/y ghost columns included,
  so edges and corners arrive filled) with point-to-point messages and
  writes them into the ghost planes.

Only data moves here; the stages themselves run in libsf.so (or in the
oracle, for the CPU tests).  The exchange is one step per RK stage, the one
collective the substep needs when a box spans ranks.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def slab_bounds(nz: int, rank: int, world: int) -> tuple[int, int]:
    """(first interior plane, number of planes) of `rank`'s slab: the nz
    planes split as evenly as possible, lower ranks taking the extra ones."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank outside the group")
    base, extra = divmod(nz, world)
    z0 = rank * base + min(rank, extra)
    return z0, base + (1 if rank < extra else 0)


def exchange_z_halos(U: torch.Tensor, g: int, group=None) -> None:
    """Fill the g ghost planes below and above the slab U (fields, nzl + 2g,
    ny', nx') from the neighbouring ranks' interior planes.  Every rank of
    the group calls it; each slab needs nzl >= g planes.  A group of one rank
    wraps its own slab periodically."""
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    nzl = U.shape[1] - 2 * g
    if nzl < g:
        raise ValueError(f"a slab of {nzl} planes cannot feed {g} ghost planes")
    if world == 1:
        U[:, :g].copy_(U[:, nzl:nzl + g])
        U[:, nzl + g:].copy_(U[:, g:2 * g])
        return
    rank = dist.get_rank(group)
    below, above = (rank - 1) % world, (rank + 1) % world
    top = U[:, nzl:nzl + g].contiguous()        # -> the rank above, its lower ghosts
    bottom = U[:, g:2 * g].contiguous()         # -> the rank below, its upper ghosts
    from_below = torch.empty_like(top)
    from_above = torch.empty_like(bottom)
    # tags tell the two messages of a two-rank ring apart (both go to one peer)
    ops = [dist.P2POp(dist.isend, top, above, group, tag=0),
           dist.P2POp(dist.isend, bottom, below, group, tag=1),
           dist.P2POp(dist.irecv, from_below, below, group, tag=0),
           dist.P2POp(dist.irecv, from_above, above, group, tag=1)]
    for req in dist.batch_isend_irecv(ops):
        req.wait()
    U[:, :g].copy_(from_below)
    U[:, nzl + g:].copy_(from_above)
