"""Halo exchange of the sub-domain decomposition (Sect. 6) between
processes.

The grid is split along its marching axis (z in (3+1)D, y in (2+1)D) into
slabs (dirac_slab_partition: slab k has n_k consecutive levels from z0_k); a
slab is stored as [planes][n + 2][...] (the rest of a level: [Ny][Nx] or
[Nx]) with one halo level below its own levels (index 0) and one above
(index n + 1).  After every time step each slab's last own level becomes its upper
neighbour's lower halo and its first own level its lower neighbour's upper
halo, periodically (the last slab's upper neighbour is the first).  Within
one device the library does this with device copies (dirac_slabs_step);
between processes the same levels travel point to point over
torch.distributed (any backend that can send the tensor: gloo for host
tensors).
"""
from __future__ import annotations

from . import dirac as D


def partition(Nz: int, world: int):
    """[(z0, nz)] per rank: the library's partition (dirac_slab_partition)."""
    return D.slab_partition(Nz, world)


def neighbours(rank: int, world: int):
    """(lower, upper) neighbour ranks along z, periodic."""
    return (rank - 1) % world, (rank + 1) % world


def global_levels(rank: int, world: int, Nz: int):
    """Global level of every stored level of this rank's slab, halos included."""
    z0, nz = partition(Nz, world)[rank]
    return [(z0 - 1 + l) % Nz for l in range(nz + 2)]


# message tags: levels travelling up (to the upper neighbour's lower halo) and down
TAG_UP, TAG_DOWN = 1, 2


def exchange_halos(local, rank: int, world: int, dist) -> None:
    """Refresh the halo levels of this rank's slab `local` (a torch tensor
    [planes][nz + 2][...]) in place from its neighbours' boundary levels."""
    import torch
    nz = local.shape[1] - 2
    if world == 1:  # its own periodic image
        local[:, 0] = local[:, nz]
        local[:, nz + 1] = local[:, 1]
        return
    lower, upper = neighbours(rank, world)
    send_up = local[:, nz].contiguous()
    send_down = local[:, 1].contiguous()
    recv_lower = torch.empty_like(send_up)   # the lower neighbour's last own level
    recv_upper = torch.empty_like(send_down)  # the upper neighbour's first own level
    reqs = [dist.isend(send_up, upper, tag=TAG_UP), dist.isend(send_down, lower, tag=TAG_DOWN),
            dist.irecv(recv_lower, lower, tag=TAG_UP), dist.irecv(recv_upper, upper, tag=TAG_DOWN)]
    for r in reqs:
        r.wait()
    local[:, 0] = recv_lower
    local[:, nz + 1] = recv_upper
