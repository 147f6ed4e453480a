"""The sub-domain decomposition's bookkeeping on the CPU: the partition of
the z levels (dirac_slab_partition, host code of the library) and the halo
exchange between processes (paper_1309_3452_gb300/slabs.py) with gloo ranks:
after one exchange every rank's halo levels hold its neighbours' boundary
levels of the global state, periodically."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1309_3452_gb300 import build as B

B.build()  # dirac_slab_partition is host code of the library

from paper_1309_3452_gb300 import dirac as D  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


@pytest.mark.parametrize("Nz,n", [(34, 4), (11, 2), (7, 3), (5, 5), (9, 1)])
def test_partition_covers_every_level_once(Nz, n):
    parts = D.slab_partition(Nz, n)
    assert [z0 for z0, _ in parts] == [sum(nz for _, nz in parts[:k]) for k in range(n)]
    assert sum(nz for _, nz in parts) == Nz
    assert max(nz for _, nz in parts) - min(nz for _, nz in parts) <= 1
    assert all(nz >= 1 for _, nz in parts)
    assert D.slab_partition(Nz, 0) == []


def global_state(P, Nz, Ny, Nx):
    g = np.zeros((P, Nz, Ny, Nx))
    g += 1000.0 * np.arange(P)[:, None, None, None] + np.arange(Nz)[None, :, None, None]
    g += 0.01 * np.arange(Ny)[None, None, :, None] + 0.0001 * np.arange(Nx)[None, None, None, :]
    return g


def _rank(rank, world, port, Nz, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from paper_1309_3452_gb300 import slabs
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = global_state(8, Nz, 3, 4)
        z0, nz = slabs.partition(Nz, world)[rank]
        local = torch.full((8, nz + 2, 3, 4), float("nan"), dtype=torch.float64)
        local[:, 1:nz + 1] = torch.from_numpy(g[:, z0:z0 + nz])
        slabs.exchange_halos(local, rank, world, dist)
        want = g[:, slabs.global_levels(rank, world, Nz)]
        out[rank] = bool(np.array_equal(local.numpy(), want))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,Nz", [(2, 11), (3, 10)])
def test_halo_exchange_between_gloo_ranks(world, Nz):
    out = mp.get_context("spawn").Manager().dict()  # no fork of this (threaded) process
    mp.spawn(_rank, args=(world, _free_port(), Nz, out), nprocs=world, join=True)
    assert dict(out) == {r: True for r in range(world)}


def test_single_rank_is_its_own_periodic_image():
    import torch
    from paper_1309_3452_gb300 import slabs
    g = global_state(4, 6, 2, 3)
    local = torch.zeros((4, 8, 2, 3), dtype=torch.float64)
    local[:, 1:7] = torch.from_numpy(g)
    slabs.exchange_halos(local, 0, 1, None)
    assert np.array_equal(local.numpy(), g[:, slabs.global_levels(0, 1, 6)])
