"""Host logic of the time-slab domain decomposition (paper_2306_01098_gb300/domain.py) on the
CPU: the partition, the halo index maps against the lattice coordinates they stand for, and
the halo exchange between two and three gloo ranks, each holding only its own slab of a
global field of site labels.  No GPU is needed."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2306_01098_gb300 import domain


@pytest.mark.parametrize("nt,nparts", [(8, 1), (8, 2), (16, 2), (16, 4), (12, 3), (14, 3), (24, 5)])
def test_partition_covers_time_in_even_slabs(nt, nparts):
    parts = domain.partition((4, 4, 4, nt), nparts)
    assert len(parts) == nparts
    t = 0
    for t0, lt in parts:
        assert t0 == t and t0 % 2 == 0 and lt % 2 == 0 and lt >= 4
        t += lt
    assert t == nt
    assert max(lt for _, lt in parts) - min(lt for _, lt in parts) <= 2


@pytest.mark.parametrize("nt,nparts", [(6, 2), (7, 1), (16, 5)])
def test_partition_rejects_impossible_cuts(nt, nparts):
    with pytest.raises(ValueError):
        domain.partition((4, 4, 4, nt), nparts)


def _half_index(dims, x, y, z, t):
    nx, ny, nz, _ = dims
    return (x + nx * (y + ny * (z + nz * t))) // 2


@pytest.mark.parametrize("dims,nparts", [((6, 4, 4, 12), 3), ((4, 6, 4, 8), 2), ((4, 4, 6, 16), 4)])
def test_halo_maps_are_the_time_neighbours_across_each_cut(dims, nparts):
    # every record of a received halo is the site (x, y, z, t0 - 3 + j) or (x, y, z, t0 + lt + j)
    # (time modulo Nt) whose face index (x + Nx (y + Ny z)) / 2 is the record's position in the
    # slice, for either parity; the block a slab receives is the block its neighbour sends
    nx, ny, nz, nt = dims
    f = nx * ny * nz // 2
    parts = domain.partition(dims, nparts)
    for r, (t0, lt) in enumerate(parts):
        below, above = domain.neighbours(r, nparts)
        lo = domain.halo_index(dims, t0, lt, "lo")
        hi = domain.halo_index(dims, t0, lt, "hi")
        assert np.array_equal(lo, domain.send_index(dims, *parts[below], "hi"))
        assert np.array_equal(hi, domain.send_index(dims, *parts[above], "lo"))
        for q in (0, 1):
            for j in range(3):
                for x in range(nx):
                    for y in range(ny):
                        for z in range(nz):
                            for first, idx in ((t0 - 3, lo), (t0 + lt, hi)):
                                t = (first + j) % nt
                                if (x + y + z + t) % 2 != q:
                                    continue
                                h = (x + nx * (y + ny * z)) // 2
                                assert idx[j * f + h] == _half_index(dims, x, y, z, t)
        rng = domain.slab_range(dims, t0, lt)
        assert rng.start == f * t0 and rng.stop == f * (t0 + lt)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _exchange_worker(rank, world, port, dims, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t0, lt = domain.partition(dims, world)[rank]
        f = domain.face_sites(dims)
        # this rank's slab of a global half-lattice field whose value at every site is its
        # global index (three colours, distinguished by a tenth)
        glob = torch.arange(f * dims[3], dtype=torch.float64)
        field = torch.stack([glob + 0.1 * c for c in range(3)], dim=1)[domain.slab_range(dims, t0, lt)].contiguous()
        send_lo, send_hi = field[:3 * f].clone(), field[-3 * f:].clone()
        recv_lo, recv_hi = torch.full_like(send_lo, -1.0), torch.full_like(send_hi, -1.0)
        domain.exchange_dist(send_lo, send_hi, recv_lo, recv_hi, rank, world)
        ok_lo = np.array_equal(recv_lo[:, 0].numpy(), domain.halo_index(dims, t0, lt, "lo").astype(np.float64))
        ok_hi = np.array_equal(recv_hi[:, 0].numpy(), domain.halo_index(dims, t0, lt, "hi").astype(np.float64))
        ok_c = bool(torch.allclose(recv_lo[:, 2] - recv_lo[:, 0], torch.full_like(recv_lo[:, 0], 0.2)))
        out[rank] = (ok_lo, ok_hi, ok_c)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,dims", [(2, (4, 4, 4, 8)), (3, (4, 4, 6, 12))])
def test_halo_exchange_between_gloo_ranks(world, dims):
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_exchange_worker, args=(world, _free_port(), dims, out), nprocs=world, join=True)
    assert dict(out) == {r: (True, True, True) for r in range(world)}


def test_single_slab_is_its_own_neighbour():
    dims = (4, 4, 4, 8)
    f = domain.face_sites(dims)
    field = torch.arange(f * 8, dtype=torch.float64)[:, None].repeat(1, 3)
    send_lo, send_hi = field[:3 * f].clone(), field[-3 * f:].clone()
    recv_lo, recv_hi = torch.empty_like(send_lo), torch.empty_like(send_hi)
    domain.exchange_dist(send_lo, send_hi, recv_lo, recv_hi, 0, 1)
    assert np.array_equal(recv_lo[:, 0].numpy(), domain.halo_index(dims, 0, 8, "lo"))
    assert np.array_equal(recv_hi[:, 0].numpy(), domain.halo_index(dims, 0, 8, "hi"))
