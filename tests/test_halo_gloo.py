"""The (x, y) domain decomposition and its two-phase halo exchange, on CPU.

Each rank of a gloo process group holds one block of a seeded global grid
(periodic x, y; free-slip walls or periodic z).  The block's padded arrays
start with NaN ghosts; the exchange of paper_2303_12374_gb300.halo (x phase,
then y phase, DistTransport over gloo) fills the x and y ghosts, a z fill by
the wall / periodic rules fills the z planes, and then:

  * every padded block equals the window of the globally padded grid
    (oracle.pad) at the block's place, bit for bit: every ghost, corners
    included, came from the right neighbour;
  * the tendencies the oracle computes on each padded block, gathered,
    equal the oracle's tendencies of the whole grid bit for bit.

The strips move through the same protocol as on GPUs; here a host packer
(below) stands in for libkl's pack / unpack kernels, whose regions it copies
from include/kl.h.  The GPU tests check those kernels against the same
regions and the decomposed step against the oracle on one GPU.
"""

from __future__ import annotations

import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

NX, NY, NZ, G = 22, 18, 10, 3


class HostProblem:
    def __init__(self, nx, ny, nz, g):
        self.nx, self.ny, self.nz, self.g = nx, ny, nz, g


def strip_slices(p, axis, side, unpack):
    """(z, y, x) slices of the strip in a padded (nz+2g, ny+2g, nx+2g) array,
    the regions of kl_halo_pack / kl_halo_unpack."""
    g = p.g
    zs = slice(g, g + p.nz)
    if axis == 0:
        if unpack:
            x0 = g + p.nx if side else 0
        else:
            x0 = g + p.nx - g if side else g
        return zs, slice(g, g + p.ny), slice(x0, x0 + g)
    if unpack:
        y0 = g + p.ny if side else 0
    else:
        y0 = g + p.ny - g if side else g
    return zs, slice(y0, y0 + g), slice(0, p.nx + 2 * g)


class HostPacker:
    def buffer(self, p, axis, nf):
        import torch
        w = p.g if axis == 0 else p.nx + 2 * p.g
        h = p.ny if axis == 0 else p.g
        return torch.empty((nf, p.nz, h, w), dtype=torch.float64)

    def pack(self, p, axis, side, fields, buf):
        import torch
        for f, a in enumerate(fields):
            buf[f].copy_(torch.from_numpy(np.ascontiguousarray(a[strip_slices(p, axis, side, False)])))

    def unpack(self, p, axis, side, fields, buf):
        for f, a in enumerate(fields):
            a[strip_slices(p, axis, side, True)] = buf[f].numpy()


def zfill(a, g, nz, walls, odd):
    """z ghost planes of a padded block, every column (x, y ghosts included)."""
    for m in range(g):
        if not walls:
            a[g - 1 - m] = a[g + nz - 1 - m]
            a[g + nz + m] = a[g + m]
        elif odd:
            a[g - 1 - m] = -a[g + 1 + m]
            a[g + nz + m] = 0.0 if m == 0 else -a[g + nz - m]
        else:
            a[g - 1 - m] = a[g + m]
            a[g + nz + m] = a[g + nz - 1 - m]


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, px, py, walls, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch.distributed as dist
    import oracle
    from paper_2303_12374_gb300 import halo, synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        d = halo.Decomposition(NX, NY, NZ, px, py, G)
        b = d.block(rank)
        zh = synth.zfaces(NZ, 1.0, 2.0 if walls else 0.0)
        f = synth.velocity_fields(NX, NY, NZ, seed=4242, walls=walls, zh=zh)
        p = HostProblem(b.nx, b.ny, NZ, G)
        pads = []
        for k in ("u", "v", "w"):
            a = np.full((NZ + 2 * G, b.ny + 2 * G, b.nx + 2 * G), np.nan)
            a[G:G + NZ, G:G + b.ny, G:G + b.nx] = f[k][:, b.y0:b.y0 + b.ny, b.x0:b.x0 + b.nx]
            pads.append(a)
        ex = halo.HaloExchange(d, {rank: p}, 3, halo.DistTransport(), HostPacker())
        ex.exchange({rank: pads})
        for a, odd in zip(pads, (False, False, True)):
            zfill(a, G, NZ, walls, odd)
        ok_pad = []
        for k, a, odd in zip(("u", "v", "w"), pads, (False, False, True)):
            gp = oracle.pad(f[k], G, walls, odd)
            # the global padded array, wrapped periodically in x and y around
            # the block's window (the block's ghosts reach across x = 0 / nx)
            ix = (np.arange(b.x0 - G, b.x0 + b.nx + G) % NX) + G
            iy = (np.arange(b.y0 - G, b.y0 + b.ny + G) % NY) + G
            win = gp[:, iy][:, :, ix]
            ok_pad.append(bool(np.array_equal(win, a)))
        t = oracle.tendencies_padded(*pads, adv=5, diff=1, g=G, walls=walls, dx=1.0 / NX,
                                     dy=1.0 / NY, zh=zh, nu=1e-3)
        res = [None] * world
        dist.all_gather_object(res, (b.x0, b.nx, b.y0, b.ny, [x.tolist() for x in t], ok_pad))
        if rank == 0:
            full = oracle.tendencies(f["u"], f["v"], f["w"], adv=5, diff=1, g=G, walls=walls,
                                     dx=1.0 / NX, dy=1.0 / NY, zh=zh, nu=1e-3)
            asm = [np.full((NZ, NY, NX), np.nan) for _ in range(3)]
            pads_ok = True
            for x0, bnx, y0, bny, tl, okp in res:
                pads_ok &= all(okp)
                for c in range(3):
                    asm[c][:, y0:y0 + bny, x0:x0 + bnx] = np.array(tl[c])
            same = all(np.array_equal(a, r) for a, r in zip(asm, full))
            with open(os.path.join(out_dir, "result.txt"), "w") as fh:
                fh.write(f"{int(pads_ok)} {int(same)}\n")
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("px,py,walls", [(2, 1, True), (1, 2, False), (2, 2, True)])
def test_gloo_ranks_exchange_halos_and_match_the_single_grid_oracle(tmp_path, px, py, walls):
    import torch.multiprocessing as mp
    world = px * py
    mp.start_processes(_rank_main, args=(world, px, py, walls, _free_port(), str(tmp_path)),
                       nprocs=world, start_method="spawn")
    pads_ok, same = (int(x) for x in open(tmp_path / "result.txt").read().split())
    assert pads_ok == 1, "a padded block differs from the global grid's window"
    assert same == 1, "assembled block tendencies differ from the whole grid's"


def test_decomposition_geometry():
    sys.path.insert(0, ROOT)
    from paper_2303_12374_gb300 import halo
    assert halo.split(10, 3) == [(0, 4), (4, 3), (7, 3)]
    d = halo.Decomposition(22, 18, 4, 3, 2, 3)
    # every interior point in exactly one block
    cover = np.zeros((18, 22), int)
    for r in range(d.size):
        b = d.block(r)
        cover[b.y0:b.y0 + b.ny, b.x0:b.x0 + b.nx] += 1
    assert np.all(cover == 1)
    # neighbours wrap and are mutual
    for r in range(d.size):
        for axis in (0, 1):
            assert d.neighbour(d.neighbour(r, axis, 1), axis, 0) == r
    assert d.neighbour(0, 0, 0) == 2 and d.neighbour(0, 1, 0) == 3
    with pytest.raises(ValueError):
        halo.Decomposition(8, 8, 4, 3, 1, 3)       # a block narrower than g
