"""(x, y) domain decomposition of one grid, and the halo exchange of its blocks.

MicroHH, the code whose stencils the paper tunes (Sec. 5.1-5.2), splits one
grid over many GPUs in x and y.  Each block keeps g ghost cells on every side
(`kl_grid.xybc = 1`: the library fills only their z planes) and receives its
x and y ghosts from its neighbours once per step:

  phase x: every block packs its g interior columns next to the west face
           (side 0) and the east face (side 1), over its interior rows and
           levels; the west strip goes to the west neighbour, which unpacks
           it into its east ghosts, and the east strip to the east neighbour
           (west ghosts);
  phase y: the same with the south / north neighbours, over rows that span
           the padded x extent, so the x ghosts received in phase x travel
           on to the diagonal neighbours: no corner messages;
  then     kl_fill_ghosts / kl_step fill the z ghost planes of every column,
           the received ones included (walls mirror, periodic z wraps).

The global grid is periodic in x and y, so the neighbours wrap around the
process grid; with one block along an axis that block is its own neighbour.

Pack and unpack run in libkl (kl_halo_pack / kl_halo_unpack).  The transport
between blocks is separate: `DistTransport` sends with torch.distributed
point-to-point operations (NCCL between GPUs), one block per process;
`LocalTransport` copies between blocks that one process holds.  This module
only decides who sends which strip to whom; every element is moved by
libkl's kernels or by the transport.
"""

from __future__ import annotations

from dataclasses import dataclass


def split(n: int, p: int):
    """[(start, size)] of p nearly equal parts of range(n), larger parts first."""
    if p < 1 or n < p:
        raise ValueError(f"cannot split {n} points into {p} parts")
    q, r = divmod(n, p)
    out, s = [], 0
    for i in range(p):
        m = q + (1 if i < r else 0)
        out.append((s, m))
        s += m
    return out


@dataclass(frozen=True)
class Block:
    rank: int
    rx: int
    ry: int
    x0: int
    nx: int
    y0: int
    ny: int


class Decomposition:
    """A global nx x ny x nz grid over px x py blocks; rank = rx + px * ry."""

    def __init__(self, nx: int, ny: int, nz: int, px: int, py: int, g: int):
        self.nx, self.ny, self.nz, self.px, self.py, self.g = nx, ny, nz, px, py, g
        self.xs, self.ys = split(nx, px), split(ny, py)
        if min(m for _, m in self.xs) < g or min(m for _, m in self.ys) < g:
            raise ValueError("every block must be at least g points wide in x and y")

    @property
    def size(self) -> int:
        return self.px * self.py

    def block(self, rank: int) -> Block:
        rx, ry = rank % self.px, rank // self.px
        (x0, bnx), (y0, bny) = self.xs[rx], self.ys[ry]
        return Block(rank, rx, ry, x0, bnx, y0, bny)

    def neighbour(self, rank: int, axis: int, side: int) -> int:
        """The block next to `rank` across its side-0 (west / south) or side-1
        (east / north) face of `axis`, periodically."""
        rx, ry = rank % self.px, rank // self.px
        d = 1 if side else -1
        if axis == 0:
            rx = (rx + d) % self.px
        else:
            ry = (ry + d) % self.py
        return rx + self.px * ry


class LocalTransport:
    """Strips between blocks held by one process: the side-s strip of block b
    lands in the side-(1-s) receive buffer of b's neighbour across side s."""

    def exchange(self, decomp: Decomposition, axis: int, send: dict, recv: dict) -> None:
        for r, bufs in send.items():
            for s in (0, 1):
                recv[decomp.neighbour(r, axis, s)][1 - s].copy_(bufs[s])


class DistTransport:
    """One block per process, strips sent with torch.distributed point-to-point
    operations (NCCL for device buffers, gloo for host buffers).

    Each process posts its two sends (side 0, side 1) and two receives (the
    upper neighbour's side-0 strip first, then the lower neighbour's side-1
    strip).  Tags name the sender's side; where both neighbours are the same
    process (two blocks along the axis) the posting order alone also pairs
    them, for backends that ignore tags."""

    def __init__(self, group=None):
        self.group = group

    def exchange(self, decomp: Decomposition, axis: int, send: dict, recv: dict) -> None:
        import torch.distributed as dist
        (rank, sbufs), = send.items()
        rbufs = recv[rank]
        lo, hi = decomp.neighbour(rank, axis, 0), decomp.neighbour(rank, axis, 1)
        if lo == rank and hi == rank:           # alone on this axis: a periodic copy
            rbufs[0].copy_(sbufs[1])
            rbufs[1].copy_(sbufs[0])
            return
        ops = [dist.P2POp(dist.isend, sbufs[0], lo, self.group, tag=2 * axis),
               dist.P2POp(dist.isend, sbufs[1], hi, self.group, tag=2 * axis + 1),
               dist.P2POp(dist.irecv, rbufs[1], hi, self.group, tag=2 * axis),
               dist.P2POp(dist.irecv, rbufs[0], lo, self.group, tag=2 * axis + 1)]
        for req in dist.batch_isend_irecv(ops):
            req.wait()


class KLPacker:
    """Strips moved by libkl's kernels (device buffers, fields as device pointers)."""

    def __init__(self, ctx, stream=None):
        self.ctx, self.stream = ctx, stream

    def buffer(self, problem, axis: int, nf: int):
        import torch
        from . import kl
        n = kl.kl_halo_bytes(problem.grid, problem.dtype, axis, nf)
        return torch.empty(n, dtype=torch.uint8, device=problem.device)

    def pack(self, problem, axis, side, fields, buf) -> None:
        from . import kl
        kl.kl_halo_pack(self.ctx, problem.dtype, problem.grid, axis, side, fields, buf.data_ptr(),
                        self._sp())

    def unpack(self, problem, axis, side, fields, buf) -> None:
        from . import kl
        kl.kl_halo_unpack(self.ctx, problem.dtype, problem.grid, axis, side, fields,
                          buf.data_ptr(), self._sp())

    def _sp(self):
        return None if self.stream is None else self.stream.cuda_stream


class HaloExchange:
    """The two-phase exchange for the blocks `ranks` of `decomp` that this
    process holds (one under torchrun, all of them in a single process).

    problems[r] is block r's Problem (xybc = 1); exchange() takes, per block,
    the fields to exchange (what the packer understands: device pointers for
    KLPacker) and leaves their x and y ghosts of interior levels filled."""

    def __init__(self, decomp: Decomposition, problems: dict, nf: int, transport, packer):
        self.decomp, self.problems, self.nf = decomp, problems, nf
        self.transport, self.packer = transport, packer
        self.send = {a: {r: [packer.buffer(p, a, nf) for _ in (0, 1)] for r, p in problems.items()}
                     for a in (0, 1)}
        self.recv = {a: {r: [packer.buffer(p, a, nf) for _ in (0, 1)] for r, p in problems.items()}
                     for a in (0, 1)}

    def exchange(self, fields: dict, sync=None) -> None:
        """fields[r]: block r's nf fields.  `sync` (optional) runs between the
        packs and the transport, e.g. a stream synchronisation."""
        for axis in (0, 1):
            for r, p in self.problems.items():
                for side in (0, 1):
                    self.packer.pack(p, axis, side, fields[r], self.send[axis][r][side])
            if sync is not None:
                sync()
            self.transport.exchange(self.decomp, axis, self.send[axis], self.recv[axis])
            if sync is not None:
                sync()
            for r, p in self.problems.items():
                for side in (0, 1):
                    self.packer.unpack(p, axis, side, fields[r], self.recv[axis][r][side])
