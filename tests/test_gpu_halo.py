"""The (x, y) decomposed path on one GPU, through the C ABI.

  * kl_halo_pack / kl_halo_unpack move exactly the strips include/kl.h
    defines (bit for bit, every storage type, 3 and 4 fields);
  * with grid.xybc = 1 the ghost fill writes only the z planes, each from its
    own column, and leaves the x / y ghosts of interior levels alone;
  * a grid split into 2 x 2 blocks (each block at least 67 columns wide, so a
    zpack kernel would wrap x itself if the block did not say xybc = 1), halo
    exchange through libkl's kernels and device copies (LocalTransport), one
    kl_step per block: the assembled tendencies equal the oracle's of the
    whole grid within the tolerances of every other parity test.
"""

from __future__ import annotations

import os

import numpy as np
import pytest

from gpu_cases import TOL, make_inputs, rel_err

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WISDOM = os.path.join(ROOT, "paper_2303_12374_gb300", "wisdom")


def _region(p, axis, side, unpack):
    """(z, y, x) slices of a strip in the padded view (include/kl.h regions)."""
    g = p.g
    zs = slice(g, g + p.nz)
    if axis == 0:
        x0 = (g + p.nx if side else 0) if unpack else (p.nx if side else g)
        return zs, slice(g, g + p.ny), slice(x0, x0 + g)
    y0 = (g + p.ny if side else 0) if unpack else (p.ny if side else g)
    return zs, slice(y0, y0 + g), slice(0, p.nx + 2 * g)


@pytest.mark.parametrize("dtype", [0, 1, 2])
@pytest.mark.parametrize("nf", [3, 4])
def test_pack_unpack_regions_bit_exact(dtype, nf):
    import torch
    from paper_2303_12374_gb300 import kl
    from paper_2303_12374_gb300.problem import Problem
    ctx = kl.kl_create(0, None)
    try:
        p = Problem(37, 29, 11, g=3, dtype=dtype, walls=True, dz=1.0 / 11, xybc=True)
        gen = torch.Generator(device="cuda").manual_seed(5 + dtype)
        bufs = [torch.randn(p.extent, generator=gen, device="cuda").to(p.tdtype) for _ in range(nf)]
        ptrs = [b.data_ptr() for b in bufs]
        for axis in (0, 1):
            nbytes = kl.kl_halo_bytes(p.grid, p.dtype, axis, nf)
            for side in (0, 1):
                sbuf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
                kl.kl_halo_pack(ctx, p.dtype, p.grid, axis, side, ptrs, sbuf.data_ptr())
                torch.cuda.synchronize()
                got = sbuf.view(p.tdtype)
                want = torch.cat([p.padded_view(b)[_region(p, axis, side, False)].reshape(-1)
                                  for b in bufs])
                assert torch.equal(got.view(torch.int16 if dtype == 2 else p.tdtype),
                                   want.view(torch.int16 if dtype == 2 else p.tdtype))
                # unpack into copies: exactly the ghost region changes
                dst = [torch.zeros_like(b) for b in bufs]
                kl.kl_halo_unpack(ctx, p.dtype, p.grid, axis, side, [d.data_ptr() for d in dst],
                                  sbuf.data_ptr())
                torch.cuda.synchronize()
                for d, b in zip(dst, bufs):
                    exp = torch.zeros_like(b)
                    p.padded_view(exp)[_region(p, axis, side, True)] = \
                        p.padded_view(b)[_region(p, axis, side, False)]
                    assert torch.equal(d.view(torch.int16 if dtype == 2 else p.tdtype),
                                       exp.view(torch.int16 if dtype == 2 else p.tdtype))
    finally:
        kl.kl_destroy(ctx)


def test_fill_with_xybc_writes_only_z_planes():
    import torch
    from paper_2303_12374_gb300 import kl
    from paper_2303_12374_gb300.problem import Problem
    ctx = kl.kl_create(0, None)
    try:
        p = Problem(20, 14, 9, g=3, dtype=1, walls=True, dz=1.0 / 9, xybc=True)
        f = make_inputs(20, 14, 9, seed=3, walls=True)
        bufs = [p.upload(f[k]) for k in ("u", "v", "w")]
        g = p.g
        for b in bufs:                               # x, y ghosts: a marker pattern
            pv = p.padded_view(b)
            pv[g:g + p.nz, :, :g] = 7.0
            pv[g:g + p.nz, :, g + p.nx:] = 8.0
            pv[g:g + p.nz, :g, g:g + p.nx] = 9.0
            pv[g:g + p.nz, g + p.ny:, g:g + p.nx] = 10.0
        before = [p.padded_view(b).clone() for b in bufs]
        kl.kl_fill_ghosts(ctx, p.dtype, p.grid, *[b.data_ptr() for b in bufs], None)
        torch.cuda.synchronize()
        for c, (b, b0) in enumerate(zip(bufs, before)):
            pv = p.padded_view(b).cpu().numpy().astype(np.float64)
            b0 = b0.cpu().numpy().astype(np.float64)
            assert np.array_equal(pv[g:g + p.nz], b0[g:g + p.nz])      # interior levels untouched
            odd = c == 2
            for m in range(g):                                          # z planes from own column
                if odd:
                    assert np.array_equal(pv[g - 1 - m], -b0[g + 1 + m])
                    exp_top = np.zeros_like(pv[0]) if m == 0 else -b0[g + p.nz - m]
                    assert np.array_equal(pv[g + p.nz + m], exp_top)
                else:
                    assert np.array_equal(pv[g - 1 - m], b0[g + m])
                    assert np.array_equal(pv[g + p.nz + m], b0[g + p.nz - 1 - m])
    finally:
        kl.kl_destroy(ctx)


@pytest.mark.parametrize("dtype,diff", [(1, 1), (0, 1), (1, 2)])
def test_decomposed_step_matches_whole_grid_oracle(oracle_mod, dtype, diff):
    import torch
    from paper_2303_12374_gb300 import halo, kl
    from paper_2303_12374_gb300.problem import Problem
    NX, NY, NZ, G, px, py = 150, 92, 20, 3, 2, 2
    f = make_inputs(NX, NY, NZ, seed=91, walls=True, var_nu=diff == 2)
    d = halo.Decomposition(NX, NY, NZ, px, py, G)
    ctx = kl.kl_create(0, WISDOM)
    try:
        probs, bufs, outs = {}, {}, {}
        for r in range(d.size):
            b = d.block(r)
            p = Problem(b.nx, b.ny, NZ, g=G, dtype=dtype, walls=True, dx=1.0 / NX, dy=1.0 / NY,
                        dz=1.0 / NZ, nu=1e-3, xybc=True)
            sl = np.s_[:, b.y0:b.y0 + b.ny, b.x0:b.x0 + b.nx]
            keys = ("u", "v", "w", "nu") if diff == 2 else ("u", "v", "w")
            bufs[r] = {k: p.upload(f[k][sl]) for k in keys}
            for k in keys:                            # ghosts must come from the exchange
                pv = p.padded_view(bufs[r][k])
                pv[G:G + NZ, :, :G] = float("nan")
                pv[G:G + NZ, :, G + b.nx:] = float("nan")
                pv[G:G + NZ, :G, :] = float("nan")
                pv[G:G + NZ, G + b.ny:, :] = float("nan")
            outs[r] = [p.empty() for _ in range(3)]
            probs[r] = p
        nf = 4 if diff == 2 else 3
        keys = ("u", "v", "w", "nu")[:nf]
        ex = halo.HaloExchange(d, probs, nf, halo.LocalTransport(), halo.KLPacker(ctx))
        ex.exchange({r: [bufs[r][k].data_ptr() for k in keys] for r in probs})
        op = kl.Op(5, diff, dtype, 0)
        for r, p in probs.items():
            fl = kl.Fields(*[bufs[r][k].data_ptr() for k in ("u", "v", "w")],
                           bufs[r]["nu"].data_ptr() if diff == 2 else None,
                           *[o.data_ptr() for o in outs[r]])
            kl.kl_step(ctx, op, p.grid, fl)
        torch.cuda.synchronize()
        asm = [np.zeros((NZ, NY, NX)) for _ in range(3)]
        for r, p in probs.items():
            b = d.block(r)
            for c in range(3):
                asm[c][:, b.y0:b.y0 + b.ny, b.x0:b.x0 + b.nx] = p.download(outs[r][c])
        p0 = probs[0]
        rin = {k: p0.rounded(f[k]) for k in ("u", "v", "w")}
        ref = oracle_mod.tendencies(rin["u"], rin["v"], rin["w"], adv=5, diff=diff, g=G,
                                    walls=True, dx=1.0 / NX, dy=1.0 / NY, zh=f["zh"], nu=1e-3,
                                    nu_field=p0.rounded(f["nu"]) if diff == 2 else None)
        for a, rr in zip(asm, ref):
            assert np.isfinite(a).all()
            assert rel_err(a, rr) <= TOL[dtype]
    finally:
        kl.kl_destroy(ctx)
