"""Shared helpers of the GPU tests: run one case through the C ABI and the
oracle on identical seeded inputs, and compare element by element.

Tolerances (max |t - t_ref| / max |t_ref| per tendency, interior points):
  f64: 1e-12; f32: 1e-5; bf16 and f16 storage with f32 compute: the output
  rounding bound 2^-8 (bf16) or 2^-11 (f16) plus 1e-5 for the f32 arithmetic.
The reference is the FP64 oracle run on the inputs rounded to the storage
type, so the comparison measures the kernel, not the input rounding.
"""

from __future__ import annotations

import numpy as np

TOL = {0: 1e-12, 1: 1e-5, 2: 2.0 ** -8 + 1e-5, 3: 2.0 ** -11 + 1e-5}


def make_inputs(nx, ny, nz, *, seed, walls, stretch=0.0, lz=1.0, var_nu=False):
    from paper_2303_12374_gb300 import synth
    zh = synth.zfaces(nz, lz, stretch)
    return synth.velocity_fields(nx, ny, nz, seed=seed, walls=walls, zh=zh,
                                 nu0=1e-3 if var_nu else None)


def poison_x_ghosts(p, buf):
    """NaN into the x ghosts of interior rows of interior levels (the cells a
    kernel that wraps x itself must never read)."""
    g = p.g
    pv = p.padded_view(buf)
    pv[g:g + p.nz, g:g + p.ny, :g] = float("nan")
    pv[g:g + p.nz, g:g + p.ny, g + p.nx:] = float("nan")


def run_gpu(ctx, f, *, adv, diff, dtype, walls, g, config=None, nu=1e-3, stretched=False,
            accumulate=False, t0=None, poison_x=False, step=False, out_f32=False):
    """Fill ghosts + tendency through the C ABI; returns (prob, rounded inputs, outputs).

    poison_x: NaN into the x ghosts of interior rows after the fill (before the
    launch); step: one kl_step call (its own fill) instead of fill + launch;
    out_f32: f32 tendency buffers (16-bit storage)."""
    import torch
    from paper_2303_12374_gb300 import kl
    from paper_2303_12374_gb300.problem import Problem
    nz, ny, nx = f["u"].shape
    zh = f["zh"] if stretched else None
    dz = None if stretched else float(f["zh"][1] - f["zh"][0])
    p = Problem(nx, ny, nz, g=g, dtype=dtype, walls=walls, zh=zh, dz=dz, nu=nu)
    bufs = {k: p.upload(f[k]) for k in ("u", "v", "w")}
    if diff == 2:
        bufs["nu"] = p.upload(f["nu"])
    outs = {}
    odt = torch.float32 if out_f32 else None
    for k in ("ut", "vt", "wt"):
        outs[k] = p.upload(t0[k], dtype=odt) if t0 is not None else p.empty(odt)
    if not step:
        kl.kl_fill_ghosts(ctx, p.dtype, p.grid, bufs["u"].data_ptr(), bufs["v"].data_ptr(),
                          bufs["w"].data_ptr(), bufs["nu"].data_ptr() if diff == 2 else None)
    if poison_x:
        for k in ("u", "v", "w"):
            poison_x_ghosts(p, bufs[k])
    op = kl.Op(adv, diff, p.dtype, 1 if accumulate else 0, 1 if out_f32 else 0)
    fl = kl.Fields(bufs["u"].data_ptr(), bufs["v"].data_ptr(), bufs["w"].data_ptr(),
                   bufs["nu"].data_ptr() if diff == 2 else None, outs["ut"].data_ptr(),
                   outs["vt"].data_ptr(), outs["wt"].data_ptr())
    if step:
        assert config is None
        kl.kl_step(ctx, op, p.grid, fl)
    elif config is None:
        kl.kl_launch(ctx, op, p.grid, fl)
    else:
        kl.kl_launch_with_config(ctx, op, config, p.grid, fl)
    torch.cuda.synchronize()
    rin = {k: p.rounded(f[k]) for k in ("u", "v", "w")}
    if diff == 2:
        rin["nu"] = p.rounded(f["nu"])
    return p, bufs, outs, rin


def oracle_ref(oracle_mod, rin, zh, *, adv, diff, walls, g, nu=1e-3, levels=None):
    nz, ny, nx = rin["u"].shape
    return oracle_mod.tendencies(rin["u"], rin["v"], rin["w"], adv=adv, diff=diff, g=g,
                                 walls=walls, dx=1.0 / nx, dy=1.0 / ny, zh=zh, nu=nu,
                                 nu_field=rin.get("nu"), levels=levels)


def rel_err(got, ref):
    scale = np.abs(ref).max()
    return float(np.abs(got - ref).max() / scale) if scale > 0 else float(np.abs(got).max())
