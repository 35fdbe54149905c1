"""kl_step: ghost fill and tendency in one call.  Same tendencies as
kl_fill_ghosts + kl_launch; with a zpack configuration selected, the x ghosts
of interior rows are left as they were (the kernel wraps x itself)."""

from __future__ import annotations

import json
import os

import numpy as np
import pytest

from gpu_cases import TOL, make_inputs, oracle_ref, poison_x_ghosts, rel_err

pytestmark = pytest.mark.gpu

TAGS = {0: "f64", 1: "f32", 2: "bf16"}


def _zpack_wisdom(path, dtype):
    """A wisdom file whose only record selects a zpack configuration."""
    cfg = "zpack:w=2,ly=2,kc=8,ns=8,minb=1" if dtype == 0 else "zpack:w=4,ly=2,kc=8,ns=8,minb=2"
    with open(os.path.join(path, f"tendency_adv5_diff1_{TAGS[dtype]}.wisdom"), "w") as fh:
        fh.write(f'device="NVIDIA GB300" cc=10.3 zbc=1 nx=64 ny=64 nz=32 config="{cfg}" '
                 f'time_us=1.0\n')


def _ghost_masks(p):
    """Boolean masks over the padded box: x ghosts of interior rows, other ghosts."""
    g = p.g
    shape = (p.nz + 2 * g, p.ny + 2 * g, p.nx + 2 * g)
    ghost = np.ones(shape, bool)
    ghost[g:g + p.nz, g:g + p.ny, g:g + p.nx] = False
    xg = np.zeros(shape, bool)
    xg[g:g + p.nz, g:g + p.ny, :g] = True
    xg[g:g + p.nz, g:g + p.ny, g + p.nx:] = True
    return xg, ghost & ~xg


@pytest.mark.parametrize("family", ["zpack", "direct"])
@pytest.mark.parametrize("dtype", [0, 1, 2])
def test_step_equals_fill_then_launch(tmp_path, oracle_mod, family, dtype):
    import torch
    from paper_2303_12374_gb300 import kl
    from paper_2303_12374_gb300.problem import Problem
    nx, ny, nz = 70, 45, 23
    f = make_inputs(nx, ny, nz, seed=17, walls=True)
    if family == "zpack":
        _zpack_wisdom(str(tmp_path), dtype)
    ctx = kl.kl_create(0, str(tmp_path) if family == "zpack" else None)
    try:
        op = kl.Op(5, 1, dtype, 0)
        res = {}
        for mode in ("separate", "step"):
            p = Problem(nx, ny, nz, g=3, dtype=dtype, walls=True, dz=1.0 / nz, nu=1e-3)
            bufs = {k: p.upload(f[k]) for k in ("u", "v", "w")}
            outs = [p.empty() for _ in range(3)]
            fl = kl.Fields(*[bufs[k].data_ptr() for k in ("u", "v", "w")], None,
                           *[o.data_ptr() for o in outs])
            if mode == "separate":
                kl.kl_fill_ghosts(ctx, p.dtype, p.grid, *[bufs[k].data_ptr() for k in "uvw"],
                                  None)
                kl.kl_launch(ctx, op, p.grid, fl)
            else:
                for k in ("u", "v", "w"):
                    poison_x_ghosts(p, bufs[k])
                kl.kl_step(ctx, op, p.grid, fl)
            torch.cuda.synchronize()
            res[mode] = ([p.download(o) for o in outs],
                         {k: p.padded_view(bufs[k]).double().cpu().numpy() for k in "uvw"})
        cfg = json.loads(kl.kl_stats(ctx))["last_config"]
        assert cfg.startswith(family), cfg
        for a, b in zip(res["separate"][0], res["step"][0]):
            assert np.array_equal(a, b)
        rin = {k: p.rounded(f[k]) for k in ("u", "v", "w")}
        ref = oracle_ref(oracle_mod, rin, f["zh"], adv=5, diff=1, walls=True, g=3)
        for a, r in zip(res["step"][0], ref):
            assert rel_err(a, r) <= TOL[dtype]
        # ghosts after the step: y rows and z planes filled; x ghosts of
        # interior rows filled by the full fill, untouched (NaN) under zpack
        xg, other = _ghost_masks(p)
        for k, odd in (("u", False), ("v", False), ("w", True)):
            want = oracle_mod.pad(rin[k], 3, True, odd)
            got = res["step"][1][k]
            assert np.array_equal(got[other], want[other]), k
            if family == "zpack":
                assert np.isnan(got[xg]).all(), k
            else:
                assert np.array_equal(got[xg], want[xg]), k
    finally:
        kl.kl_destroy(ctx)


def test_step_rejects_before_launching():
    from paper_2303_12374_gb300 import kl
    ctx = kl.kl_create(0, None)
    try:
        with pytest.raises(kl.KLError) as e:
            kl.kl_step(ctx, kl.Op(5, 1, 7, 0), kl.Grid(), kl.Fields())
        assert e.value.status == -1
    finally:
        kl.kl_destroy(ctx)
