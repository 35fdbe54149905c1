"""The smallest grids the layout allows, through every family of the tunable
space: three points along x or y (as many as the ghost width), four levels
between free-slip walls (the least with three ghost planes), three levels
periodic in z.  Tiles then hold a few columns or rows, a z chunk or a
persistent CTA's range holds a few levels, and most of a TMA box lies
outside the grid.  The tendencies must equal the oracle's."""

from __future__ import annotations

import pytest

from gpu_cases import TOL, make_inputs, oracle_ref, rel_err, run_gpu

pytestmark = pytest.mark.gpu

SIZES = [
    # nx, ny, nz, walls
    (3, 3, 4, True),
    (5, 4, 3, False),
    (64, 3, 4, True),
    (70, 5, 5, False),     # the x halo wraps inside one zpack tile
    (3, 70, 4, True),
]

CONFIGS = [
    "default",
    "direct:bx=32,by=4,bz=2,tx=2,tz=2,ux=1,uz=1,cx=1,cz=1,perm=ZXY,minb=2",
    "zmarch:bx=32,by=4,px=1,py=2,kc=8,ns=8,minb=1",
    "zpack:w=2,ly=2,kc=4,ns=8,minb=1",
    "zpack:w=2,ly=2,kc=4,ns=6,minb=1",
    "zpack:w=4,ly=3,kc=4,ns=6,minb=1,pe=1",
    "zpack:w=8,ly=4,kc=32,ns=6,minb=1,pe=2",
    "zpack:w=2,ly=2,kc=4,ns=7,minb=1,yx=2",
    "zpack:w=2,ly=2,kc=4,ns=8,minb=1,cs=1",
]


@pytest.fixture(scope="module")
def ctx():
    from paper_2303_12374_gb300 import kl
    c = kl.kl_create(0, None)
    yield c
    kl.kl_destroy(c)


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("size", SIZES)
@pytest.mark.parametrize("diff", [1, 2])
def test_smallest_grids_every_family(ctx, oracle_mod, dtype, size, diff):
    from paper_2303_12374_gb300 import kl
    nx, ny, nz, walls = size
    f = make_inputs(nx, ny, nz, seed=nx * 100 + ny + nz, walls=walls, stretch=2.0 if walls else 0.0,
                    var_nu=diff == 2)
    ran = 0
    for cfg in CONFIGS:
        try:
            kl.kl_config_normalize(kl.Op(5, diff, dtype, 0), cfg)
        except kl.KLError:
            continue          # outside the space for this op (shared memory, nu, cs)
        p, _, outs, rin = run_gpu(ctx, f, adv=5, diff=diff, dtype=dtype, walls=walls, g=3,
                                  stretched=walls, config=cfg)
        ref = oracle_ref(oracle_mod, rin, f["zh"], adv=5, diff=diff, walls=walls, g=3)
        for name, r in zip(("ut", "vt", "wt"), ref):
            e = rel_err(p.download(outs[name]), r)
            assert e <= TOL[dtype], (cfg, name, e)
        ran += 1
    assert ran >= 4
