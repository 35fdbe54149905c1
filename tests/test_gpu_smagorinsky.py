"""kl_smagorinsky on the GPU against the oracle: the eddy viscosity on ragged
and stretched grids in every storage type, the ghost fill of nu it performs,
the chain nu -> variable-nu tendencies (the LES step of Sec. 5.2's diff_uvw),
and sampled levels of the full 1024 x 1024 x 64 stretched workload."""

from __future__ import annotations

import numpy as np
import pytest

from gpu_cases import TOL, make_inputs, rel_err

pytestmark = pytest.mark.gpu

CS = 0.12


@pytest.fixture(scope="module")
def ctx():
    from paper_2303_12374_gb300 import kl
    c = kl.kl_create(0, None)
    yield c
    kl.kl_destroy(c)


def _gpu_nu(ctx, f, *, dtype, walls, g, stretched, fill=True):
    import torch
    from paper_2303_12374_gb300 import kl
    from paper_2303_12374_gb300.problem import Problem
    nz, ny, nx = f["u"].shape
    p = Problem(nx, ny, nz, g=g, dtype=dtype, walls=walls, zh=f["zh"] if stretched else None,
                dz=None if stretched else float(f["zh"][1] - f["zh"][0]), nu=1e-3)
    bufs = {k: p.upload(f[k]) for k in ("u", "v", "w")}
    nu = p.empty()
    nu.fill_(float("nan"))
    kl.kl_fill_ghosts(ctx, p.dtype, p.grid, *[bufs[k].data_ptr() for k in ("u", "v", "w")])
    kl.kl_smagorinsky(ctx, p.dtype, p.grid, CS, *[bufs[k].data_ptr() for k in ("u", "v", "w")],
                      nu.data_ptr(), fill)
    torch.cuda.synchronize()
    rin = {k: p.rounded(f[k]) for k in ("u", "v", "w")}
    return p, bufs, nu, rin


def _oracle_nu(oracle_mod, rin, zh, *, walls, g, levels=None):
    nz, ny, nx = rin["u"].shape
    return oracle_mod.smagorinsky(rin["u"], rin["v"], rin["w"], g=g, walls=walls, dx=1.0 / nx,
                                  dy=1.0 / ny, zh=zh, cs=CS, levels=levels)


CASES = [
    # nx, ny, nz, g, walls, stretch
    (37, 21, 17, 3, True, 2.0),
    (40, 24, 10, 1, False, 0.0),
    (13, 11, 9, 1, True, 0.0),
    (33, 9, 40, 3, False, 1.5),
    (64, 34, 40, 3, True, 2.0),     # two rows per thread, ragged in y, several level chunks
    (36, 10, 7, 1, False, 0.0),     # two rows per thread, g = 1
]


@pytest.mark.parametrize("dtype", [0, 1, 2, 3])
@pytest.mark.parametrize("case", CASES)
def test_viscosity_parity(ctx, oracle_mod, dtype, case):
    nx, ny, nz, g, walls, stretch = case
    f = make_inputs(nx, ny, nz, seed=nx + 7 * nz, walls=walls, stretch=stretch)
    p, bufs, nu, rin = _gpu_nu(ctx, f, dtype=dtype, walls=walls, g=g, stretched=stretch > 0)
    ref = _oracle_nu(oracle_mod, rin, f["zh"], walls=walls, g=g)
    got = p.download(nu)
    assert np.isfinite(got).all()
    assert rel_err(got, ref) <= TOL[dtype], (case, rel_err(got, ref))
    assert (got >= 0).all()
    # the ghosts of nu follow the fill rules of its interior (bit for bit)
    pv = p.padded_view(nu).double().cpu().numpy()
    assert np.array_equal(pv, oracle_mod.pad(got, g, walls, False))


def test_interior_only_leaves_ghosts(ctx, oracle_mod):
    import torch
    f = make_inputs(20, 16, 8, seed=3, walls=True)
    p, bufs, nu, rin = _gpu_nu(ctx, f, dtype=1, walls=True, g=1, stretched=False, fill=False)
    pv = p.padded_view(nu)
    assert torch.isnan(pv[0]).all() and torch.isnan(pv[:, :, 0]).all()
    assert not torch.isnan(p.view(nu)).any()


@pytest.mark.parametrize("dtype", [0, 1])
def test_les_chain(ctx, oracle_mod, dtype):
    """nu from the velocities, then the 5th-order advection + variable-nu
    diffusion tendencies with that nu, against the same chain in the oracle."""
    import torch
    from paper_2303_12374_gb300 import kl
    nx, ny, nz = 70, 45, 23
    f = make_inputs(nx, ny, nz, seed=41, walls=True, stretch=2.0)
    p, bufs, nu, rin = _gpu_nu(ctx, f, dtype=dtype, walls=True, g=3, stretched=True)
    outs = [p.empty() for _ in range(3)]
    fl = kl.Fields(*[bufs[k].data_ptr() for k in ("u", "v", "w")], nu.data_ptr(),
                   *[o.data_ptr() for o in outs])
    kl.kl_launch(ctx, kl.Op(5, 2, dtype, 0), p.grid, fl)
    torch.cuda.synchronize()
    nu_ref = _oracle_nu(oracle_mod, rin, f["zh"], walls=True, g=3)
    ref = oracle_mod.tendencies(rin["u"], rin["v"], rin["w"], adv=5, diff=2, g=3, walls=True,
                                dx=1.0 / nx, dy=1.0 / ny, zh=f["zh"], nu_field=nu_ref)
    for o, r in zip(outs, ref):
        assert rel_err(p.download(o), r) <= TOL[dtype]


def test_argument_errors(ctx):
    from paper_2303_12374_gb300 import kl
    from paper_2303_12374_gb300.problem import Problem
    p = Problem(8, 8, 8, g=1, dtype="f32", walls=True, dz=1 / 8, nu=1e-3)
    a, b = p.empty(), p.empty()
    for cs, nu, dt in ((-1.0, b, 1), (float("nan"), b, 1), (0.1, a, 1), (0.1, b, 7)):
        with pytest.raises(kl.KLError) as e:
            kl.kl_smagorinsky(ctx, dt, p.grid, cs, a.data_ptr(), a.data_ptr(), a.data_ptr(),
                              nu.data_ptr())
        assert e.value.status == -1


def test_les_1024x1024x64_sampled_levels(ctx, oracle_mod):
    from paper_2303_12374_gb300 import synth
    spec = synth.WORKLOADS["les1024x1024x64_stretched_varnu"]
    zh = synth.zfaces(64, spec["lz"], spec["stretch"])
    f = synth.velocity_fields(1024, 1024, 64, seed=synth.seed_of(4), walls=True, zh=zh)
    p, bufs, nu, rin = _gpu_nu(ctx, f, dtype=1, walls=True, g=3, stretched=True)
    got = p.download(nu)
    slabs = ((0, 2), (31, 33), (62, 64))
    ref = np.concatenate([_oracle_nu(oracle_mod, rin, zh, walls=True, g=3, levels=s) for s in slabs])
    assert rel_err(np.concatenate([got[a:b] for a, b in slabs]), ref) <= TOL[1]


@pytest.mark.parametrize("dtype", [0, 1])
def test_cs_creates_no_table_and_scales_nu_by_cs_squared(dtype):
    """cs is a kernel argument: one delta_k^2 table per vertical grid, however
    many values of cs a caller uses, and nu scales as cs^2."""
    import json

    import torch
    from paper_2303_12374_gb300 import kl
    from paper_2303_12374_gb300.problem import Problem
    f = make_inputs(40, 24, 12, seed=31, walls=True, stretch=2.0)
    c = kl.kl_create(0, None)
    try:
        p = Problem(40, 24, 12, g=3, dtype=dtype, walls=True, zh=f["zh"], nu=1e-3)
        bufs = [p.upload(f[k]) for k in ("u", "v", "w")]
        kl.kl_fill_ghosts(c, p.dtype, p.grid, *[b.data_ptr() for b in bufs])
        res = []
        for cs in (0.1, 0.17, 0.2):
            nu = p.empty()
            kl.kl_smagorinsky(c, p.dtype, p.grid, cs, *[b.data_ptr() for b in bufs], nu.data_ptr(), False)
            torch.cuda.synchronize()
            res.append(p.download(nu))
        assert json.loads(kl.kl_stats(c))["tables"] == 1
        tol = 1e-14 if dtype == 0 else 1e-6
        for cs, r in zip((0.17, 0.2), res[1:]):
            assert np.abs(r - res[0] * (cs / 0.1) ** 2).max() <= tol * np.abs(r).max()
    finally:
        kl.kl_destroy(c)


def test_two_row_kernel_agrees_with_the_one_row_kernel(ctx):
    """f32 with an even ny runs two rows per thread, an odd ny one row per
    thread.  The same values enter the same expressions; the compiler may
    contract different products into FMAs in the two instances, so on the
    rows both grids share (away from the y boundary, whose periodic
    neighbours differ) the viscosities agree to a few units in the last place
    of f32."""
    import torch
    from paper_2303_12374_gb300 import kl
    from paper_2303_12374_gb300.problem import Problem
    nx, nz = 64, 40
    f = make_inputs(nx, 25, nz, seed=31, walls=True, stretch=2.0)
    res = []
    for ny in (25, 24):
        p = Problem(nx, ny, nz, g=3, dtype=1, walls=True, zh=f["zh"], dx=1.0 / nx, dy=1.0 / 25,
                    nu=1e-3)
        bufs = [p.upload(f[k][:, :ny, :]) for k in ("u", "v", "w")]
        nu = p.empty()
        kl.kl_fill_ghosts(ctx, p.dtype, p.grid, *[b.data_ptr() for b in bufs])
        kl.kl_smagorinsky(ctx, p.dtype, p.grid, CS, *[b.data_ptr() for b in bufs], nu.data_ptr(),
                          False)
        torch.cuda.synchronize()
        res.append(p.download(nu))
    a, b = res[0][:, 1:23, :], res[1][:, 1:23, :]
    assert np.abs(a - b).max() <= 4 * 2.0 ** -24 * np.abs(a).max()
