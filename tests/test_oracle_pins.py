"""Pins of the FP64 oracle against facts fixed by mathematics, not by itself.

Each test names what it pins:
  * constant fields give exactly zero tendency (every scheme, every BC);
  * convergence order 2 of every term against exact symbolic tendencies
    (periodic, walls, stretched z, constant and variable viscosity);
  * order 5 (upwind F5), 6 (centred I6) and 2 (centred I2) of the
    interpolations when the advecting velocity is constant, on every axis and
    both flow directions;
  * the exact Fourier symbol of the textbook 5th-order upwind face value
    (Wicker & Skamarock 2002), to rounding;
  * linearity of diffusion, quadratic homogeneity of advection (bitwise);
  * discrete conservation of momentum (periodic and wall-bounded, dz-weighted);
  * discrete energy conservation of the 2nd-order scheme on a divergence-free
    field, and energy dissipation of the upwind 5th-order scheme;
  * stress-divergence == nu * Laplacian for constant nu and zero divergence;
  * x<->y symmetry and translation invariance;
  * ghost filling == numpy.pad ('wrap', 'symmetric', odd 'reflect');
  * vertical profiles against their defining relations.
"""

from __future__ import annotations

import math

import numpy as np
import pytest

from paper_2303_12374_gb300 import synth

analytic = pytest.importorskip("analytic")
sp = analytic.sp


def run(oracle_mod, f, *, adv, diff, g=3, walls=False, nu=1e-3, nu_field=None):
    nz, ny, nx = f["u"].shape
    return oracle_mod.tendencies(f["u"], f["v"], f["w"], adv=adv, diff=diff, g=g, walls=walls,
                                 dx=1.0 / nx, dy=1.0 / ny, zh=f["zh"], nu=nu,
                                 nu_field=nu_field)


# ------------------------------------------------------------ constant fields

@pytest.mark.parametrize("adv", [0, 2, 5, 6])
@pytest.mark.parametrize("diff", [0, 1, 2])
@pytest.mark.parametrize("walls", [False, True])
def test_constant_fields_give_exact_zero(oracle_mod, adv, diff, walls):
    nx, ny, nz = 9, 7, 8
    zh = synth.zfaces(nz, 1.0, stretch=2.0 if walls else 0.0)
    f = {"u": np.full((nz, ny, nx), 0.7), "v": np.full((nz, ny, nx), -1.3),
         "w": np.full((nz, ny, nx), 0.0 if walls else 0.45), "zh": zh}
    nuf = synth.velocity_fields(nx, ny, nz, seed=5, walls=walls, nu0=1e-3)["nu"]
    ut, vt, wt = run(oracle_mod, f, adv=adv, diff=diff, walls=walls, nu_field=nuf)
    for t in (ut, vt, wt):
        assert np.all(t == 0.0)


# ------------------------------------------------------------- convergence 2

SPEC_U = [(1.0, 1, 2, 1, 0.3), (0.5, 2, -1, 1, 1.1)]
SPEC_V = [(0.8, 1, 1, 2, 2.0), (-0.4, 2, 1, 1, 0.2)]
SPEC_W = [(0.6, 1, -1, 1, 0.7), (0.3, 1, 2, 2, 2.5)]


def _exact(walls, lz, adv, diff, nu, nu_expr=None):
    u = analytic.mode_sum(SPEC_U, walls, lz, "even")
    v = analytic.mode_sum(SPEC_V, walls, lz, "even")
    w = analytic.mode_sum(SPEC_W, walls, lz, "odd")
    return (u, v, w), analytic.exact_tendencies(u, v, w, adv=adv, diff=diff, nu=nu,
                                                nu_expr=nu_expr)


def _conv_errors(oracle_mod, *, adv, diff, walls, stretch, ns, nu=0.05, var_nu=False):
    """Max relative errors per grid: (away from the wall-adjacent levels, at them)."""
    lz = 1.0
    nu_expr = None
    if var_nu:
        nu_expr = nu * (1.0 + 0.5 * sp.sin(2 * sp.pi * (analytic.X + analytic.Y)) *
                        (sp.cos(sp.pi * analytic.Z / lz) if walls else
                         sp.cos(2 * sp.pi * analytic.Z / lz)))
    vel, ex = _exact(walls, lz, adv != 0, diff, nu, nu_expr)
    inner, edge = [], []
    for n in ns:
        zh = synth.zfaces(n, lz, stretch)
        pts = analytic.staggered_points(n, n, zh)
        f = {name: analytic.evaluate(e, *pts[name]) for name, e in zip("uvw", vel)}
        f["zh"] = zh
        nuf = analytic.evaluate(nu_expr, *pts["c"]) if var_nu else None
        got = run(oracle_mod, f, adv=adv, diff=diff, walls=walls, nu=nu, nu_field=nuf)
        ei = eb = 0.0
        for name, t, exe in zip("uvw", got, ex):
            ref = analytic.evaluate(exe, *pts[name])
            scale = np.abs(ref).max()
            err = np.abs(t - ref).max(axis=(1, 2)) / scale
            if walls and name == "w":
                err = err[1:]
            ei = max(ei, err[1:-1].max())
            eb = max(eb, err[0], err[-1])
        inner.append(ei)
        edge.append(eb)
    return np.array(inner), np.array(edge)


@pytest.mark.parametrize("adv,diff,walls,stretch,var_nu", [
    (2, 0, False, 0.0, False),
    (5, 0, False, 0.0, False),
    (2, 1, False, 0.0, False),
    (5, 1, True, 0.0, False),
    (5, 1, True, 2.0, False),
    (0, 1, True, 2.0, False),
    (0, 2, False, 0.0, True),
    (0, 2, True, 2.0, True),
    (5, 2, True, 2.0, True),
])
def test_convergence_order_two(oracle_mod, adv, diff, walls, stretch, var_nu):
    """Order 2 everywhere on uniform grids; on a stretched grid order 2 away from
    the walls and order >= 1 in the wall-adjacent cell (the 3-point flux form's
    upper-face gradient sits (dz1-dz0)/4 off the face there, with no cancelling
    error at the wall face)."""
    ns = [16, 32, 64] if stretch == 0.0 else [32, 64, 128]
    inner, edge = _conv_errors(oracle_mod, adv=adv, diff=diff, walls=walls, stretch=stretch,
                               ns=ns, var_nu=var_nu)
    hs = [1.0 / n for n in ns]
    s = analytic.slope(hs, inner)
    assert 1.85 < s < 2.4, (inner, s)
    assert inner[-1] < 2e-2
    se = analytic.slope(hs, edge)
    if stretch == 0.0:
        assert 1.85 < se < 2.4, (edge, se)
    else:
        assert se > 0.9, (edge, se)
        assert edge[-1] < 2e-2


# --------------------------------------------- interpolation order, const U

def _const_velocity_case(oracle_mod, n, axis, adv, vel0):
    """Advect smooth profiles along `axis` with a constant velocity vel0."""
    small = 4
    shape = [small, small, small]
    shape[axis] = n
    nx, ny, nz = shape
    zh = synth.zfaces(nz, 1.0)
    pts = analytic.staggered_points(nx, ny, zh)
    prof = lambda s: np.sin(analytic.TWO_PI * s + 0.4) + 0.3 * np.cos(2 * analytic.TWO_PI * s)
    dprof = lambda s: analytic.TWO_PI * (np.cos(analytic.TWO_PI * s + 0.4)
                                         - 0.6 * np.sin(2 * analytic.TWO_PI * s))
    names = ["u", "v", "w"]
    carrier = names[axis]
    f = {}
    exact = {}
    for name in names:
        xs, ys, zs = pts[name]
        coord = (xs, ys, zs)[axis]
        zz, yy, xx = np.meshgrid(zs, ys, xs, indexing="ij")
        cc = (xx, yy, zz)[axis]
        if name == carrier:
            f[name] = np.full((nz, ny, nx), vel0)
            exact[name] = np.zeros((nz, ny, nx))
        else:
            f[name] = prof(cc)
            exact[name] = -vel0 * dprof(cc)
        del coord
    f["zh"] = zh
    got = oracle_mod.tendencies(f["u"], f["v"], f["w"], adv=adv, diff=0, g=3, walls=False,
                                dx=1.0 / nx, dy=1.0 / ny, zh=zh)
    err = 0.0
    for name, t in zip(names, got):
        if name == carrier:
            assert np.all(t == 0.0)
            continue
        err = max(err, np.abs(t - exact[name]).max() / np.abs(exact[name]).max())
    return err


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("vel0", [1.3, -0.7])
@pytest.mark.parametrize("adv,order", [(2, 2.0), (5, 5.0), (6, 6.0)])
def test_interpolation_order_with_constant_velocity(oracle_mod, axis, vel0, adv, order):
    ns = [16, 32, 64, 128] if adv != 2 else [32, 64, 128]
    errs = [_const_velocity_case(oracle_mod, n, axis, adv, vel0) for n in ns]
    s = analytic.slope([1.0 / n for n in ns], errs)
    assert abs(s - order) < 0.25, (errs, s)


@pytest.mark.parametrize("kappa", [1, 3, 7])
@pytest.mark.parametrize("vel0", [0.9, -1.7])
def test_fourier_symbol_of_upwind5(oracle_mod, kappa, vel0):
    """v = A sin(2 pi kappa x + psi) advected by constant u: vt equals the exact symbol."""
    nx, ny, nz = 32, 4, 4
    dx = 1.0 / nx
    theta = 2 * math.pi * kappa * dx
    amp, psi = 1.4, 0.37
    i = np.arange(nx)
    vrow = amp * np.sin(theta * (i + 0.5) + psi)
    f = {"u": np.full((nz, ny, nx), vel0), "v": np.broadcast_to(vrow, (nz, ny, nx)).copy(),
         "w": np.zeros((nz, ny, nx)), "zh": synth.zfaces(nz)}
    _, vt, _ = oracle_mod.tendencies(f["u"], f["v"], f["w"], adv=5, diff=0, g=3, walls=False,
                                     dx=dx, dy=1.0 / ny, zh=f["zh"])
    S = analytic.fourier_symbol_upwind5(theta, vel0 > 0)
    expect = -(vel0 / dx) * np.imag(amp * np.exp(1j * psi) * np.exp(1j * theta * (i + 0.5)) * S)
    assert np.abs(vt[0, 0] - expect).max() <= 1e-13 * np.abs(expect).max() + 1e-12
    assert np.all(vt == vt[0, 0])


# ------------------------------------------------------ algebraic properties

def _fields(n=(12, 10, 8), seed=11, walls=False, stretch=0.0, nu0=None):
    nx, ny, nz = n
    zh = synth.zfaces(nz, 1.0, stretch)
    return synth.velocity_fields(nx, ny, nz, seed=seed, walls=walls, zh=zh, nu0=nu0)


@pytest.mark.parametrize("diff", [1, 2])
@pytest.mark.parametrize("walls", [False, True])
def test_diffusion_is_linear(oracle_mod, diff, walls):
    f = _fields(walls=walls, stretch=2.0 if walls else 0.0, nu0=1e-3)
    h = _fields(seed=12, walls=walls, stretch=2.0 if walls else 0.0)
    a, b = 0.75, -1.9
    comb = {k: a * f[k] + b * h[k] for k in "uvw"}
    comb["zh"] = f["zh"]
    tf = run(oracle_mod, f, adv=0, diff=diff, walls=walls, nu_field=f["nu"])
    th = run(oracle_mod, h, adv=0, diff=diff, walls=walls, nu_field=f["nu"])
    tc = run(oracle_mod, comb, adv=0, diff=diff, walls=walls, nu_field=f["nu"])
    for x, y, z in zip(tf, th, tc):
        ref = a * x + b * y
        assert np.abs(z - ref).max() <= 1e-13 * np.abs(ref).max()
    f2 = {k: 2.0 * f[k] for k in "uvw"}
    f2["zh"] = f["zh"]
    t2 = run(oracle_mod, f2, adv=0, diff=diff, walls=walls, nu_field=f["nu"])
    for x, y in zip(tf, t2):
        assert np.array_equal(2.0 * x, y)


@pytest.mark.parametrize("adv", [2, 5])
def test_advection_is_quadratic_bitwise(oracle_mod, adv):
    f = _fields(walls=True, stretch=2.0)
    f2 = {k: 2.0 * f[k] for k in "uvw"}
    f2["zh"] = f["zh"]
    t1 = run(oracle_mod, f, adv=adv, diff=0, walls=True)
    t2 = run(oracle_mod, f2, adv=adv, diff=0, walls=True)
    for x, y in zip(t1, t2):
        assert np.array_equal(4.0 * x, y)


@pytest.mark.parametrize("adv,diff", [(2, 1), (5, 1), (5, 2), (0, 2)])
def test_momentum_conservation_periodic(oracle_mod, adv, diff):
    f = _fields(nu0=1e-3)
    ts = run(oracle_mod, f, adv=adv, diff=diff, nu_field=f["nu"])
    for t in ts:
        assert abs(t.sum()) <= 1e-13 * np.abs(t).sum()


@pytest.mark.parametrize("adv,diff", [(5, 1), (5, 2), (2, 1)])
def test_momentum_conservation_walls_dz_weighted(oracle_mod, adv, diff):
    f = _fields(walls=True, stretch=2.0, nu0=1e-3)
    dz, _ = oracle_mod.zprofile(8, 3, True, f["zh"])
    ut, vt, _ = run(oracle_mod, f, adv=adv, diff=diff, walls=True, nu_field=f["nu"])
    wgt = dz[3:3 + 8][:, None, None]
    for t in (ut, vt):
        assert abs((t * wgt).sum()) <= 1e-13 * np.abs(t * wgt).sum()
        # without the dz weight the sum is not zero on a stretched grid
        assert abs(t.sum()) > 1e-9 * np.abs(t).sum()


@pytest.mark.parametrize("adv,diff", [(5, 1), (2, 1), (5, 2), (0, 1)])
def test_momentum_conservation_periodic_stretched(oracle_mod, adv, diff):
    """Periodic z on a non-uniform grid: the flux differences telescope for any
    spacing, so sum ut dz_k, sum vt dz_k and sum wt dzh_k vanish to rounding
    (the metric each component's divergence divides by is the right one)."""
    f = _fields(n=(10, 8, 12), walls=False, stretch=2.0, nu0=1e-3)
    dz, dzh = oracle_mod.zprofile(12, 3, False, f["zh"])
    ut, vt, wt = run(oracle_mod, f, adv=adv, diff=diff, walls=False, nu_field=f["nu"])
    for t, wgt in ((ut, dz), (vt, dz), (wt, dzh)):
        tw = t * wgt[3:15][:, None, None]
        assert abs(tw.sum()) <= 1e-13 * np.abs(tw).sum()


def divergence_free(n=(16, 16, 16), seed=3):
    """C-grid velocity = discrete curl of random edge potentials (div = 0 to rounding)."""
    nx, ny, nz = n
    rng = np.random.default_rng(seed)
    ax, ay, az = (rng.standard_normal((nz, ny, nx)) / nx for _ in range(3))
    dx, dy, dz = 1.0 / nx, 1.0 / ny, 1.0 / nz
    nxt = lambda a, axis: np.roll(a, -1, axis=axis)  # a(i+1) along axis (0=k, 1=j, 2=i)
    u = (nxt(az, 1) - az) / dy - (nxt(ay, 0) - ay) / dz
    v = (nxt(ax, 0) - ax) / dz - (nxt(az, 2) - az) / dx
    w = (nxt(ay, 2) - ay) / dx - (nxt(ax, 1) - ax) / dy
    div = (nxt(u, 2) - u) / dx + (nxt(v, 1) - v) / dy + (nxt(w, 0) - w) / dz
    assert np.abs(div).max() < 1e-10 * np.abs(u).max() * nx
    return {"u": u, "v": v, "w": w, "zh": synth.zfaces(nz)}


def test_energy_conservation_of_second_order_scheme(oracle_mod):
    f = divergence_free()
    ut, vt, wt = run(oracle_mod, f, adv=2, diff=0)
    terms = f["u"] * ut + f["v"] * vt + f["w"] * wt
    assert abs(terms.sum()) <= 1e-12 * np.abs(terms).sum()


def test_upwind5_dissipates_energy(oracle_mod):
    f = divergence_free()
    ut, vt, wt = run(oracle_mod, f, adv=5, diff=0)
    terms = f["u"] * ut + f["v"] * vt + f["w"] * wt
    assert terms.sum() < -1e-3 * np.abs(terms).sum()
    # the centred 6th-order interpolation alone is not dissipative to this degree
    u6, v6, w6 = run(oracle_mod, f, adv=6, diff=0)
    t6 = f["u"] * u6 + f["v"] * v6 + f["w"] * w6
    assert abs(t6.sum()) < abs(terms.sum())


def test_stress_divergence_equals_laplacian_when_divergence_free(oracle_mod):
    f = divergence_free()
    nu0 = 3e-3
    nuf = np.full(f["u"].shape, nu0)
    t2 = run(oracle_mod, f, adv=0, diff=2, nu_field=nuf)
    t1 = run(oracle_mod, f, adv=0, diff=1, nu=nu0)
    for a, b in zip(t1, t2):
        assert np.abs(a - b).max() <= 1e-11 * np.abs(a).max()


@pytest.mark.parametrize("adv,diff", [(5, 1), (2, 2)])
def test_x_y_swap_symmetry(oracle_mod, adv, diff):
    f = _fields(n=(10, 10, 6), nu0=1e-3)
    sw = lambda a: np.ascontiguousarray(a.transpose(0, 2, 1))
    g = {"u": sw(f["v"]), "v": sw(f["u"]), "w": sw(f["w"]), "zh": f["zh"]}
    ut, vt, wt = run(oracle_mod, f, adv=adv, diff=diff, nu_field=f["nu"])
    us, vs, ws = run(oracle_mod, g, adv=adv, diff=diff, nu_field=sw(f["nu"]))
    for a, b in ((us, sw(vt)), (vs, sw(ut)), (ws, sw(wt))):
        assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_translation_invariance_bitwise(oracle_mod, axis):
    f = _fields(nu0=1e-3)
    r = lambda a: np.roll(a, 1, axis=axis)
    g = {k: r(f[k]) for k in ("u", "v", "w")}
    g["zh"] = f["zh"]
    t = run(oracle_mod, f, adv=5, diff=2, nu_field=f["nu"])
    s = run(oracle_mod, g, adv=5, diff=2, nu_field=r(f["nu"]))
    for a, b in zip(t, s):
        assert np.array_equal(r(a), b)


# ------------------------------------------------------------- ghost fill

@pytest.mark.parametrize("g", [1, 3])
def test_ghost_fill_matches_numpy_pad(oracle_mod, g):
    rng = np.random.default_rng(0)
    a = rng.standard_normal((6, 5, 7))
    per = oracle_mod.pad(a, g, walls=False, odd=False)
    assert np.array_equal(per, np.pad(a, g, mode="wrap"))
    assert np.array_equal(oracle_mod.pad(a, g, walls=False, odd=True), per)
    even = oracle_mod.pad(a, g, walls=True, odd=False)
    ref = np.pad(np.pad(a, ((0, 0), (g, g), (g, g)), mode="wrap"), ((g, g), (0, 0), (0, 0)),
                 mode="symmetric")
    assert np.array_equal(even, ref)
    w = a.copy()
    w[0] = 0.0
    odd = oracle_mod.pad(w, g, walls=True, odd=True)
    ext = np.concatenate([w, np.zeros((1,) + w.shape[1:])], axis=0)  # w(0..nz), w(nz)=0
    ext = np.pad(ext, ((0, 0), (g, g), (g, g)), mode="wrap")
    lo = -ext[1:g + 1][::-1]
    hi = -ext[-1 - g:-1][::-1]
    ref = np.concatenate([lo, ext, hi[:-1]], axis=0)  # ext already holds w(nz) = 0
    assert np.array_equal(odd, ref)


def test_vertical_profiles(oracle_mod):
    nz, g = 16, 3
    zh = synth.zfaces(nz, 0.5, stretch=2.0)
    dz, dzh = oracle_mod.zprofile(nz, g, True, zh)
    assert np.allclose(dz[g:g + nz], np.diff(zh), rtol=0, atol=1e-15)
    assert abs(dz[g:g + nz].sum() - 0.5) < 1e-14
    # dzh is the midpoint spacing: (dz_{k-1} + dz_k)/2
    assert np.allclose(dzh[1:], 0.5 * (dz[:-1] + dz[1:]), rtol=1e-13, atol=0)
    # walls mirror the grid
    assert np.allclose(dz[:g], dz[g:2 * g][::-1], rtol=1e-13)
    assert np.allclose(dz[g + nz:], dz[nz:g + nz][::-1], rtol=1e-13)
    u = synth.zfaces(nz, 1.0)
    dzu, dzhu = oracle_mod.zprofile(nz, g, False, u)
    assert np.allclose(dzu, 1.0 / nz, rtol=1e-13) and np.allclose(dzhu, 1.0 / nz, rtol=1e-13)


def test_diag_definitions(oracle_mod):
    rng = np.random.default_rng(4)
    t = rng.standard_normal(1000)
    r = rng.standard_normal(1000)
    d = oracle_mod.diag(t, r)
    assert d[0] == np.abs(t - r).max() and d[2] == np.abs(r).max()
    assert math.isclose(d[1], math.sqrt(np.mean((t - r) ** 2)), rel_tol=1e-14)
    assert math.isclose(d[4], math.fsum(t), rel_tol=1e-12)
