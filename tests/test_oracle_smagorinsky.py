"""Pins of the oracle's Smagorinsky viscosity, nu = (cs delta)^2 sqrt(2 S_ij S_ij).

- A linear velocity field u_i = G_ij x_j on a stretched grid has the constant
  strain S = (G + G^T)/2, and every difference of the C-grid discretisation is
  exact for it.  So nu must equal (cs delta_k)^2 sqrt(2 sum S_ij^2) level by
  level, to rounding.  A random G exercises every term: a dropped or
  transposed term, a wrong factor or a shifted index fails.
- A rotation (antisymmetric G) has no strain: nu = 0.
- nu scales with cs^2 and is unchanged by a constant velocity.
- For a smooth periodic field, nu^2 / (cs delta)^4 converges to the exact
  2 S_ij S_ij at second order (edge means taken at the right places).
"""

from __future__ import annotations

import numpy as np
import pytest


def _zh_all(nz, g, lz=1.0, s=0.4):
    """Face heights zh_k for k = -g .. nz+g (a smooth stretching)."""
    k = np.arange(-g, nz + g + 1) / nz
    return lz * (k + s * k * k)


def _linear(Gm, nx, ny, nz, g, dx, dy, zh):
    """Padded u, v, w of u_i = Gm[i] . (x, y, z) at their staggered positions,
    and dz, dzh for levels -g .. nz+g-1 (index k+g)."""
    zc = 0.5 * (zh[:-1] + zh[1:])              # centres z_k, k = -g .. nz+g-1
    zf = zh[:-1]                               # faces zh_k, same range
    dz = zh[1:] - zh[:-1]
    dzh = np.empty_like(dz)
    dzh[1:] = zc[1:] - zc[:-1]
    dzh[0] = zc[0] - (zh[0] - 0.5 * dz[0])     # one more centre below (linear grid edge)
    i = np.arange(-g, nx + g)
    j = np.arange(-g, ny + g)
    xh, xc = i * dx, (i + 0.5) * dx
    yh, yc = j * dy, (j + 0.5) * dy

    def field(row, X, Y, Z):
        return (row[0] * X[None, None, :] + row[1] * Y[None, :, None] + row[2] * Z[:, None, None])
    up = field(Gm[0], xh, yc, zc)
    vp = field(Gm[1], xc, yh, zc)
    wp = field(Gm[2], xc, yc, zf)
    return up, vp, wp, dz, dzh


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_linear_field_is_exact(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    Gm = rng.standard_normal((3, 3))
    nx, ny, nz, g = 9, 7, 6, 1
    dx, dy, cs = 0.13, 0.21, 0.17
    zh = _zh_all(nz, g)
    up, vp, wp, dz, dzh = _linear(Gm, nx, ny, nz, g, dx, dy, zh)
    nu = oracle_mod.smagorinsky_padded(up, vp, wp, g=g, dx=dx, dy=dy, dz=dz, dzh=dzh, cs=cs)
    S = 0.5 * (Gm + Gm.T)
    s_abs = np.sqrt(2.0 * (S * S).sum())
    for k in range(nz):
        delta = (dx * dy * dz[k + g]) ** (1.0 / 3.0)
        expect = (cs * delta) ** 2 * s_abs
        assert np.allclose(nu[k], expect, rtol=1e-12, atol=0), (k, nu[k].max(), expect)


def test_rotation_has_no_strain(oracle_mod):
    Gm = np.array([[0.0, -1.3, 0.4], [1.3, 0.0, -0.7], [-0.4, 0.7, 0.0]])
    zh = _zh_all(5, 1)
    up, vp, wp, dz, dzh = _linear(Gm, 6, 6, 5, 1, 0.1, 0.1, zh)
    nu = oracle_mod.smagorinsky_padded(up, vp, wp, g=1, dx=0.1, dy=0.1, dz=dz, dzh=dzh, cs=0.2)
    assert np.abs(nu).max() < 1e-9 * 0.2 ** 2 * 0.1 ** 2


def _fields(n=(10, 9, 8), seed=4):
    rng = np.random.default_rng(seed)
    return [rng.standard_normal(n) for _ in range(3)]


def test_cs_scaling_and_galilean_invariance(oracle_mod):
    u, v, w = _fields()
    nz = u.shape[0]
    zh = np.linspace(0, 1, nz + 1) ** 1.2
    kw = dict(g=1, walls=False, dx=0.1, dy=0.12, zh=zh)
    a = oracle_mod.smagorinsky(u, v, w, cs=0.1, **kw)
    b = oracle_mod.smagorinsky(u, v, w, cs=0.2, **kw)
    assert np.array_equal(b, 4 * a)
    c = oracle_mod.smagorinsky(u + 3.0, v - 1.5, w + 0.25, cs=0.1, **kw)
    assert np.allclose(c, a, rtol=1e-12, atol=1e-14)
    assert (a > 0).all()


def _exact_s2(x, y, z):
    """2 S_ij S_ij of u = sin(2 pi y) cos(2 pi z), v = sin(2 pi x), w = cos(2 pi x) / 2."""
    p = 2 * np.pi
    dudy = p * np.cos(p * y) * np.cos(p * z)
    dudz = -p * np.sin(p * y) * np.sin(p * z)
    dvdx = p * np.cos(p * x)
    dwdx = -p * np.sin(p * x) / 2
    sxy, sxz = 0.5 * (dudy + dvdx), 0.5 * (dudz + dwdx)
    return 4 * (sxy ** 2 + sxz ** 2)


def test_second_order_convergence(oracle_mod):
    errs = []
    cs = 0.2
    for n in (16, 32, 64):
        h = 1.0 / n
        i = np.arange(n)
        xc, xh = (i + 0.5) * h, i * h
        yc, zc = xc, xc
        u = np.sin(2 * np.pi * yc)[None, :, None] * np.cos(2 * np.pi * zc)[:, None, None] \
            + 0 * xh[None, None, :]
        v = np.broadcast_to(np.sin(2 * np.pi * xc)[None, None, :], (n, n, n)).copy()
        w = np.broadcast_to(0.5 * np.cos(2 * np.pi * xc)[None, None, :], (n, n, n)).copy()
        zh = np.linspace(0, 1, n + 1)
        nu = oracle_mod.smagorinsky(u, v, w, g=1, walls=False, dx=h, dy=h, zh=zh, cs=cs)
        s2 = nu ** 2 / (cs * h) ** 4
        Z, Y, X = np.meshgrid(zc, yc, xc, indexing="ij")
        errs.append(np.abs(s2 - _exact_s2(X, Y, Z)).max())
    rates = [np.log2(errs[q] / errs[q + 1]) for q in range(2)]
    assert all(r > 1.8 for r in rates), (errs, rates)


def test_wall_mirror_symmetry(oracle_mod):
    """Free-slip walls: reflecting the flow about the mid-plane (u, v even,
    w odd, faces k <-> nz - k) reflects nu level by level, so the bottom and
    top wall ghosts are handled alike."""
    rng = np.random.default_rng(9)
    nz, ny, nx = 7, 6, 8
    u, v = rng.standard_normal((nz, ny, nx)), rng.standard_normal((nz, ny, nx))
    w = rng.standard_normal((nz, ny, nx))
    w[0] = 0.0                                    # the bottom wall face
    um, vm = u[::-1].copy(), v[::-1].copy()
    wm = np.zeros_like(w)
    wm[1:] = -w[1:][::-1]                         # face k of the mirror = -face nz-k
    zh = np.linspace(0.0, 1.0, nz + 1)
    kw = dict(g=1, walls=True, dx=1 / nx, dy=1 / ny, zh=zh, cs=0.15)
    a = oracle_mod.smagorinsky(u, v, w, **kw)
    b = oracle_mod.smagorinsky(um, vm, wm, **kw)
    assert np.allclose(b, a[::-1], rtol=1e-13, atol=0)
    # and the mirror is not trivially equal to the original
    assert not np.allclose(a, a[::-1])


# ------------------------------------------------- planted mistakes
# Each mutant plants one plausible mistake in a copy of oracle.c (built on
# the CPU); a fast subset of the pins above must reject it, and the
# unmodified source must pass the same subset.

SMAG_MUTANTS = [
    ("half factor", "return 0.5 * ((DU(i, j, k) - DU(i, j - 1, k)) / D->G->dy +",
     "return 1.0 * ((DU(i, j, k) - DU(i, j - 1, k)) / D->G->dy +"),
    ("edge mean", "mxy += e1 * e1 / 4.0;", "mxy += e1 * e1 / 2.0;"),
    ("edge level", "double e2 = exz(D, i + a, j, k + b);", "double e2 = exz(D, i + a, j, k + b - 1);"),
    ("szz metric", "double szz = (DW(i, j, k + 1) - DW(i, j, k)) / dz[k + g];",
     "double szz = (DW(i, j, k + 1) - DW(i, j, k)) / dzh[k + g];"),
    ("delta metric", "double delta = cbrt(dx * dy * dz[k + g]);",
     "double delta = cbrt(dx * dy * dzh[k + g]);"),
    ("normal weight", "double s2 = 2.0 * (sxx * sxx + syy * syy + szz * szz)",
     "double s2 = 1.0 * (sxx * sxx + syy * syy + szz * szz)"),
    ("cross index", "return 0.5 * ((DV(i, j, k) - DV(i, j, k - 1)) / D->G->dzh[k + D->G->g] +\n"
                    "                  (DW(i, j, k) - DW(i, j - 1, k)) / D->G->dy);",
     "return 0.5 * ((DV(i, j, k) - DV(i, j, k - 1)) / D->G->dzh[k + D->G->g] +\n"
     "                  (DW(i, j, k) - DW(i - 1, j, k)) / D->G->dy);"),
]


def _smag_pins_pass(mod) -> bool:
    try:
        for seed in range(2):
            test_linear_field_is_exact(mod, seed)
        test_rotation_has_no_strain(mod)
        test_wall_mirror_symmetry(mod)
        errs = []
        for n in (16, 32):
            h = 1.0 / n
            xc = (np.arange(n) + 0.5) * h
            u = np.sin(2 * np.pi * xc)[None, :, None] * np.cos(2 * np.pi * xc)[:, None, None] \
                + np.zeros((1, 1, n))
            v = np.broadcast_to(np.sin(2 * np.pi * xc)[None, None, :], (n, n, n)).copy()
            w = np.broadcast_to(0.5 * np.cos(2 * np.pi * xc)[None, None, :], (n, n, n)).copy()
            nu = mod.smagorinsky(u, v, w, g=1, walls=False, dx=h, dy=h, zh=np.linspace(0, 1, n + 1),
                                 cs=0.2)
            Z, Y, X = np.meshgrid(xc, xc, xc, indexing="ij")
            errs.append(np.abs(nu ** 2 / (0.2 * h) ** 4 - _exact_s2(X, Y, Z)).max())
        return np.log2(errs[0] / errs[1]) > 1.7
    except AssertionError:
        return False


@pytest.fixture()
def swap_lib(oracle_mod):
    saved = oracle_mod._lib
    yield
    oracle_mod._lib = saved


def _use_source(oracle_mod, tmp_path, text):
    import ctypes
    import subprocess
    c, so = tmp_path / "m.c", tmp_path / "m.so"
    c.write_text(text)
    subprocess.check_call(["gcc", "-O1", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(so),
                           str(c), "-lm"])
    lib = ctypes.CDLL(str(so))
    ref = oracle_mod._load()
    for name in ("or_zprofile", "or_fill_ghosts", "or_tendency", "or_diag", "or_smagorinsky"):
        getattr(lib, name).argtypes = getattr(ref, name).argtypes
    oracle_mod._lib = lib


def _source(oracle_mod):
    import os
    return open(os.path.join(os.path.dirname(oracle_mod.__file__), "oracle.c")).read()


def test_unmodified_source_passes_the_subset(oracle_mod, tmp_path, swap_lib):
    _use_source(oracle_mod, tmp_path, _source(oracle_mod))
    assert _smag_pins_pass(oracle_mod)


@pytest.mark.parametrize("name,old,new", SMAG_MUTANTS, ids=[m[0] for m in SMAG_MUTANTS])
def test_planted_mistake_is_caught(oracle_mod, tmp_path, swap_lib, name, old, new):
    text = _source(oracle_mod)
    assert text.count(old) == 1, name
    _use_source(oracle_mod, tmp_path, text.replace(old, new))
    with np.errstate(all="ignore"):
        assert not _smag_pins_pass(oracle_mod), f"mutant '{name}' passed every pin"
