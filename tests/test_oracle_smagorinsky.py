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
