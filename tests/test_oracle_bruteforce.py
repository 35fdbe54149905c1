"""Brute-force pin of the oracle's tendencies on tiny grids.

An evaluator written independently here, in plain Python floats, recomputes
every face flux of every point straight from the definitions of the scheme
(C grid, flux form, Sec. 5.2's advection and diffusion kernels read as the
textbook operators):

  I6(a; m) = (a[m-2] - 8 a[m-1] + 37 a[m] + 37 a[m+1] - 8 a[m+2] + a[m+3]) / 60
  D6(a; m) = (a[m-2] - 5 a[m-1] + 10 a[m] - 10 a[m+1] + 5 a[m+2] - a[m+3]) / 60
  F5(U, a; m) = U I6 + |U| D6          (upwind-biased 5th order, Wicker-Skamarock)
  F2(U, a; m) = U (a[m] + a[m+1]) / 2  (centred 2nd order)

with the advecting velocity U the 2-point mean at the face, constant-nu
diffusion as the 3-point Laplacian with the non-uniform z metric, and
variable-nu diffusion as the stress divergence d_j[nu (d_j u_i + d_i u_j)]
(nu at centres, 4-point means on edges).  Boundary values come from index
rules (periodic wrap; even mirror of u, v, nu and odd mirror of w about the
wall faces), not from the oracle's ghost fill; the vertical metric of the
ghost levels mirrors (walls) or repeats (periodic) the grid.

Nothing is shared with the oracle: no padding, no flux reuse, a different
loop structure.  Grids 8^3 and 13 x 7 x 5, every scheme x diffusion x
boundary, uniform and stretched z.
"""

from __future__ import annotations

import numpy as np
import pytest

from paper_2303_12374_gb300 import synth


class Grid:
    def __init__(self, f, walls, nuf):
        self.u, self.v, self.w = f["u"], f["v"], f["w"]
        self.nu = nuf
        self.nz, self.ny, self.nx = self.u.shape
        self.walls = walls
        zh = f["zh"]
        nz = self.nz
        lz = zh[nz] - zh[0]

        def face(k):
            if 0 <= k <= nz:
                return float(zh[k])
            if walls:
                return 2 * zh[0] - zh[-k] if k < 0 else 2 * zh[nz] - zh[2 * nz - k]
            return zh[k + nz] - lz if k < 0 else zh[k - nz] + lz

        self.face = face
        self.dx, self.dy = 1.0 / self.nx, 1.0 / self.ny

    # ---- metric
    def zc(self, k):
        return 0.5 * (self.face(k) + self.face(k + 1))

    def dz(self, k):
        return self.face(k + 1) - self.face(k)

    def dzh(self, k):
        return self.zc(k) - self.zc(k - 1)

    # ---- field values with the boundary rules
    def _ij(self, i, j):
        return i % self.nx, j % self.ny

    def _centred(self, a, i, j, k):
        i, j = self._ij(i, j)
        nz = self.nz
        if self.walls:
            if k < 0:
                k = -1 - k
            elif k >= nz:
                k = 2 * nz - 1 - k
        else:
            k %= nz
        return float(a[k, j, i])

    def U(self, i, j, k):
        return self._centred(self.u, i, j, k)

    def V(self, i, j, k):
        return self._centred(self.v, i, j, k)

    def N(self, i, j, k):
        return self._centred(self.nu, i, j, k)

    def W(self, i, j, k):
        i, j = self._ij(i, j)
        nz = self.nz
        if not self.walls:
            return float(self.w[k % nz, j, i])
        if k < 0:
            return -float(self.w[-k, j, i])
        if k == nz:
            return 0.0
        if k > nz:
            return -float(self.w[2 * nz - k, j, i])
        return float(self.w[k, j, i])


def flux(adv, U, a, m):
    if adv == 2:
        return U * (a(m) + a(m + 1)) / 2.0
    i6 = (a(m - 2) - 8 * a(m - 1) + 37 * a(m) + 37 * a(m + 1) - 8 * a(m + 2) + a(m + 3)) / 60.0
    d6 = (a(m - 2) - 5 * a(m - 1) + 10 * a(m) - 10 * a(m + 1) + 5 * a(m + 2) - a(m + 3)) / 60.0
    return U * i6 + abs(U) * d6


def tendency_at(G, adv, diff, nu, i, j, k):
    """(tu, tv, tw) at one point, every face flux evaluated here."""
    U, V, W = G.U, G.V, G.W
    dx, dy, dz, dzh = G.dx, G.dy, G.dz(k), G.dzh(k)
    tu = tv = tw = 0.0
    if adv:
        def Fux(ii):
            return flux(adv, (U(ii, j, k) + U(ii + 1, j, k)) / 2, lambda m: U(m, j, k), ii)

        def Fuy(jj):
            return flux(adv, (V(i - 1, jj, k) + V(i, jj, k)) / 2, lambda m: U(i, m, k), jj - 1)

        def Fuz(kk):
            return flux(adv, (W(i - 1, j, kk) + W(i, j, kk)) / 2, lambda m: U(i, j, m), kk - 1)

        def Fvx(ii):
            return flux(adv, (U(ii, j - 1, k) + U(ii, j, k)) / 2, lambda m: V(m, j, k), ii - 1)

        def Fvy(jj):
            return flux(adv, (V(i, jj, k) + V(i, jj + 1, k)) / 2, lambda m: V(i, m, k), jj)

        def Fvz(kk):
            return flux(adv, (W(i, j - 1, kk) + W(i, j, kk)) / 2, lambda m: V(i, j, m), kk - 1)

        def Fwx(ii):
            return flux(adv, (U(ii, j, k - 1) + U(ii, j, k)) / 2, lambda m: W(m, j, k), ii - 1)

        def Fwy(jj):
            return flux(adv, (V(i, jj, k - 1) + V(i, jj, k)) / 2, lambda m: W(i, m, k), jj - 1)

        def Fwz(kk):
            return flux(adv, (W(i, j, kk) + W(i, j, kk + 1)) / 2, lambda m: W(i, j, m), kk)

        tu -= (Fux(i) - Fux(i - 1)) / dx + (Fuy(j + 1) - Fuy(j)) / dy + (Fuz(k + 1) - Fuz(k)) / dz
        tv -= (Fvx(i + 1) - Fvx(i)) / dx + (Fvy(j) - Fvy(j - 1)) / dy + (Fvz(k + 1) - Fvz(k)) / dz
        tw -= ((Fwx(i + 1) - Fwx(i)) / dx + (Fwy(j + 1) - Fwy(j)) / dy
               + (Fwz(k) - Fwz(k - 1)) / dzh)
    if diff == 1:
        def lap(a, zup, zdn, zc):
            return ((a(i + 1, j, k) - 2 * a(i, j, k) + a(i - 1, j, k)) / dx ** 2
                    + (a(i, j + 1, k) - 2 * a(i, j, k) + a(i, j - 1, k)) / dy ** 2
                    + ((a(i, j, k + 1) - a(i, j, k)) / zup - (a(i, j, k) - a(i, j, k - 1)) / zdn) / zc)
        tu += nu * lap(U, G.dzh(k + 1), G.dzh(k), dz)
        tv += nu * lap(V, G.dzh(k + 1), G.dzh(k), dz)
        tw += nu * lap(W, G.dz(k), G.dz(k - 1), dzh)
    elif diff == 2:
        N = G.N

        def sxx(ii):      # centre (ii, j, k), between u(ii) and u(ii+1)
            return 2 * N(ii, j, k) * (U(ii + 1, j, k) - U(ii, j, k)) / dx

        def syy(jj):
            return 2 * N(i, jj, k) * (V(i, jj + 1, k) - V(i, jj, k)) / dy

        def szz(kk):
            return 2 * N(i, j, kk) * (W(i, j, kk + 1) - W(i, j, kk)) / G.dz(kk)

        def sxy(ii, jj):  # edge (xh_ii, yh_jj, z_k)
            nu_e = 0.25 * (N(ii - 1, jj - 1, k) + N(ii, jj - 1, k) + N(ii - 1, jj, k) + N(ii, jj, k))
            return nu_e * ((U(ii, jj, k) - U(ii, jj - 1, k)) / dy + (V(ii, jj, k) - V(ii - 1, jj, k)) / dx)

        def sxz(ii, kk):  # edge (xh_ii, y_j, zh_kk)
            nu_e = 0.25 * (N(ii - 1, j, kk - 1) + N(ii, j, kk - 1) + N(ii - 1, j, kk) + N(ii, j, kk))
            return nu_e * ((U(ii, j, kk) - U(ii, j, kk - 1)) / G.dzh(kk)
                           + (W(ii, j, kk) - W(ii - 1, j, kk)) / dx)

        def syz(jj, kk):  # edge (x_i, yh_jj, zh_kk)
            nu_e = 0.25 * (N(i, jj - 1, kk - 1) + N(i, jj, kk - 1) + N(i, jj - 1, kk) + N(i, jj, kk))
            return nu_e * ((V(i, jj, kk) - V(i, jj, kk - 1)) / G.dzh(kk)
                           + (W(i, jj, kk) - W(i, jj - 1, kk)) / dy)

        tu += (sxx(i) - sxx(i - 1)) / dx + (sxy(i, j + 1) - sxy(i, j)) / dy \
            + (sxz(i, k + 1) - sxz(i, k)) / dz
        tv += (sxy(i + 1, j) - sxy(i, j)) / dx + (syy(j) - syy(j - 1)) / dy \
            + (syz(j, k + 1) - syz(j, k)) / dz
        tw += (sxz(i + 1, k) - sxz(i, k)) / dx + (syz(j + 1, k) - syz(j, k)) / dy \
            + (szz(k) - szz(k - 1)) / dzh
    if G.walls and k == 0:
        tw = 0.0
    return tu, tv, tw


CASES = [(adv, diff, walls, stretch)
         for adv in (2, 5) for diff in (1, 2) for walls in (False, True)
         for stretch in ((0.0, 2.0) if walls else (0.0,))]


@pytest.mark.parametrize("shape", [(8, 8, 8), (13, 7, 5)])
@pytest.mark.parametrize("adv,diff,walls,stretch", CASES)
def test_oracle_equals_brute_force(oracle_mod, shape, adv, diff, walls, stretch):
    nx, ny, nz = shape
    zh = synth.zfaces(nz, 1.0, stretch)
    f = synth.velocity_fields(nx, ny, nz, seed=77 + nx + 3 * nz, walls=walls, zh=zh, nu0=1e-3)
    nuf = f["nu"] * 50.0      # a viscosity large enough that diffusion is not lost in rounding
    nu = 5e-2
    G = Grid(f, walls, nuf)
    ref = np.zeros((3, nz, ny, nx))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                ref[:, k, j, i] = tendency_at(G, adv, diff, nu, i, j, k)
    got = oracle_mod.tendencies(f["u"], f["v"], f["w"], adv=adv, diff=diff, g=3, walls=walls,
                                dx=1.0 / nx, dy=1.0 / ny, zh=zh, nu=nu,
                                nu_field=nuf if diff == 2 else None)
    for r, t in zip(ref, got):
        scale = np.abs(r).max()
        assert scale > 0
        assert np.abs(t - r).max() <= 1e-15 * scale, np.abs(t - r).max() / scale


def test_openmp_timing_build_is_bitwise_serial(oracle_mod):
    """The oracle's OpenMP build (used only to time it on all host cores)
    computes every point with the same code as the serial build."""
    if not oracle_mod.omp_available():
        pytest.skip("gcc without OpenMP")
    nx, ny, nz = 24, 20, 18
    zh = synth.zfaces(nz, 1.0, 2.0)
    f = synth.velocity_fields(nx, ny, nz, seed=11, walls=True, zh=zh, nu0=1e-3)
    for diff in (1, 2):
        kw = dict(adv=5, diff=diff, g=3, walls=True, dx=1.0 / nx, dy=1.0 / ny, zh=zh, nu=1e-3,
                  nu_field=f["nu"] if diff == 2 else None)
        a = oracle_mod.tendencies(f["u"], f["v"], f["w"], **kw)
        b = oracle_mod.tendencies(f["u"], f["v"], f["w"], threads=4, **kw)
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
