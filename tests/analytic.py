"""Exact (symbolic) tendencies of smooth fields, used to pin the oracle.

The continuous operators are written here from their textbook definitions and
differentiated by sympy; nothing here is a discretisation.  Evaluated at the
staggered points of the C grid, they are what the discrete tendencies converge
to as the grid is refined.
"""

from __future__ import annotations

import math

import numpy as np
import pytest

sp = pytest.importorskip("sympy")

X, Y, Z = sp.symbols("x y z", real=True)


def mode_sum(spec, walls: bool, lz: float, zkind: str):
    """sum A sin(2pi(kx x + ky y [+ kz z/lz]) + phase) [* cos/sin(pi kz z/lz)]."""
    e = 0
    for amp, kx, ky, kz, ph in spec:
        if walls:
            zf = sp.cos(sp.pi * kz * Z / lz) if zkind == "even" else sp.sin(sp.pi * kz * Z / lz)
            e += amp * sp.sin(2 * sp.pi * (kx * X + ky * Y) + ph) * zf
        else:
            e += amp * sp.sin(2 * sp.pi * (kx * X + ky * Y + kz * Z / lz) + ph)
    return e


def exact_tendencies(u, v, w, *, adv: bool, diff: int, nu=0.0, nu_expr=None):
    """Symbolic (ut, vt, wt): -div(u_j u_i) [+ nu lap u_i | + d_j(nu(d_j u_i + d_i u_j))]."""
    vel = (u, v, w)
    ax = (X, Y, Z)
    out = []
    for i in range(3):
        t = 0
        if adv:
            t += -sum(sp.diff(vel[j] * vel[i], ax[j]) for j in range(3))
        if diff == 1:
            t += nu * sum(sp.diff(vel[i], a, 2) for a in ax)
        elif diff == 2:
            t += sum(sp.diff(nu_expr * (sp.diff(vel[i], ax[j]) + sp.diff(vel[j], ax[i])), ax[j])
                     for j in range(3))
        out.append(t)
    return out


def evaluate(expr, xs, ys, zs):
    """expr on the tensor grid (zs, ys, xs) -> array (nz, ny, nx)."""
    f = sp.lambdify((X, Y, Z), expr, "numpy")
    zz, yy, xx = np.meshgrid(zs, ys, xs, indexing="ij")
    val = f(xx, yy, zz)
    return np.broadcast_to(np.asarray(val, dtype=np.float64), zz.shape).copy()


def staggered_points(nx, ny, zh):
    """Coordinates of u, v, w points: dict name -> (xs, ys, zs)."""
    xh = np.arange(nx) / nx
    xc = (np.arange(nx) + 0.5) / nx
    yh = np.arange(ny) / ny
    yc = (np.arange(ny) + 0.5) / ny
    zc = 0.5 * (zh[:-1] + zh[1:])
    zf = zh[:-1]
    return {"u": (xh, yc, zc), "v": (xc, yh, zc), "w": (xc, yc, zf), "c": (xc, yc, zc)}


def slope(hs, errs):
    """Least-squares slope of log(err) against log(h)."""
    return float(np.polyfit(np.log(hs), np.log(errs), 1)[0])


def fourier_symbol_upwind5(theta: float, positive: bool) -> complex:
    """Flux-difference symbol of the textbook 5th-order upwind face value.

    Face value at m+1/2 for flow in +x: (2 a_{m-2} - 13 a_{m-1} + 47 a_m
    + 27 a_{m+1} - 3 a_{m+2}) / 60 (Wicker & Skamarock 2002, Eq. 4); the
    mirror image for flow in -x.  Returns S with
    F_{m+1/2} - F_{m-1/2} = U * S * exp(i theta m) for a_m = exp(i theta m).
    """
    c = [2.0, -13.0, 47.0, 27.0, -3.0, 0.0] if positive else [0.0, -3.0, 27.0, 47.0, -13.0, 2.0]
    face = sum(cq / 60.0 * np.exp(1j * theta * (q - 2)) for q, cq in enumerate(c))
    return face * (1.0 - np.exp(-1j * theta))


TWO_PI = 2.0 * math.pi
