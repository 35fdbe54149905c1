"""Seeded synthetic inputs for the stencil workloads (data only, no stencil arithmetic).

This module is the one piece shared by the CPU oracle's tests and the GPU path:
it draws velocity fields, the eddy-viscosity field, vertical grids and batch
sizes from a counter-based generator so that both sides see identical inputs.
It holds no finite-difference, interpolation or boundary-condition arithmetic.

The paper's workloads are MicroHH runs on 256^3 and 512^3 grids in single and
double precision (Sec. 5.3, Table 3); those fields are not available, so these
seeded Fourier fields stand in for them at the same sizes.

Generator: SplitMix64 (Steele, Lea, Flood 2014), output n = mix(seed + n*gamma)
for n = 1, 2, ...; uniforms on [0,1) are the top 53 bits times 2^-53; normals
use Box-Muller with two uniforms per normal (the sine branch is discarded).

Draw order for one grid: for each of u, v, w (in that order) and each of its
`modes` Fourier modes: kx, ky, kz in {1..4} (u64 mod 4, plus 1), amplitude
N(0,1) (two draws), phase U[0, 2pi) (one draw); then noise U(-amp, amp), one
draw per interior point in k, j, i order, for u, then v, then w; then, if asked
for, the eddy viscosity nu = nu0 * (1 + U[0,1)) per interior point in k, j, i
order.
"""

from __future__ import annotations

import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
BASE_SEED = 2303123740
_BLOCK = 1 << 18


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


class SplitMix64:
    """Counter-based SplitMix64 stream; draws are vectorised over counters."""

    def __init__(self, seed: int):
        self.seed = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
        self.pos = 0

    def u64(self, n: int) -> np.ndarray:
        out = np.empty(n, dtype=np.uint64)
        with np.errstate(over="ignore"):
            # blocks of counters small enough for the temporaries to stay in cache
            t = np.empty(min(n, _BLOCK), dtype=np.uint64)
            for s in range(0, n, _BLOCK):
                m = min(_BLOCK, n - s)
                z = out[s:s + m]
                z[:] = np.arange(self.pos + 1 + s, self.pos + 1 + s + m, dtype=np.uint64)
                z *= GAMMA
                z += self.seed
                # the mix of _mix, in place
                tt = t[:m]
                np.right_shift(z, np.uint64(30), out=tt)
                z ^= tt
                z *= _M1
                np.right_shift(z, np.uint64(27), out=tt)
                z ^= tt
                z *= _M2
                np.right_shift(z, np.uint64(31), out=tt)
                z ^= tt
        self.pos += n
        return out

    def uniform(self, n: int) -> np.ndarray:
        """n uniforms on [0, 1)."""
        u = self.u64(n)
        u >>= np.uint64(11)
        f = u.astype(np.float64)
        f *= 2.0 ** -53
        return f

    def normal(self) -> float:
        u1, u2 = self.uniform(2)
        return math.sqrt(-2.0 * math.log(1.0 - u1)) * math.cos(2.0 * math.pi * u2)

    def int_1_to_4(self) -> int:
        return int(self.u64(1)[0] % np.uint64(4)) + 1


def zfaces(nz: int, lz: float = 1.0, stretch: float = 0.0) -> np.ndarray:
    """Face heights zh_0..zh_nz of the vertical grid.

    stretch == 0: uniform spacing lz/nz.  stretch = s > 0: tanh stretching
    zh_k = lz * (1 + tanh(s*(k/nz - 1)) / tanh(s)), clustered at the bottom.
    """
    k = np.arange(nz + 1, dtype=np.float64)
    if stretch == 0.0:
        return k * (lz / nz)
    return lz * (1.0 + np.tanh(stretch * (k / nz - 1.0)) / math.tanh(stretch))


def _add_mode(f, amp, phase, kx, ky, kz, xs, ys, zs, lz, walls, zfun):
    """f[k, j, i] += amp * sin(2pi(kx x + ky y [+ kz z/lz]) + phase) [* zfac(z)]."""
    tx = 2.0 * math.pi * kx * xs
    ty = 2.0 * math.pi * ky * ys
    if walls:
        tyz = ty[None, :] + phase + 0.0 * zs[:, None]
        zfac = zfun(math.pi * kz * zs / lz)
    else:
        tyz = ty[None, :] + (2.0 * math.pi * kz / lz) * zs[:, None] + phase
        zfac = np.ones_like(zs)
    sx, cx = np.sin(tx), np.cos(tx)
    syz, cyz = np.sin(tyz), np.cos(tyz)
    for k in range(len(zs)):
        a = amp * zfac[k]
        f[k] += a * (np.outer(cyz[k], sx) + np.outer(syz[k], cx))


def velocity_fields(nx: int, ny: int, nz: int, *, seed: int, walls: bool,
                    zh: np.ndarray | None = None, lz: float = 1.0,
                    modes: int = 4, noise: float = 1e-3,
                    nu0: float | None = None) -> dict:
    """Seeded u, v, w (and optionally nu) on interior points, float64, shape (nz, ny, nx).

    Staggering (Arakawa C): u at (i dx, (j+1/2) dy, z_k), v at ((i+1/2) dx, j dy, z_k),
    w at ((i+1/2) dx, (j+1/2) dy, zh_k), nu at cell centres; dx = 1/nx, dy = 1/ny,
    z_k = (zh_k + zh_{k+1}) / 2.  With walls (`walls=True`) the z factor of a mode
    is cos(pi kz z / lz) for u, v and sin(pi kz z / lz) for w, and w on the bottom
    wall (k = 0) is zero.
    """
    if zh is None:
        zh = zfaces(nz, lz)
    zh = np.asarray(zh, dtype=np.float64)
    assert zh.shape == (nz + 1,)
    lz = float(zh[-1] - zh[0])
    zc = 0.5 * (zh[:-1] + zh[1:]) - zh[0]
    zf = zh[:-1] - zh[0]
    xh = np.arange(nx, dtype=np.float64) / nx
    xc = (np.arange(nx, dtype=np.float64) + 0.5) / nx
    yh = np.arange(ny, dtype=np.float64) / ny
    yc = (np.arange(ny, dtype=np.float64) + 0.5) / ny
    pos = {"u": (xh, yc, zc, np.cos), "v": (xc, yh, zc, np.cos),
           "w": (xc, yc, zf, np.sin)}

    rng = SplitMix64(seed)
    draws = {}
    for name in ("u", "v", "w"):
        lst = []
        for _ in range(modes):
            kx, ky, kz = rng.int_1_to_4(), rng.int_1_to_4(), rng.int_1_to_4()
            amp = rng.normal()
            phase = 2.0 * math.pi * rng.uniform(1)[0]
            lst.append((amp, phase, kx, ky, kz))
        draws[name] = lst

    out = {}
    n = nx * ny * nz
    for name in ("u", "v", "w"):
        xs, ys, zs, zfun = pos[name]
        f = np.zeros((nz, ny, nx), dtype=np.float64)
        for amp, phase, kx, ky, kz in draws[name]:
            _add_mode(f, amp, phase, kx, ky, kz, xs, ys, zs, lz, walls, zfun)
        out[name] = f
    for name in ("u", "v", "w"):
        if noise:
            out[name] += (noise * (2.0 * rng.uniform(n) - 1.0)).reshape(nz, ny, nx)
    if walls:
        out["w"][0] = 0.0
    if nu0 is not None:
        out["nu"] = (nu0 * (1.0 + rng.uniform(n))).reshape(nz, ny, nx)
    out["zh"] = zh
    out["modes"] = draws
    return out


def batch_sizes(seed: int, count: int = 64) -> list[tuple[int, int, int]]:
    """Grid sizes of a batch: nx, ny in {32, 48, ..., 192}, nz in {32, 48, ..., 128}."""
    rng = SplitMix64(seed)
    sizes = []
    for _ in range(count):
        a, b, c = rng.u64(3)
        nx = 32 + 16 * int(a % np.uint64(11))
        ny = 32 + 16 * int(b % np.uint64(11))
        nz = 32 + 16 * int(c % np.uint64(7))
        sizes.append((nx, ny, nz))
    return sizes


# The five workloads: name -> description.  Index i uses seed BASE_SEED + i.
WORKLOADS = {
    "periodic64_adv2_f64": dict(index=0, nx=64, ny=64, nz=64, g=1, walls=False,
                                adv=2, diff=1, nu=1e-3, dtypes=("f64",)),
    "walls256_adv5_diff": dict(index=1, nx=256, ny=256, nz=256, g=3, walls=True,
                               adv=5, diff=1, nu=1e-3, dtypes=("f32", "f64")),
    "walls512x512x256_precision": dict(index=2, nx=512, ny=512, nz=256, g=3,
                                       walls=True, adv=5, diff=1, nu=1e-3,
                                       dtypes=("f64", "f32", "bf16", "f16")),
    "batch64_uneven": dict(index=3, count=64, g=3, walls=True, adv=5, diff=1,
                           nu=1e-3, dtypes=("f32",)),
    "les1024x1024x64_stretched_varnu": dict(index=4, nx=1024, ny=1024, nz=64, g=3,
                                            walls=True, adv=5, diff=2, nu=1e-3,
                                            lz=64.0 / 1024.0, stretch=2.0,
                                            dtypes=("f32",)),
}


def seed_of(index: int) -> int:
    return BASE_SEED + index
