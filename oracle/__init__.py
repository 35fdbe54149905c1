"""FP64 CPU oracle of the stencil tendencies and the Smagorinsky viscosity
(test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import
this package.  The product path (paper_2303_12374_gb300) never does; the two
share no code.  `build()` compiles oracle.c with gcc into oracle/_build/:
liboracle.so, the serial build every test pins, and liboracle_omp.so, the same
source with -fopenmp (the tendency loop split over the host cores), used only
to time the oracle on all cores (`tendencies(..., threads=n)`).

Arrays are numpy float64 in (nz, ny, nx) order (x fastest), interior only,
unless a name says "padded".
"""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_SO_OMP = os.path.join(_HERE, "_build", "liboracle_omp.so")
_lib = None
_lib_omp = None


def _compile(out: str, extra) -> None:
    src = os.path.join(_HERE, "oracle.c")
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                           "-shared", *extra, "-o", tmp, src, "-lm"])
    os.replace(tmp, out)


def build(force: bool = False) -> str:
    """Compile oracle.c (plain C, FP64, no FMA contraction) into a shared
    library, and its OpenMP timing build when gcc supports -fopenmp."""
    src = os.path.join(_HERE, "oracle.c")
    for out, extra in ((_SO, []), (_SO_OMP, ["-fopenmp"])):
        if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
            try:
                _compile(out, extra)
            except (subprocess.CalledProcessError, OSError):
                if out == _SO:
                    raise
    return _SO


def _declare(lib):
    dp = ctypes.POINTER(ctypes.c_double)
    lib.or_zprofile.argtypes = [ctypes.c_int] * 3 + [dp, dp, dp]
    lib.or_fill_ghosts.argtypes = [ctypes.c_int] * 6 + [dp]
    lib.or_tendency.argtypes = ([ctypes.c_int] * 5 + [ctypes.c_double] * 2 + [dp, dp]
                                + [ctypes.c_int] * 2 + [ctypes.c_double] + [dp] * 4
                                + [ctypes.c_int] * 2 + [dp] * 3)
    lib.or_diag.argtypes = [ctypes.c_size_t, dp, dp, dp, dp]
    lib.or_smagorinsky.argtypes = ([ctypes.c_int] * 4 + [ctypes.c_double] * 2 + [dp, dp]
                                   + [ctypes.c_double] + [dp] * 3 + [ctypes.c_int] * 2 + [dp])
    lib.or_set_threads.argtypes = [ctypes.c_int]
    lib.or_set_threads.restype = ctypes.c_int
    return lib


def _load_omp():
    """The OpenMP timing build, or None where it could not be built."""
    global _lib_omp
    if _lib_omp is None:
        build()
        if not os.path.exists(_SO_OMP):
            return None
        _lib_omp = _declare(ctypes.CDLL(_SO_OMP))
    return _lib_omp


def omp_available() -> bool:
    return _load_omp() is not None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.or_zprofile.argtypes = [ctypes.c_int] * 3 + [dp, dp, dp]
        lib.or_fill_ghosts.argtypes = [ctypes.c_int] * 6 + [dp]
        lib.or_tendency.argtypes = ([ctypes.c_int] * 5 + [ctypes.c_double] * 2 + [dp, dp]
                                    + [ctypes.c_int] * 2 + [ctypes.c_double] + [dp] * 4
                                    + [ctypes.c_int] * 2 + [dp] * 3)
        lib.or_diag.argtypes = [ctypes.c_size_t, dp, dp, dp, dp]
        lib.or_smagorinsky.argtypes = ([ctypes.c_int] * 4 + [ctypes.c_double] * 2 + [dp, dp]
                                       + [ctypes.c_double] + [dp] * 3 + [ctypes.c_int] * 2 + [dp])
        lib.or_set_threads.argtypes = [ctypes.c_int]
        lib.or_set_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def zprofile(nz: int, g: int, walls: bool, zh: np.ndarray):
    """dz_k and dzh_k for k in [-g, nz+g), index k+g."""
    lib = _load()
    zh = np.ascontiguousarray(zh, dtype=np.float64)
    dz = np.empty(nz + 2 * g)
    dzh = np.empty(nz + 2 * g)
    lib.or_zprofile(nz, g, int(walls), _p(zh), _p(dz), _p(dzh))
    return dz, dzh


def pad(a: np.ndarray, g: int, walls: bool, odd: bool) -> np.ndarray:
    """Padded copy of an interior field with its ghost cells filled."""
    lib = _load()
    nz, ny, nx = a.shape
    out = np.zeros((nz + 2 * g, ny + 2 * g, nx + 2 * g))
    out[g:g + nz, g:g + ny, g:g + nx] = a
    lib.or_fill_ghosts(nx, ny, nz, g, int(walls), int(odd), _p(out))
    return out


def tendencies(u, v, w, *, adv: int, diff: int, g: int, walls: bool, dx: float,
               dy: float, zh: np.ndarray, nu: float = 0.0, nu_field=None, levels=None,
               threads: int = 1):
    """(ut, vt, wt) on the interior; inputs are interior fields (nz, ny, nx).

    levels=(k0, k1) computes only interior levels k0 <= k < k1 (outputs of
    shape (k1-k0, ny, nx)); the default is every level.  threads > 1 runs the
    tendency loop of the OpenMP timing build on that many threads (same
    results); it raises if that build is unavailable.
    """
    if threads > 1:
        lib = _load_omp()
        if lib is None:
            raise RuntimeError("the OpenMP build of the oracle is unavailable")
        lib.or_set_threads(threads)
    else:
        lib = _load()
    nz, ny, nx = u.shape
    u, v, w = (np.ascontiguousarray(x, dtype=np.float64) for x in (u, v, w))
    up, vp, wp = pad(u, g, walls, False), pad(v, g, walls, False), pad(w, g, walls, True)
    np_ = pad(np.ascontiguousarray(nu_field, dtype=np.float64), g, walls, False) \
        if nu_field is not None else None
    dz, dzh = zprofile(nz, g, walls, zh)
    k0, k1 = (0, nz) if levels is None else levels
    assert 0 <= k0 < k1 <= nz
    ut, vt, wt = (np.empty((k1 - k0, ny, nx)) for _ in range(3))
    lib.or_tendency(nx, ny, nz, g, int(walls), dx, dy, _p(dz), _p(dzh), adv, diff, nu,
                    _p(up), _p(vp), _p(wp), _p(np_), k0, k1, _p(ut), _p(vt), _p(wt))
    return ut, vt, wt


def tendencies_padded(up, vp, wp, *, adv: int, diff: int, g: int, walls: bool, dx: float,
                      dy: float, zh: np.ndarray, nu: float = 0.0, np_=None):
    """(ut, vt, wt) on the interior from padded u, v, w (and nu) whose ghosts
    the caller has set, e.g. one block of a decomposed grid after its halo
    exchange; dx, dy are the grid spacings, zh the block's nz+1 faces."""
    lib = _load()
    nzp, nyp, nxp = up.shape
    nz, ny, nx = nzp - 2 * g, nyp - 2 * g, nxp - 2 * g
    up, vp, wp = (np.ascontiguousarray(x, dtype=np.float64) for x in (up, vp, wp))
    if np_ is not None:
        np_ = np.ascontiguousarray(np_, dtype=np.float64)
    dz, dzh = zprofile(nz, g, walls, zh)
    ut, vt, wt = (np.empty((nz, ny, nx)) for _ in range(3))
    lib.or_tendency(nx, ny, nz, g, int(walls), dx, dy, _p(dz), _p(dzh), adv, diff, nu,
                    _p(up), _p(vp), _p(wp), _p(np_), 0, nz, _p(ut), _p(vt), _p(wt))
    return ut, vt, wt


def smagorinsky_padded(up, vp, wp, *, g: int, dx: float, dy: float, dz: np.ndarray,
                       dzh: np.ndarray, cs: float, levels=None):
    """Smagorinsky nu at the interior cell centres from padded u, v, w whose
    ghosts the caller has set (any values: analytic fields may fill them)."""
    lib = _load()
    nzp, nyp, nxp = up.shape
    nz, ny, nx = nzp - 2 * g, nyp - 2 * g, nxp - 2 * g
    k0, k1 = (0, nz) if levels is None else levels
    assert 0 <= k0 < k1 <= nz and g >= 1
    up, vp, wp = (np.ascontiguousarray(x, dtype=np.float64) for x in (up, vp, wp))
    dz, dzh = (np.ascontiguousarray(x, dtype=np.float64) for x in (dz, dzh))
    out = np.empty((k1 - k0, ny, nx))
    lib.or_smagorinsky(nx, ny, nz, g, dx, dy, _p(dz), _p(dzh), cs, _p(up), _p(vp), _p(wp),
                       k0, k1, _p(out))
    return out


def smagorinsky(u, v, w, *, g: int, walls: bool, dx: float, dy: float, zh: np.ndarray,
                cs: float, levels=None):
    """Smagorinsky nu on the interior from interior u, v, w (ghosts by the fill rules)."""
    nz = u.shape[0]
    up, vp, wp = pad(u, g, walls, False), pad(v, g, walls, False), pad(w, g, walls, True)
    dz, dzh = zprofile(nz, g, walls, zh)
    return smagorinsky_padded(up, vp, wp, g=g, dx=dx, dy=dy, dz=dz, dzh=dzh, cs=cs, levels=levels)


def diag(t: np.ndarray, ref: np.ndarray | None = None, wgt: np.ndarray | None = None):
    """[max|t-r|, rms(t-r), max|r|, rms(r), sum t, sum t*wgt] in FP64."""
    lib = _load()
    t = np.ascontiguousarray(t, dtype=np.float64).ravel()
    r = None if ref is None else np.ascontiguousarray(ref, dtype=np.float64).ravel()
    wv = None if wgt is None else np.ascontiguousarray(wgt, dtype=np.float64).ravel()
    out = np.zeros(6)
    lib.or_diag(t.size, _p(t), _p(r), _p(wv), _p(out))
    return out
