"""The pins catch plausible mistakes: each test plants one mistake in a
temporary copy of oracle/oracle.c (on the CPU), builds it, and checks that a
fast subset of the pins of test_oracle_pins rejects the mutant while the
unmodified oracle passes the same subset."""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_2303_12374_gb300 import synth

analytic = pytest.importorskip("analytic")
pins = pytest.importorskip("test_oracle_pins")

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

# (name, text to replace, replacement) -- one plausible mistake each
MUTANTS = [
    ("i6 coefficient", "+ 37.0 * a[2] + 37.0 * a[3]", "+ 36.0 * a[2] + 37.0 * a[3]"),
    ("d6 sign", "return U * I6(a) + fabs(U) * D6(a);", "return U * I6(a) - fabs(U) * D6(a);"),
    ("dropped |U|", "return U * I6(a) + fabs(U) * D6(a);", "return U * I6(a) + U * D6(a);"),
    ("u window offset", "window(C, C->u, 0, i, j, k, -2, a);", "window(C, C->u, 0, i, j, k, -3, a);"),
    ("v advecting velocity", "(U_(i, j - 1, k) + U_(i, j, k)) / 2.0", "(U_(i, j, k) + U_(i, j + 1, k)) / 2.0"),
    ("dropped w z flux", "- (Fwz(C, i, j, k) - Fwz(C, i, j, k - 1)) / dzhk;", ";"),
    ("u z metric", "(up - dn) / G->dz[k + G->g];", "(up - dn) / G->dzh[k + G->g];"),
    ("w laplacian metric", "(c - a[P(G, i, j, k - 1)]) / G->dz[k - 1 + G->g];",
     "(c - a[P(G, i, j, k - 1)]) / G->dz[k + G->g];"),
    ("stress cross term", "(DV(i, j, k) - DV(i - 1, j, k)) / D->G->dx);",
     "(DV(i, j, k) - DV(i, j - 1, k)) / D->G->dx);"),
    ("nu edge average", "return (DN(i - 1, j - 1, k) + DN(i, j - 1, k) + DN(i - 1, j, k) + DN(i, j, k)) / 4.0;",
     "return (DN(i - 1, j - 1, k) + DN(i, j - 1, k) + DN(i - 1, j, k) + DN(i, j, k)) / 2.0;"),
    ("odd mirror sign", "if (k < 0) { sk = -k; sign = -1.0; }", "if (k < 0) { sk = -k; sign = 1.0; }"),
    ("even mirror index", "if (k < 0) sk = -1 - k;", "if (k < 0) sk = -k;"),
]


def _build(tmp_path, text):
    c = tmp_path / "m.c"
    so = tmp_path / "m.so"
    c.write_text(text)
    subprocess.check_call(["gcc", "-O1", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(so),
                           str(c), "-lm"])
    return str(so)


def _use(so_path):
    """Point the oracle wrapper at another build of the library."""
    lib = ctypes.CDLL(so_path)
    ref = oracle._load()
    for name in ("or_zprofile", "or_fill_ghosts", "or_tendency", "or_diag"):
        getattr(lib, name).argtypes = getattr(ref, name).argtypes
    oracle._lib = lib


def _pins_pass() -> bool:
    """A fast subset of the pins; True when every one holds."""
    checks = [
        lambda: pins._conv_errors(oracle, adv=5, diff=1, walls=True, stretch=0.0, ns=[16, 32]),
        lambda: pins._conv_errors(oracle, adv=0, diff=2, walls=True, stretch=2.0, ns=[32, 64],
                                  var_nu=True),
    ]
    try:
        for adv, order in ((5, 5.0), (2, 2.0)):
            for axis in (0, 1, 2):
                errs = [pins._const_velocity_case(oracle, n, axis, adv, 1.3) for n in (32, 64)]
                s = analytic.slope([1 / 32, 1 / 64], errs)
                if not abs(s - order) < 0.4:
                    return False
        for fn in checks:
            inner, edge = fn()
            hs = [1.0 / n for n in ((16, 32) if len(inner) == 2 and inner[0] > inner[1] * 3.5 else (32, 64))]
            s = analytic.slope(hs, inner)
            if not (1.7 < s < 2.5) or inner[-1] > 2e-2 or edge[-1] > 3e-2:
                return False
        f = pins._fields(walls=True, stretch=2.0, nu0=1e-3)
        dz, _ = oracle.zprofile(8, 3, True, f["zh"])
        ut, vt, wt = pins.run(oracle, f, adv=5, diff=2, walls=True, nu_field=f["nu"])
        wgt = dz[3:11][:, None, None]
        for t in (ut, vt):
            if abs((t * wgt).sum()) > 1e-12 * np.abs(t * wgt).sum():
                return False
        a = np.random.default_rng(0).standard_normal((6, 5, 7))
        w = a.copy()
        w[0] = 0.0
        ext = np.concatenate([w, np.zeros((1,) + w.shape[1:])], axis=0)
        ext = np.pad(ext, ((0, 0), (3, 3), (3, 3)), mode="wrap")
        ref = np.concatenate([-ext[1:4][::-1], ext, -ext[-4:-1][::-1][:-1]], axis=0)
        if not np.array_equal(oracle.pad(w, 3, walls=True, odd=True), ref):
            return False
        even = np.pad(np.pad(a, ((0, 0), (3, 3), (3, 3)), mode="wrap"), ((3, 3), (0, 0), (0, 0)),
                      mode="symmetric")
        if not np.array_equal(oracle.pad(a, 3, walls=True, odd=False), even):
            return False
        fsym = pins.divergence_free(n=(12, 12, 12))
        sw = lambda x: np.ascontiguousarray(x.transpose(0, 2, 1))
        nuf = synth.velocity_fields(12, 12, 12, seed=2, walls=False, nu0=1e-3)["nu"]
        g = {"u": sw(fsym["v"]), "v": sw(fsym["u"]), "w": sw(fsym["w"]), "zh": fsym["zh"]}
        t1 = pins.run(oracle, fsym, adv=5, diff=2, nu_field=nuf)
        t2 = pins.run(oracle, g, adv=5, diff=2, nu_field=sw(nuf))
        for x, y in ((t2[0], sw(t1[1])), (t2[1], sw(t1[0])), (t2[2], sw(t1[2]))):
            if np.abs(x - y).max() > 1e-12 * np.abs(y).max():
                return False
        # const-nu diffusion on a stretched wall grid converges at order 2
        inner, edge = pins._conv_errors(oracle, adv=0, diff=1, walls=True, stretch=2.0,
                                        ns=[32, 64])
        if not (1.7 < analytic.slope([1 / 32, 1 / 64], inner) < 2.5):
            return False
        # periodic stretched z: each component's metric-weighted sum vanishes
        fp = pins._fields(n=(10, 8, 12), walls=False, stretch=2.0, nu0=1e-3)
        dzp, dzhp = oracle.zprofile(12, 3, False, fp["zh"])
        for diff in (1, 2):
            ts = pins.run(oracle, fp, adv=5, diff=diff, walls=False, nu_field=fp["nu"])
            for t, wv in zip(ts, (dzp, dzp, dzhp)):
                tw = t * wv[3:15][:, None, None]
                if abs(tw.sum()) > 1e-12 * np.abs(tw).sum():
                    return False
        # upwinding dissipates energy (a downwind-biased scheme is 5th order too)
        fdf = pins.divergence_free(n=(12, 12, 12))
        ut, vt, wt = pins.run(oracle, fdf, adv=5, diff=0)
        terms = fdf["u"] * ut + fdf["v"] * vt + fdf["w"] * wt
        if not terms.sum() < -1e-3 * np.abs(terms).sum():
            return False
        # the textbook upwind-5 symbol on one Fourier mode
        nx, dx, vel0 = 32, 1.0 / 32, 0.9
        theta = 2 * np.pi * 3 * dx
        i = np.arange(nx)
        vrow = 1.4 * np.sin(theta * (i + 0.5) + 0.37)
        fm = {"u": np.full((4, 4, nx), vel0), "v": np.broadcast_to(vrow, (4, 4, nx)).copy(),
              "w": np.zeros((4, 4, nx)), "zh": synth.zfaces(4)}
        _, vt, _ = oracle.tendencies(fm["u"], fm["v"], fm["w"], adv=5, diff=0, g=3, walls=False,
                                     dx=dx, dy=0.25, zh=fm["zh"])
        S = analytic.fourier_symbol_upwind5(theta, True)
        expect = -(vel0 / dx) * np.imag(1.4 * np.exp(1j * 0.37) * np.exp(1j * theta * (i + 0.5)) * S)
        if np.abs(vt[0, 0] - expect).max() > 1e-12 * np.abs(expect).max():
            return False
    except (AssertionError, FloatingPointError, ValueError):
        return False
    return True


@pytest.fixture()
def restore():
    saved = oracle._lib
    yield
    oracle._lib = saved


def test_unmodified_oracle_passes_the_subset(tmp_path, restore):
    _use(_build(tmp_path, open(SRC).read()))
    assert _pins_pass()


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(tmp_path, restore, name, old, new):
    text = open(SRC).read()
    assert text.count(old) >= 1, name
    _use(_build(tmp_path, text.replace(old, new, 1)))
    with np.errstate(all="ignore"):
        assert not _pins_pass(), f"mutant '{name}' passed every pin"
