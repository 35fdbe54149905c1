"""Host logic of the scenario study (Sec. 5.4-5.5): the performance
portability metric (harmonic mean of efficiencies, 0 where unsupported),
histogram binning, and the matrix/PPM assembly from two passes of timings."""

from __future__ import annotations

import pytest

from paper_2303_12374_gb300 import portability as pt


def test_ppm_is_the_harmonic_mean_or_zero():
    assert pt.ppm([1.0, 1.0, 1.0]) == 1.0
    assert pt.ppm([1.0, 0.5]) == pytest.approx(2 / 3)
    assert pt.ppm([0.9, 0.6, 0.3]) == pytest.approx(3 / (1 / 0.9 + 1 / 0.6 + 1 / 0.3))
    assert pt.ppm([1.0, None]) == 0.0
    assert pt.ppm([]) == 0.0


def test_histogram_bins():
    assert pt.histogram([0.05, 0.95, 1.0, 1.2, 0.5, 0.0]) == [2, 0, 0, 0, 0, 1, 0, 0, 0, 3]


def test_analyse_two_scenarios():
    a, b = ("advec", "256^3", "f32"), ("advec", "256^3", "f64")
    tuned = {"advec-256^3-f32": "cfgA", "advec-256^3-f64": "cfgB"}
    logs = {"advec-256^3-f32": {"random": [("x", 200.0), ("y", 100.0), ("z", None)],
                                 "bayes": [("cfgA", 50.0)]},
            "advec-256^3-f64": {"random": [("x", 300.0)], "bayes": [("cfgB", 150.0)]}}
    cross = {"advec-256^3-f32": {"default": (100.0, 0.0), "cfgA": (50.0, 1e-7), "cfgB": None},
             "advec-256^3-f64": {"default": (400.0, 0.0), "cfgA": (200.0, 0.0),
                                  "cfgB": (160.0, 1e-3)}}     # cfgB fails verification on f64
    res = pt.analyse([a, b], tuned, logs, cross)
    assert res["optimum_us"] == {"advec-256^3-f32": 50.0, "advec-256^3-f64": 200.0}
    m = res["matrix"]
    assert m["advec-256^3-f32"] == {"advec-256^3-f32": 1.0, "advec-256^3-f64": 1.0}
    assert m["advec-256^3-f64"] == {"advec-256^3-f32": None, "advec-256^3-f64": None}
    assert res["default"] == {"advec-256^3-f32": 0.5, "advec-256^3-f64": 0.5}
    rows = {r["config"]: r for r in res["ppm"]["advec"]}
    assert rows["(default configuration)"]["ppm"] == pytest.approx(0.5)
    assert rows["tuned for advec-256^3-f32"]["ppm"] == 1.0
    assert rows["tuned for advec-256^3-f64"]["ppm"] == 0.0
    assert rows["run-time selection (own record)"]["ppm"] == 1.0
    h = res["histograms"]["advec-256^3-f32"]
    assert h["ok"] == 2 and h["evals"] == 3 and h["within_10pct"] == 0.0
    assert h["bins"][2] == 1 and h["bins"][5] == 1        # 50/200 and 50/100
    assert "| advec-256^3-f32 | `cfgA` | 50.0 |" in pt.markdown(res)
