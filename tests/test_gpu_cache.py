"""The on-disk cubin cache on the GPU: a second context with the same
directory loads every variant from disk (no NVRTC), produces the same bits
and matches the oracle; a cache filled ahead of time on the host
(kl_cache_prepare) is used by a context's first launch; batched launches
cache their variant too."""

from __future__ import annotations

import json
import os

import numpy as np
import pytest

from gpu_cases import TOL, make_inputs, oracle_ref, rel_err, run_gpu

pytestmark = pytest.mark.gpu

WISDOM = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                      "paper_2303_12374_gb300", "wisdom")


def _run(ctx, f, step=True):
    p, bufs, outs, rin = run_gpu(ctx, f, adv=5, diff=1, dtype=1, walls=True, g=3, step=step)
    return p, [p.download(outs[k]) for k in ("ut", "vt", "wt")], rin


def test_second_context_loads_from_disk(tmp_path, oracle_mod):
    from paper_2303_12374_gb300 import kl
    f = make_inputs(72, 64, 48, seed=5, walls=True)
    res, stats = [], []
    for _ in range(2):
        ctx = kl.kl_create(0, WISDOM)
        try:
            kl.kl_set_cache_dir(ctx, str(tmp_path))
            p, out, rin = _run(ctx, f)
            res.append(out)
            stats.append(json.loads(kl.kl_stats(ctx)))
        finally:
            kl.kl_destroy(ctx)
    first, second = stats
    assert first["disk_cache"] == {"on": True, "hits": 0, "writes": 1, "read_ms": 0.0}
    assert first["stage_ms"]["nvrtc"] > 0
    assert second["disk_cache"]["hits"] == 1 and second["disk_cache"]["writes"] == 0
    assert second["stage_ms"]["nvrtc"] == 0 and second["last_config"] == first["last_config"]
    assert second["last_config"].startswith("zpack:")
    for a, b in zip(*res):
        assert np.array_equal(a, b)
    ref = oracle_ref(oracle_mod, rin, f["zh"], adv=5, diff=1, walls=True, g=3)
    for a, r in zip(res[1], ref):
        assert rel_err(a, r) <= TOL[1]


def test_prepared_cache_and_environment(tmp_path, monkeypatch):
    from paper_2303_12374_gb300 import kl
    d = str(tmp_path)
    op = kl.Op(5, 1, 1, 0)
    cfg = "zpack:w=4,ly=2,kc=8,ns=8,minb=2"
    assert kl.kl_cache_prepare(d, op, cfg, 1, 1) is False
    monkeypatch.setenv("KL_CACHE_DIR", d)
    ctx = kl.kl_create(0, None)
    try:
        f = make_inputs(70, 40, 20, seed=9, walls=True)
        run_gpu(ctx, f, adv=5, diff=1, dtype=1, walls=True, g=3, config=cfg)
        st = json.loads(kl.kl_stats(ctx))
        assert st["disk_cache"]["on"] and st["disk_cache"]["hits"] == 1
        assert st["stage_ms"]["nvrtc"] == 0
        kl.kl_set_cache_dir(ctx, None)
        assert json.loads(kl.kl_stats(ctx))["disk_cache"]["on"] is False
        with pytest.raises(kl.KLError) as e:
            kl.kl_set_cache_dir(ctx, str(tmp_path / "nope"))
        assert e.value.status == -4
    finally:
        kl.kl_destroy(ctx)
