"""Batched execution: many grids of uneven sizes under the configuration of
the wisdom record nearest to the batch's total point count (grids it does
not fit take their own nearest-size record, Sec. 4.5 and Sec. 6 fuzzy
matching); one launch per configuration class, one CUDA graph."""

from __future__ import annotations

import json

import numpy as np
import pytest

from gpu_cases import TOL, make_inputs, oracle_ref, rel_err

pytestmark = pytest.mark.gpu

SIZES = [(40, 36, 20), (64, 48, 16), (33, 70, 24), (96, 40, 12), (48, 48, 32), (17, 23, 9)]


def _setup(dtype, stretched):
    from paper_2303_12374_gb300 import kl
    from paper_2303_12374_gb300.problem import Problem
    probs = []
    for q, (nx, ny, nz) in enumerate(SIZES):
        f = make_inputs(nx, ny, nz, seed=300 + q, walls=True, stretch=2.0 if stretched else 0.0)
        p = Problem(nx, ny, nz, g=3, dtype=dtype, walls=True, zh=f["zh"] if stretched else None,
                    dz=None if stretched else 1.0 / nz, nu=1e-3)
        bufs = [p.upload(f[k]) for k in ("u", "v", "w")]
        outs = [p.empty() for _ in range(3)]
        fl = kl.Fields(*[b.data_ptr() for b in bufs], None, *[o.data_ptr() for o in outs])
        probs.append((f, p, bufs, outs, fl))
    return probs


def _wisdom(path, dtype_tag, records):
    with open(path, "w") as fh:
        fh.write("# batch test wisdom\n")
        for (nx, ny, nz), cfg in records:
            fh.write(f'device="NVIDIA GB300" cc=10.3 zbc=1 nx={nx} ny={ny} nz={nz} '
                     f'config="{cfg}" time_us=1.0\n')


@pytest.mark.parametrize("dtype,tag", [(1, "f32"), (0, "f64"), (2, "bf16")])
@pytest.mark.parametrize("stretched", [False, True])
def test_batched_matches_oracle_and_single_launches(tmp_path, oracle_mod, dtype, tag, stretched):
    import torch
    from paper_2303_12374_gb300 import kl
    small = "zmarch:bx=32,by=4,px=1,py=2,kc=8,ns=8,minb=2"
    big = ("zpack:w=4,ly=2,kc=16,ns=8,minb=2" if dtype != 0
           else "direct:bx=64,by=2,tx=1,ty=2,uy=1,cy=1,minb=2")
    _wisdom(tmp_path / f"tendency_adv5_diff1_{tag}.wisdom", tag,
            [((32, 32, 16), small), ((80, 48, 24), big)])
    ctx = kl.kl_create(0, str(tmp_path))
    try:
        probs = _setup(dtype, stretched)
        op = kl.Op(5, 1, probs[0][1].dtype, 0)
        for f, p, bufs, outs, fl in probs:
            kl.kl_fill_ghosts(ctx, p.dtype, p.grid, *[b.data_ptr() for b in bufs], None)
        grids = [pr[1].grid for pr in probs]
        fields = [pr[4] for pr in probs]
        kl.kl_launch_batched(ctx, op, grids, fields)
        torch.cuda.synchronize()
        got = [[p.download(o) for o in outs] for f, p, bufs, outs, fl in probs]
        st = json.loads(kl.kl_stats(ctx))
        assert st["tables"] >= 1
        # the same batch again reuses its device tables and replays its graph
        kl.kl_launch_batched(ctx, op, grids, fields)
        torch.cuda.synchronize()
        st2 = json.loads(kl.kl_stats(ctx))
        assert st2["tables"] == st["tables"]
        assert st2["graphs"] == 1 and st2["graph_replays"] == 1
        again = [[p.download(o) for o in outs] for f, p, bufs, outs, fl in probs]
        for a3, b3 in zip(got, again):
            for a, b in zip(a3, b3):
                assert np.array_equal(a, b)
        for (f, p, bufs, outs, fl), g3 in zip(probs, got):
            rin = {k: p.rounded(f[k]) for k in ("u", "v", "w")}
            ref = oracle_ref(oracle_mod, rin, f["zh"], adv=5, diff=1, walls=True, g=3)
            for name, a, r in zip(("ut", "vt", "wt"), g3, ref):
                assert rel_err(a, r) <= TOL[p.dtype], (p.nx, p.ny, p.nz, name)
        # single launches with the wisdom-selected configuration give the same fields
        for (f, p, bufs, outs, fl), g3 in zip(probs, got):
            for o in outs:
                o.zero_()
            kl.kl_launch(ctx, op, p.grid, fl)
            torch.cuda.synchronize()
            for o, a in zip(outs, g3):
                b = p.download(o)
                assert np.abs(a - b).max() <= TOL[p.dtype] * max(np.abs(b).max(), 1e-300)
    finally:
        kl.kl_destroy(ctx)


def test_batched_inside_a_caller_capture(tmp_path):
    """A batch seen before can be recorded into the caller's own CUDA graph:
    its launches join the caller's capture instead of a graph of its own."""
    import torch
    from paper_2303_12374_gb300 import kl
    _wisdom(tmp_path / "tendency_adv5_diff1_f32.wisdom", "f32",
            [((32, 32, 16), "zmarch:bx=32,by=4,px=1,py=2,kc=8,ns=8,minb=2"),
             ((80, 48, 24), "zpack:w=4,ly=2,kc=16,ns=8,minb=2")])
    ctx = kl.kl_create(0, str(tmp_path))
    try:
        probs = _setup(1, False)
        op = kl.Op(5, 1, 1, 0)
        for f, p, bufs, outs, fl in probs:
            kl.kl_fill_ghosts(ctx, p.dtype, p.grid, *[b.data_ptr() for b in bufs], None)
        grids = [pr[1].grid for pr in probs]
        fields = [pr[4] for pr in probs]
        kl.kl_launch_batched(ctx, op, grids, fields)        # tables, kernels, own graph
        torch.cuda.synchronize()
        want = [[p.download(o) for o in outs] for f, p, bufs, outs, fl in probs]
        for f, p, bufs, outs, fl in probs:
            for o in outs:
                o.zero_()
        torch.cuda.synchronize()
        side = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side):
            kl.kl_launch_batched(ctx, op, grids, fields, side.cuda_stream)
        g.replay()
        torch.cuda.synchronize()
        got = [[p.download(o) for o in outs] for f, p, bufs, outs, fl in probs]
        for a3, b3 in zip(want, got):
            for a, b in zip(a3, b3):
                assert np.array_equal(a, b)
    finally:
        kl.kl_destroy(ctx)


def test_batched_rejects_bad_grid_before_launching():
    from paper_2303_12374_gb300 import kl
    ctx = kl.kl_create(0, None)
    try:
        probs = _setup(1, False)[:2]
        grids = [pr[1].grid for pr in probs]
        bad = kl.Grid.from_buffer_copy(grids[1])
        bad.sj = 4      # row pitch smaller than a padded row
        with pytest.raises(kl.KLError) as e:
            kl.kl_launch_batched(ctx, kl.Op(5, 1, 1, 0), [grids[0], bad],
                                 [probs[0][4], probs[1][4]])
        assert e.value.status == -7 and "grid 1" in str(e.value)
    finally:
        kl.kl_destroy(ctx)
