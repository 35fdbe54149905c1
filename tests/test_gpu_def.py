"""User-defined tunable kernels on the GPU: launch of every configuration of a
vector add (exact), capture -> tune -> wisdom -> run-time selection (Sec. 4.2
to 4.5), a kernel with dynamic shared memory and an in/out buffer (tuning
restores it before every candidate), a templated kernel, and the on-disk
cubin cache."""

from __future__ import annotations

import json
import os

import numpy as np
import pytest

from test_def_host import SCALE, VADD, vadd_def

pytestmark = pytest.mark.gpu

SMOOTH = r"""
extern "C" __global__ void smooth(const float *x, float *y, int n, float w)
{
    // y += w (x[i-1] + 2 x[i] + x[i+1]), zero outside 0..n-1, staged in shared memory
    extern __shared__ float s[];
    long i = (long)blockIdx.x * BLOCK + threadIdx.x;
    s[threadIdx.x + 1] = i < n ? x[i] : 0.f;
    if (threadIdx.x == 0) s[0] = (i > 0 && i - 1 < n) ? x[i - 1] : 0.f;
    if (threadIdx.x == BLOCK - 1) s[BLOCK + 1] = i + 1 < n ? x[i + 1] : 0.f;
    __syncthreads();
    if (i < n) y[i] += w * (s[threadIdx.x] + 2.f * s[threadIdx.x + 1] + s[threadIdx.x + 2]);
}
"""


@pytest.fixture()
def ctx():
    from paper_2303_12374_gb300 import kl
    c = kl.kl_create(0, None)
    yield c
    kl.kl_destroy(c)


def _vadd_data(n, seed=0):
    import torch
    g = torch.Generator(device="cuda").manual_seed(seed)
    a = torch.randn(n, generator=g, device="cuda")
    b = torch.randn(n, generator=g, device="cuda")
    return a, b, torch.full((n,), float("nan"), device="cuda")


def _smooth_ref(x, y0, w):
    import torch
    xp = torch.nn.functional.pad(x.double(), (1, 1))
    return y0.double() + w * (xp[:-2] + 2 * xp[1:-1] + xp[2:])


def test_vadd_every_configuration(ctx):
    import torch
    d = vadd_def()
    n = 1_000_003
    a, b, c = _vadd_data(n)
    raw, valid = d.space_size()
    ran = 0
    for idx in range(raw):
        cfg, ok = d.config_at(idx)
        if not ok:
            continue
        c.fill_(float("nan"))
        d.launch_config(ctx, cfg, (n,), [("in", a), ("in", b), ("out", c), ("i32", n)])
        torch.cuda.synchronize()
        assert torch.equal(c, a + b), cfg
        ran += 1
    assert ran == valid == 23


def test_capture_tune_select(ctx, tmp_path):
    import torch
    from paper_2303_12374_gb300 import kl
    d = vadd_def()
    n = 1 << 22
    a, b, c = _vadd_data(n, seed=1)
    args = [("in", a), ("in", b), ("out", c), ("i32", n)]
    cap = str(tmp_path / "vadd.klcap")
    d.capture(ctx, (n,), args, cap)
    head = open(cap, "rb").read(400)
    assert head.startswith(b"KLDEFCAP1\nname vadd\nfunction vadd\nproblem 4194304 1 1\nnargs 4\n")
    # inputs and the scalar are stored, the output is not
    assert os.path.getsize(cap) - head.index(b"END\n") - 4 == 2 * 4 * n + 4
    wdir = tmp_path / "wisdom"
    wdir.mkdir()
    log = str(tmp_path / "tune.jsonl")
    d.tune(ctx, cap, f"strategy=exhaustive max_evals=100 log={log}", str(wdir / "vadd.wisdom"))
    evals = [json.loads(l) for l in open(log)]
    assert len(evals) == 23 and all(e["ok"] for e in evals)
    assert len({e["config"] for e in evals}) == 23
    rec = [l for l in open(wdir / "vadd.wisdom") if not l.startswith("#")]
    assert len(rec) == 1 and "kernel=vadd" in rec[0] and "strategy=exhaustive" in rec[0]
    tuned = rec[0].split('config="')[1].split('"')[0]
    c2 = kl.kl_create(0, str(wdir))
    try:
        c.fill_(float("nan"))
        d.launch(c2, (n,), args)
        torch.cuda.synchronize()
        assert torch.equal(c, a + b)
        assert d.selected() == (tuned, 1)
        # another size: the nearest record (rule 2), still exact
        m = 777_777
        d.launch(c2, (m,), [("in", a), ("in", b), ("out", c), ("i32", m)])
        torch.cuda.synchronize()
        assert d.selected() == (tuned, 2)
        assert torch.equal(c[:m], (a + b)[:m])
    finally:
        kl.kl_destroy(c2)


def test_shared_memory_and_inout_buffer(ctx, tmp_path):
    import torch
    from paper_2303_12374_gb300 import kl
    d = kl.KernelDef("smooth", SMOOTH, "smooth")
    d.param("BLOCK", [64, 128, 256, 512, 1024], 256)
    d.geometry(block=("BLOCK",), grid=("div_ceil(problem_x, BLOCK)",),
               shared_memory="(BLOCK + 2) * 4")
    n, w = 300_001, 0.25
    g = torch.Generator(device="cuda").manual_seed(3)
    x = torch.randn(n, generator=g, device="cuda")
    y0 = torch.randn(n, generator=g, device="cuda")
    ref = _smooth_ref(x, y0, w)
    for blk in (64, 1024):
        y = y0.clone()
        d.launch_config(ctx, f"BLOCK={blk}", (n,), [("in", x), ("inout", y), ("i32", n), ("f32", w)])
        torch.cuda.synchronize()
        assert float((y.double() - ref).abs().max()) <= 1e-6 * float(ref.abs().max())
    y = y0.clone()
    cap = str(tmp_path / "smooth.klcap")
    d.capture(ctx, (n,), [("in", x), ("inout", y), ("i32", n), ("f32", w)], cap)
    log = str(tmp_path / "t.jsonl")
    d.tune(ctx, cap, f"strategy=bayes max_evals=5 log={log}", str(tmp_path / "smooth.wisdom"))
    evals = [json.loads(l) for l in open(log)]
    # every candidate started from the captured y (else the sums would drift)
    assert len(evals) == 5 and all(e["ok"] for e in evals), evals
    assert y.equal(y0)          # the caller's buffers are not touched by tuning


def test_template_kernel(ctx):
    import torch
    from paper_2303_12374_gb300 import kl
    d = kl.KernelDef("scalep", SCALE, "scale<FACTOR>").param("FACTOR", [2, 4], 2)
    d.param("BLOCK", [128, 256], 128).geometry(block=("BLOCK",), grid=("div_ceil(problem_x, BLOCK)",))
    n = 5000
    x = torch.arange(n, device="cuda", dtype=torch.float32)
    d.launch_config(ctx, "FACTOR=4,BLOCK=256", (n,), [("inout", x), ("i32", n)])
    d.launch(ctx, (n,), [("inout", x), ("i32", n)])          # no wisdom: the default, FACTOR=2
    torch.cuda.synchronize()
    assert torch.equal(x, 8 * torch.arange(n, device="cuda", dtype=torch.float32))
    assert d.selected() == ("FACTOR=2,BLOCK=128", 5)


def test_disk_cache_and_argument_errors(tmp_path):
    import torch
    from paper_2303_12374_gb300 import kl
    d = vadd_def()
    n = 4096
    a, b, c = _vadd_data(n, seed=2)
    args = [("in", a), ("in", b), ("out", c), ("i32", n)]
    stats = []
    for _ in range(2):
        cx = kl.kl_create(0, None)
        try:
            kl.kl_set_cache_dir(cx, str(tmp_path))
            d.launch_config(cx, "BLOCK=64,ELEMS=2", (n,), args)
            torch.cuda.synchronize()
            stats.append(json.loads(kl.kl_stats(cx)))
            if len(stats) == 2:
                with pytest.raises(kl.KLError):           # no grid for an empty problem
                    d.launch_config(cx, "default", (0,), args)
                with pytest.raises(kl.KLError):           # restriction
                    d.launch_config(cx, "BLOCK=1024,ELEMS=8", (n,), args)
                bad = (kl.Arg * 1)(kl.Arg(None, 4, 0, 0))  # scalar without a value
                assert kl.load().kl_def_launch_config(cx, d.h, b"default", kl._problem((n,)), 1,
                                                      bad, None) == -1
        finally:
            kl.kl_destroy(cx)
    assert stats[0]["disk_cache"]["writes"] == 1 and stats[0]["stage_ms"]["nvrtc"] > 0
    assert stats[1]["disk_cache"]["hits"] == 1 and stats[1]["stage_ms"]["nvrtc"] == 0
    assert torch.equal(c, a + b)
