"""Capture (Sec. 4.2), tuning (Sec. 4.3), wisdom (Sec. 4.4) and run-time
selection (Sec. 4.5) end to end on the GPU, through the C ABI."""

from __future__ import annotations

import json
import os

import numpy as np
import pytest

from gpu_cases import TOL, make_inputs, oracle_ref, rel_err, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture()
def ctx():
    from paper_2303_12374_gb300 import kl
    c = kl.kl_create(0, None)
    yield c
    kl.kl_destroy(c)


def _problem(ctx, nx=48, ny=40, nz=20, dtype=1, diff=1):
    f = make_inputs(nx, ny, nz, seed=17, walls=True, stretch=2.0, var_nu=diff == 2)
    return f, run_gpu(ctx, f, adv=5, diff=diff, dtype=dtype, walls=True, g=3, stretched=True)


def _fields(p, bufs, outs, diff):
    from paper_2303_12374_gb300 import kl
    return kl.Fields(bufs["u"].data_ptr(), bufs["v"].data_ptr(), bufs["w"].data_ptr(),
                     bufs["nu"].data_ptr() if diff == 2 else None, outs["ut"].data_ptr(),
                     outs["vt"].data_ptr(), outs["wt"].data_ptr())


def _header(path):
    head = b""
    with open(path, "rb") as f:
        while not head.endswith(b"END\n"):
            head += f.read(1)
    return head


@pytest.mark.parametrize("diff", [1, 2])
def test_capture_file_holds_definition_and_data(ctx, tmp_path, diff):
    from paper_2303_12374_gb300 import kl
    f, (p, bufs, outs, rin) = _problem(ctx, diff=diff)
    path = str(tmp_path / "c.klcap")
    op = kl.Op(5, diff, p.dtype, 0)
    kl.kl_capture(ctx, op, p.grid, _fields(p, bufs, outs, diff), path)
    head = _header(path)
    nblobs = 4 if diff == 2 else 3
    # size accounting: header + every input buffer in full (ghosts included)
    assert os.path.getsize(path) == len(head) + nblobs * p.extent * 4
    text = head.decode()
    assert f"adv=5 diff={diff} dtype=1" in text and "nx=48 ny=40 nz=20 g=3" in text
    assert "zh=21 " in text and 'device="' in text
    # the data is the buffers as the kernel saw them
    with open(path, "rb") as fh:
        fh.seek(len(head))
        u = np.frombuffer(fh.read(p.extent * 4), dtype=np.float32)
    assert np.array_equal(u, bufs["u"].cpu().numpy())


def test_tune_16bit_storage_with_f32_tendencies(ctx, tmp_path):
    """A capture of an accumulating bf16 op with f32 tendencies carries the f32
    output blobs; tuning replays it and verifies candidates in f32."""
    import torch
    from paper_2303_12374_gb300 import kl
    nx, ny, nz = 40, 24, 12
    f = make_inputs(nx, ny, nz, seed=3, walls=True)
    rng = np.random.default_rng(1)
    t0 = {k: rng.standard_normal((nz, ny, nx)) for k in ("ut", "vt", "wt")}
    p, bufs, outs, rin = run_gpu(ctx, f, adv=5, diff=1, dtype=2, walls=True, g=3,
                                 accumulate=True, t0=t0, out_f32=True)
    op = kl.Op(5, 1, 2, 1, 1)
    cap = str(tmp_path / "c.klcap")
    kl.kl_capture(ctx, op, p.grid, _fields(p, bufs, outs, 1), cap)
    head = _header(cap)
    assert b"out_f32=1" in head
    # u, v, w in bf16, ut, vt, wt in f32
    assert os.path.getsize(cap) == len(head) + 3 * p.extent * 2 + 3 * p.extent * 4
    wpath = str(tmp_path / "tendency_adv5_diff1_bf16.wisdom")
    log = str(tmp_path / "tune.jsonl")
    kl.kl_tune(ctx, cap, f"strategy=random max_evals=5 budget_s=60 seed=2 log={log}", wpath)
    evals = [json.loads(l) for l in open(log)]
    assert any(e["ok"] for e in evals)
    assert all(e["err"] <= 1e-4 for e in evals if e["ok"])


def test_capture_env_hook(ctx, tmp_path, monkeypatch):
    from paper_2303_12374_gb300 import kl
    monkeypatch.setenv("KERNEL_LAUNCHER_CAPTURE", "other,tendency")
    monkeypatch.setenv("KL_CAPTURE_DIR", str(tmp_path))
    f, (p, bufs, outs, rin) = _problem(ctx)
    files = sorted(os.listdir(tmp_path))
    assert files == ["tendency_adv5_diff1_f32_48x40x20_zbc1.klcap"]


def test_tune_writes_wisdom_that_launch_selects(ctx, tmp_path, oracle_mod):
    from paper_2303_12374_gb300 import kl
    f, (p, bufs, outs, rin) = _problem(ctx)
    op = kl.Op(5, 1, p.dtype, 0)
    cap = str(tmp_path / "c.klcap")
    kl.kl_capture(ctx, op, p.grid, _fields(p, bufs, outs, 1), cap)
    wdir = tmp_path / "wisdom"
    wdir.mkdir()
    wpath = str(wdir / "tendency_adv5_diff1_f32.wisdom")
    log = str(tmp_path / "tune.jsonl")
    kl.kl_tune(ctx, cap, f"strategy=random max_evals=6 budget_s=60 seed=3 log={log}", wpath)
    lines = [l for l in open(wpath) if not l.startswith("#")]
    assert len(lines) == 1 and "speedup=" in lines[0] and "strategy=random" in lines[0]
    evals = [json.loads(l) for l in open(log)]
    assert len(evals) == 6 and any(e["ok"] for e in evals)
    rec = dict(tok.split("=", 1) for tok in lines[0].replace('"', "").split() if "=" in tok)
    # a fresh context reading that wisdom directory picks the record (rule 1)
    c2 = kl.kl_create(0, str(wdir))
    try:
        fl = _fields(p, bufs, outs, 1)
        for o in outs.values():
            o.zero_()
        kl.kl_launch(c2, op, p.grid, fl)
        import torch
        torch.cuda.synchronize()
        st = json.loads(kl.kl_stats(c2))
        assert st["last_config"] == kl.kl_config_normalize(op, rec["config"])
        assert list(st["rules"].values()) == [1]
        ref = oracle_ref(oracle_mod, rin, f["zh"], adv=5, diff=1, walls=True, g=3)
        for name, r in zip(("ut", "vt", "wt"), ref):
            assert rel_err(p.download(outs[name]), r) <= TOL[1]
        # first launch: the four stages of Sec. 5.6 were timed
        assert st["stage_ms"]["nvrtc"] > 0 and st["cache_misses"] >= 1
    finally:
        kl.kl_destroy(c2)


def test_tune_resumes_from_its_log(ctx, tmp_path):
    from paper_2303_12374_gb300 import kl
    f, (p, bufs, outs, rin) = _problem(ctx, nx=32, ny=32, nz=16)
    op = kl.Op(5, 1, p.dtype, 0)
    cap = str(tmp_path / "c.klcap")
    kl.kl_capture(ctx, op, p.grid, _fields(p, bufs, outs, 1), cap)
    log = str(tmp_path / "tune.jsonl")
    w = str(tmp_path / "w.wisdom")
    kl.kl_tune(ctx, cap, f"strategy=local max_evals=4 seed=5 log={log}", w)
    first = [json.loads(l)["config"] for l in open(log)]
    kl.kl_tune(ctx, cap, f"strategy=local max_evals=8 seed=5 log={log}", w)
    allc = [json.loads(l)["config"] for l in open(log)]
    assert len(first) == 4 and len(allc) == 8
    assert allc[:4] == first and len(set(allc)) == 8     # nothing evaluated twice
    assert sum(1 for l in open(w) if not l.startswith("#")) == 2


def test_tune_rejects_bad_options(ctx, tmp_path):
    from paper_2303_12374_gb300 import kl
    with pytest.raises(kl.KLError) as e:
        kl.kl_tune(ctx, str(tmp_path / "none.klcap"), "strategy=annealing", str(tmp_path / "w"))
    assert e.value.status == -1
    with pytest.raises(kl.KLError) as e:
        kl.kl_tune(ctx, str(tmp_path / "none.klcap"), "strategy=random", str(tmp_path / "w"))
    assert e.value.status == -4


@pytest.mark.parametrize("family", ["zpack", "all"])
def test_bayes_tuning(ctx, tmp_path, family):
    """strategy=bayes: an initial random design of 8, then one surrogate-chosen
    candidate per evaluation; nothing is evaluated twice, every candidate is
    verified, and the record names the strategy."""
    from paper_2303_12374_gb300 import kl
    f, (p, bufs, outs, rin) = _problem(ctx)
    op = kl.Op(5, 1, p.dtype, 0)
    cap = str(tmp_path / "c.klcap")
    kl.kl_capture(ctx, op, p.grid, _fields(p, bufs, outs, 1), cap)
    log = str(tmp_path / "tune.jsonl")
    w = str(tmp_path / "w.wisdom")
    kl.kl_tune(ctx, cap, f"strategy=bayes family={family} max_evals=20 budget_s=120 seed=7 "
                         f"log={log}", w)
    evals = [json.loads(l) for l in open(log)]
    confs = [e["config"] for e in evals]
    assert len(confs) == 20 and len(set(confs)) == 20
    assert sum(e["ok"] for e in evals) >= 15
    assert all(e["err"] <= 1e-4 for e in evals if e["ok"])     # the tuner's f32 tolerance
    if family == "zpack":
        assert all(c.startswith("zpack:") for c in confs)
    lines = [l for l in open(w) if not l.startswith("#")]
    assert len(lines) == 1 and "strategy=bayes" in lines[0]
