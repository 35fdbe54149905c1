"""Command-line tuning of a workload (the tuning step of Sec. 4.3).

Builds one of the seeded workloads on the GPU, captures a launch with
kl_capture (Sec. 4.2), tunes the capture with kl_tune and appends the best
configuration to the wisdom file of the op (Sec. 4.4), which kl_launch then
selects at run time (Sec. 4.5).

    python -m paper_2303_12374_gb300.tune_cli --workload walls256_adv5_diff \
        --dtype f32 --wisdom-dir paper_2303_12374_gb300/wisdom \
        --opts "strategy=random family=zpack budget_s=120 max_evals=300" \
        --log tune_walls256_f32.jsonl
"""

from __future__ import annotations

import argparse
import os
import sys
import tempfile
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))


def build_problem(workload: str, dtype: str, size=None):
    import torch
    from paper_2303_12374_gb300 import kl, synth
    from paper_2303_12374_gb300.problem import Problem
    spec = dict(synth.WORKLOADS[workload])
    nx, ny, nz = size if size else (spec["nx"], spec["ny"], spec["nz"])
    stretch = spec.get("stretch", 0.0)
    lz = spec.get("lz", 1.0)
    zh = synth.zfaces(nz, lz, stretch)
    f = synth.velocity_fields(nx, ny, nz, seed=synth.seed_of(spec["index"]), walls=spec["walls"],
                              zh=zh, nu0=1e-3 if spec["diff"] == 2 else None)
    p = Problem(nx, ny, nz, g=spec["g"], dtype=dtype, walls=spec["walls"],
                zh=zh if stretch else None, dz=None if stretch else lz / nz, nu=spec["nu"])
    bufs = {k: p.upload(f[k]) for k in ("u", "v", "w")}
    if spec["diff"] == 2:
        bufs["nu"] = p.upload(f["nu"])
    outs = [p.empty() for _ in range(3)]
    op = kl.Op(spec["adv"], spec["diff"], p.dtype, 0)
    fl = kl.Fields(bufs["u"].data_ptr(), bufs["v"].data_ptr(), bufs["w"].data_ptr(),
                   bufs["nu"].data_ptr() if "nu" in bufs else None,
                   *[o.data_ptr() for o in outs])
    torch.cuda.synchronize()
    return p, op, bufs, outs, fl


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--workload", default="walls256_adv5_diff")
    ap.add_argument("--dtype", default="f32")
    ap.add_argument("--size", default=None, help="nx,ny,nz (default: the workload's)")
    ap.add_argument("--wisdom-dir", default=os.path.join(HERE, "wisdom"))
    ap.add_argument("--opts", default="strategy=random budget_s=60 max_evals=200")
    ap.add_argument("--log", default=None, help="JSON-lines log of every evaluation")
    ap.add_argument("--capture", default=None, help="keep the capture file at this path")
    args = ap.parse_args(argv)

    from paper_2303_12374_gb300 import kl
    size = tuple(int(x) for x in args.size.split(",")) if args.size else None
    ctx = kl.kl_create(0, None)
    try:
        p, op, bufs, outs, fl = build_problem(args.workload, args.dtype, size)
        kl.kl_fill_ghosts(ctx, p.dtype, p.grid, bufs["u"].data_ptr(), bufs["v"].data_ptr(),
                          bufs["w"].data_ptr(), bufs["nu"].data_ptr() if "nu" in bufs else None)
        cap = args.capture or os.path.join(tempfile.mkdtemp(), "capture.klcap")
        t0 = time.time()
        kl.kl_capture(ctx, op, p.grid, fl, cap)
        t_cap = time.time() - t0
        del bufs, outs
        os.makedirs(args.wisdom_dir, exist_ok=True)
        from paper_2303_12374_gb300.problem import Problem  # noqa: F401  (keeps torch alive)
        wisdom = os.path.join(args.wisdom_dir, wisdom_file(op))
        opts = args.opts + (f" log={args.log}" if args.log else "")
        t0 = time.time()
        kl.kl_tune(ctx, cap, opts, wisdom)
        print(f"capture {os.path.getsize(cap) / 1e6:.1f} MB in {t_cap:.2f} s; "
              f"tuning {time.time() - t0:.1f} s -> {wisdom}")
        print(open(wisdom).read().strip().splitlines()[-1])
        if not args.capture:
            os.remove(cap)
    finally:
        kl.kl_destroy(ctx)


def wisdom_file(op) -> str:
    names = {0: "f64", 1: "f32", 2: "bf16", 3: "f16"}
    return (f"tendency_adv{op.adv}_diff{op.diff}_{names[op.dtype]}"
            f"{'_acc' if op.accumulate else ''}.wisdom")


if __name__ == "__main__":
    main()
