"""Launch one configuration of one workload a few times (for profilers).

    python -m paper_2303_12374_gb300.run_config --workload walls256_adv5_diff \
        --dtype f32 --config "zpack:w=4,ly=2,kc=16,ns=8,minb=2" --reps 3

Fills the ghosts once, then calls kl_launch_with_config `reps` times (or
kl_launch with the committed wisdom when --config is "wisdom").  With --time
the launches are timed with CUDA events (after three warm-up launches) and a
JSON line gives the median kernel time, Gpts/s and algorithmic GB/s for each
configuration of a list separated by ';'.  With --diag none|ref, one launch
is followed by `reps` FP64 diagnostics (kl_diag) of ut, without a reference
or against an FP64 copy of it.
"""

from __future__ import annotations

import argparse
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="walls256_adv5_diff")
    ap.add_argument("--dtype", default="f32")
    ap.add_argument("--size", default=None, help="nx,ny,nz (default: the workload's)")
    ap.add_argument("--config", default="wisdom")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--time", action="store_true", help="time the launches (CUDA events)")
    ap.add_argument("--diag", choices=["none", "ref"], default=None,
                    help="after one launch, `reps` kl_diag calls on ut: without a reference, "
                         "or with an FP64 reference field")
    args = ap.parse_args(argv)
    import torch
    from paper_2303_12374_gb300 import kl
    from paper_2303_12374_gb300.tune_cli import build_problem
    size = tuple(int(x) for x in args.size.split(",")) if args.size else None
    ctx = kl.kl_create(0, os.path.join(HERE, "wisdom"))
    try:
        p, op, bufs, outs, fl = build_problem(args.workload, args.dtype, size)
        kl.kl_fill_ghosts(ctx, p.dtype, p.grid, bufs["u"].data_ptr(), bufs["v"].data_ptr(),
                          bufs["w"].data_ptr(), bufs["nu"].data_ptr() if "nu" in bufs else None)
        if args.diag:
            kl.kl_launch(ctx, op, p.grid, fl)
            ref = None
            if args.diag == "ref":
                ref = torch.zeros(p.extent, dtype=torch.float64, device=outs[0].device)
                p.view(ref).copy_(p.view(outs[0]).to(torch.float64))
            for _ in range(args.reps):
                vals = kl.kl_diag(ctx, p.dtype, p.grid, 0, outs[0].data_ptr(),
                                  None if ref is None else ref.data_ptr())
            torch.cuda.synchronize()
            print("diag", list(vals))
        elif args.time:
            import json
            import statistics
            from paper_2303_12374_gb300 import synth
            spec = synth.WORKLOADS[args.workload]
            es = {0: 8, 1: 4, 2: 2, 3: 2}[p.dtype]
            pts = p.nx * p.ny * p.nz
            nbytes = (6 + (1 if spec["diff"] == 2 else 0)) * es * pts
            res = {"workload": args.workload, "dtype": args.dtype, "grid": [p.nx, p.ny, p.nz]}
            for cfg in args.config.split(";"):
                def launch():
                    if cfg == "wisdom":
                        kl.kl_launch(ctx, op, p.grid, fl)
                    else:
                        kl.kl_launch_with_config(ctx, op, cfg, p.grid, fl)
                try:
                    for _ in range(3):
                        launch()
                except kl.KLError as e:          # outside the space for this problem
                    res[cfg] = {"error": str(e)}
                    continue
                ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                      for _ in range(args.reps)]
                for a, b in ev:
                    a.record()
                    launch()
                    b.record()
                torch.cuda.synchronize()
                us = 1e3 * statistics.median(a.elapsed_time(b) for a, b in ev)
                name = json.loads(kl.kl_stats(ctx))["last_config"] if cfg == "wisdom" else cfg
                res[name] = {"us": us, "gpts": pts / us / 1e3, "alg_gbs": nbytes / us / 1e3}
            kl.kl_check(ctx)
            print(json.dumps(res))
        else:
            for _ in range(args.reps):
                if args.config == "wisdom":
                    kl.kl_launch(ctx, op, p.grid, fl)
                else:
                    kl.kl_launch_with_config(ctx, op, args.config, p.grid, fl)
            torch.cuda.synchronize()
            print("ran", args.reps, "launches of", kl.kl_stats(ctx))
    finally:
        kl.kl_destroy(ctx)


if __name__ == "__main__":
    main()
