"""Launch one configuration of one workload a few times (for profilers).

    python -m paper_2303_12374_gb300.run_config --workload walls256_adv5_diff \
        --dtype f32 --config "zpack:w=4,ly=2,kc=16,ns=8,minb=2" --reps 3

Fills the ghosts once, then calls kl_launch_with_config `reps` times (or
kl_launch with the committed wisdom when --config is "wisdom").
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
