"""Launch the LES step's kernels on the 1024 x 1024 x 64 stretched workload
a few times (for profilers): ghost fill of u, v, w, then `reps` times the
Smagorinsky viscosity (with its ghost fill) and the variable-nu tendencies.

    python -m paper_2303_12374_gb300.run_les --reps 3
"""

from __future__ import annotations

import argparse
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--dtype", default="f32")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--cs", type=float, default=0.1)
    args = ap.parse_args(argv)
    import torch
    from paper_2303_12374_gb300 import kl
    from paper_2303_12374_gb300.tune_cli import build_problem
    ctx = kl.kl_create(0, os.path.join(HERE, "wisdom"))
    try:
        p, op, bufs, outs, fl = build_problem("les1024x1024x64_stretched_varnu", args.dtype)
        uvw = [bufs[k].data_ptr() for k in ("u", "v", "w")]
        kl.kl_fill_ghosts(ctx, p.dtype, p.grid, *uvw, None)
        for _ in range(args.reps):
            kl.kl_smagorinsky(ctx, p.dtype, p.grid, args.cs, *uvw, bufs["nu"].data_ptr(), True)
            kl.kl_launch(ctx, op, p.grid, fl)
        torch.cuda.synchronize()
        print(kl.kl_stats(ctx))
    finally:
        kl.kl_destroy(ctx)


if __name__ == "__main__":
    main()
