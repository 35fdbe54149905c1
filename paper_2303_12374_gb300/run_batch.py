"""Launch the 64-grid batch a few times (for profilers): the seeded uneven
grids of the batched workload, ghosts filled once, then `reps` calls of
kl_launch_batched (one launch per configuration class, replayed as one CUDA
graph), or, with --separate, 64 separate kl_launch calls with the same
wisdom selection.

    python -m paper_2303_12374_gb300.run_batch --reps 3
    python -m paper_2303_12374_gb300.run_batch --reps 3 --separate

Prints the configuration classes of the batch (a configuration and its
number of grids), the record each grid selects in a single launch, and the
context statistics.
"""

from __future__ import annotations

import argparse
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--separate", action="store_true")
    args = ap.parse_args(argv)
    import torch
    from paper_2303_12374_gb300 import kl, synth
    from paper_2303_12374_gb300.problem import Problem
    spec = synth.WORKLOADS["batch64_uneven"]
    sizes = synth.batch_sizes(synth.seed_of(spec["index"]), spec["count"])
    ctx = kl.kl_create(0, os.path.join(HERE, "wisdom"))
    try:
        probs = []
        for q, (nx, ny, nz) in enumerate(sizes):
            f = synth.velocity_fields(nx, ny, nz, seed=synth.seed_of(spec["index"]) * 1000 + q,
                                      walls=True)
            p = Problem(nx, ny, nz, g=spec["g"], dtype="f32", walls=True, dz=1.0 / nz,
                        nu=spec["nu"])
            bufs = [p.upload(f[k]) for k in ("u", "v", "w")]
            outs = [p.empty() for _ in range(3)]
            fl = kl.Fields(*[b.data_ptr() for b in bufs], None, *[o.data_ptr() for o in outs])
            kl.kl_fill_ghosts(ctx, p.dtype, p.grid, *[b.data_ptr() for b in bufs], None)
            probs.append((p, bufs, outs, fl))
        op = kl.Op(5, 1, 1, 0)
        classes = {}
        for p, _, _, fl in probs:
            kl.kl_launch(ctx, op, p.grid, fl)
            cfg = json.loads(kl.kl_stats(ctx))["last_config"]
            classes.setdefault(cfg, []).append(f"{p.nx}x{p.ny}x{p.nz}")
        torch.cuda.synchronize()
        grids = [pr[0].grid for pr in probs]
        fields = [pr[3] for pr in probs]
        for _ in range(args.reps):
            if args.separate:
                for p, _, _, fl in probs:
                    kl.kl_launch(ctx, op, p.grid, fl)
            else:
                kl.kl_launch_batched(ctx, op, grids, fields)
        torch.cuda.synchronize()
        kl.kl_check(ctx)
        print(json.dumps({"batch_classes": json.loads(kl.kl_stats(ctx))["last_batch"],
                          "single_launch_classes": {k: len(v) for k, v in classes.items()},
                          "grids": {k: v for k, v in classes.items()}}))
        print(kl.kl_stats(ctx))
    finally:
        kl.kl_destroy(ctx)


if __name__ == "__main__":
    main()
