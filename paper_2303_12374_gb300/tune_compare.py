"""Random search against Bayesian optimisation on one capture (Sec. 5.3, Fig. 3).

The paper tunes each captured kernel with Kernel Tuner's random search and
Bayesian optimisation and reports how long the latter takes to come within
10 % and 5 % of the optimum (the best configuration after an hour).  This
runs the same comparison with kl_tune's `random` and `bayes` strategies on
one seeded workload: every session replays the same capture, logs every
evaluation, and the summary gives, per strategy and seed, the best time, the
evaluations and seconds until the best is within 10 %, 5 % and 2 % of the
optimum, and the median evaluated time (how strongly the search prefers fast
configurations).  Each session runs in a fresh context, so no compiled kernel
carries over from one session to the next.  The optimum is the best evaluation of
all sessions, or a given reference time (an exhaustive search) if lower.

    python -m paper_2303_12374_gb300.tune_compare --family zpack --evals 100 \
        --seeds 1,2,3 --optimum-us 203.4 --out compare.json
"""

from __future__ import annotations

import argparse
import json
import os
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))


def read_log(path):
    out = []
    for line in open(path):
        e = json.loads(line)
        out.append((e["t_s"], e["time_us"] if e["ok"] and e["time_us"] > 0 else float("inf")))
    return out


def reach(evals, target):
    """(evaluations, seconds) until the best so far is <= target, or (None, None)."""
    best = float("inf")
    for q, (t, us) in enumerate(evals):
        best = min(best, us)
        if best <= target:
            return q + 1, t
    return None, None


def summarise(runs, optimum):
    rows = []
    for (strategy, seed), evals in sorted(runs.items()):
        times = sorted(us for _, us in evals if us < float("inf"))
        best = times[0] if times else float("inf")
        row = {"strategy": strategy, "seed": seed, "evals": len(evals), "best_us": best,
               "seconds": evals[-1][0] if evals else 0.0,
               "median_eval_us": times[len(times) // 2] if times else None,
               "ok": len(times)}
        for pct in (10, 5, 2):
            n, t = reach(evals, optimum * (1 + pct / 100))
            row[f"evals_to_{pct}pct"] = n
            row[f"s_to_{pct}pct"] = t
        rows.append(row)
    return rows


def markdown(rows, optimum):
    def f(x, fmt="{:.1f}"):
        return "-" if x is None else fmt.format(x)
    lines = [f"optimum {optimum:.1f} us", "",
             "| strategy | seed | evals | best (us) | evals/s to 10 % | evals/s to 5 % | "
             "evals/s to 2 % | median evaluated (us) |",
             "|---|---|---|---|---|---|---|---|"]
    for r in rows:
        lines.append(
            f"| {r['strategy']} | {r['seed']} | {r['evals']} | {r['best_us']:.1f} | "
            f"{f(r['evals_to_10pct'], '{}')} / {f(r['s_to_10pct'])} | "
            f"{f(r['evals_to_5pct'], '{}')} / {f(r['s_to_5pct'])} | "
            f"{f(r['evals_to_2pct'], '{}')} / {f(r['s_to_2pct'])} | {f(r['median_eval_us'])} |")
    return "\n".join(lines)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--workload", default="walls256_adv5_diff")
    ap.add_argument("--dtype", default="f32")
    ap.add_argument("--family", default="zpack")
    ap.add_argument("--evals", type=int, default=100)
    ap.add_argument("--budget-s", type=float, default=300)
    ap.add_argument("--seeds", default="1,2,3")
    ap.add_argument("--strategies", default="random,bayes")
    ap.add_argument("--optimum-us", type=float, default=None,
                    help="reference optimum (e.g. of an exhaustive search)")
    ap.add_argument("--out", default=None, help="JSON summary with every session's log")
    args = ap.parse_args(argv)

    from paper_2303_12374_gb300 import kl
    from paper_2303_12374_gb300.tune_cli import build_problem
    work = tempfile.mkdtemp()
    ctx = kl.kl_create(0, None)
    try:
        p, op, bufs, outs, fl = build_problem(args.workload, args.dtype)
        kl.kl_fill_ghosts(ctx, p.dtype, p.grid, bufs["u"].data_ptr(), bufs["v"].data_ptr(),
                          bufs["w"].data_ptr(), bufs["nu"].data_ptr() if "nu" in bufs else None)
        cap = os.path.join(work, "capture.klcap")
        kl.kl_capture(ctx, op, p.grid, fl, cap)
        del bufs, outs, fl
        runs = {}
        for strategy in args.strategies.split(","):
            for seed in (int(s) for s in args.seeds.split(",")):
                log = os.path.join(work, f"{strategy}_{seed}.jsonl")
                wis = os.path.join(work, f"{strategy}_{seed}.wisdom")
                # a fresh context per session: no compiled kernel carries over
                tctx = kl.kl_create(0, None)
                try:
                    kl.kl_tune(tctx, cap, f"strategy={strategy} family={args.family} seed={seed} "
                                          f"max_evals={args.evals} budget_s={args.budget_s} log={log}",
                               wis)
                finally:
                    kl.kl_destroy(tctx)
                runs[(strategy, seed)] = read_log(log)
                print(f"{strategy} seed {seed}: {len(runs[(strategy, seed)])} evals, best "
                      f"{min(us for _, us in runs[(strategy, seed)]):.1f} us", flush=True)
        optimum = min(min(us for _, us in ev) for ev in runs.values())
        if args.optimum_us:
            optimum = min(optimum, args.optimum_us)
        rows = summarise(runs, optimum)
        print(markdown(rows, optimum))
        if args.out:
            with open(args.out, "w") as fh:
                json.dump({"workload": args.workload, "dtype": args.dtype, "family": args.family,
                           "optimum_us": optimum, "rows": rows,
                           "logs": {f"{s}:{k}": v for (s, k), v in runs.items()}}, fh)
        os.remove(cap)
    finally:
        kl.kl_destroy(ctx)


if __name__ == "__main__":
    main()
