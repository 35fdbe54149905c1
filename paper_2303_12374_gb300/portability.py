"""Search-space distributions, configuration portability and the PPM on one
GPU model (the study of Sec. 5.4 and 5.5, Fig. 4-5, Tables 3-4).

A scenario is a kernel, a grid and a precision (the paper adds the GPU; one
GPU model is measured here).  The two kernels mirror the paper's:
`advec` is 5th-order flux-form advection of u, v, w alone (advec_u), `diff`
the variable-nu stress-form diffusion of u, v, w alone (diff_uvw).  All
grids have z walls and three ghost cells.

Pass 1, per scenario: capture one launch, then tune it twice in fresh
contexts.  The first session is `random`; its evaluated times relative to the
scenario's optimum give the histogram of Fig. 4.  The second is `bayes`.  The
fastest configuration of the two sessions becomes the scenario's tuned
configuration.

Pass 2, per scenario B: time the default configuration and every scenario's
tuned configuration on B, verifying each output against the default's.  This
gives the matrix of Fig. 5: each configuration's fraction of B's best-known
time.  A configuration outside B's space (for example too much shared memory
for f64) counts as unsupported.

Per configuration and per kernel, the PPM of Pennycook et al. is the
harmonic mean of its fractions over the kernel's scenarios, and 0 if any
scenario does not support it.  Run-time selection of each scenario's own
record scores 1 by construction.

Inputs are seeded normal fields generated on the device; nu is
1e-3 (1 + U[0, 1)).  Kernel times do not depend on the values.

    python -m paper_2303_12374_gb300.portability --out portability.json
"""

from __future__ import annotations

import argparse
import json
import os
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

KERNELS = {"advec": (5, 0), "diff": (0, 2)}
GRIDS = {"256^3": (256, 256, 256), "512x512x256": (512, 512, 256), "1024x1024x64": (1024, 1024, 64)}
PRECISIONS = {"f32": 1, "f64": 0}
TOL = {1: 1e-4, 0: 1e-10}


def scenarios(kernels=None, grids=None, precisions=None):
    return [(k, g, d) for k in (kernels or KERNELS) for g in (grids or GRIDS)
            for d in (precisions or PRECISIONS)]


def label(s) -> str:
    return "-".join(s)


def ppm(fractions) -> float:
    """Harmonic mean of the efficiencies; 0 if any scenario is unsupported (None)."""
    if not fractions or any(f is None or f <= 0 for f in fractions):
        return 0.0
    return len(fractions) / sum(1.0 / f for f in fractions)


def histogram(fractions, bins=10):
    """Counts of fractions of optimum in [0, 0.1), ..., [0.9, 1.0] (1.0 and above in the top bin)."""
    out = [0] * bins
    for f in fractions:
        out[min(bins - 1, max(0, int(f * bins)))] += 1
    return out


def make_problem(sc, seed):
    import torch
    from paper_2303_12374_gb300 import kl
    from paper_2303_12374_gb300.problem import Problem
    k, gname, dname = sc
    adv, diff = KERNELS[k]
    nx, ny, nz = GRIDS[gname]
    p = Problem(nx, ny, nz, g=3, dtype=dname, walls=True, dz=1.0 / nz, nu=1e-3)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    bufs = {}
    for name in ("u", "v", "w"):
        b = p.empty()
        p.view(b).copy_(torch.randn((nz, ny, nx), generator=gen, device="cuda", dtype=p.tdtype))
        bufs[name] = b
    if diff == 2:
        b = p.empty()
        p.view(b).copy_(1e-3 * (1 + torch.rand((nz, ny, nx), generator=gen, device="cuda",
                                               dtype=p.tdtype)))
        bufs["nu"] = b
    outs = [p.empty() for _ in range(3)]
    op = kl.Op(adv, diff, p.dtype, 0)
    fl = kl.Fields(bufs["u"].data_ptr(), bufs["v"].data_ptr(), bufs["w"].data_ptr(),
                   bufs["nu"].data_ptr() if "nu" in bufs else None, *[o.data_ptr() for o in outs])
    return p, op, bufs, outs, fl


def read_log(path):
    out = []
    for line in open(path):
        e = json.loads(line)
        out.append((e["config"], e["time_us"] if e["ok"] and e["time_us"] > 0 else None))
    return out


def tune_pass(sc, seed, work, rand_evals, bayes_evals):
    from paper_2303_12374_gb300 import kl
    ctx = kl.kl_create(0, None)
    cap = os.path.join(work, label(sc).replace("^", "") + ".klcap")
    try:
        p, op, bufs, outs, fl = make_problem(sc, seed)
        kl.kl_fill_ghosts(ctx, p.dtype, p.grid, bufs["u"].data_ptr(), bufs["v"].data_ptr(),
                          bufs["w"].data_ptr(), bufs["nu"].data_ptr() if "nu" in bufs else None)
        kl.kl_capture(ctx, op, p.grid, fl, cap)
        del p, bufs, outs, fl
    finally:
        kl.kl_destroy(ctx)
    res = {}
    for strategy, n in (("random", rand_evals), ("bayes", bayes_evals)):
        log = cap + f".{strategy}.jsonl"
        tctx = kl.kl_create(0, None)
        try:
            kl.kl_tune(tctx, cap, f"strategy={strategy} family=all seed={seed} max_evals={n} "
                                  f"budget_s=600 log={log}", cap + f".{strategy}.wisdom")
        finally:
            kl.kl_destroy(tctx)
        res[strategy] = read_log(log)
    os.remove(cap)
    return res


def cross_pass(sc, seed, configs, reps=20, warm=3):
    """{config: (median us, relative error vs default) or None if unsupported}."""
    import torch
    from paper_2303_12374_gb300 import kl
    ctx = kl.kl_create(0, None)
    out = {}
    try:
        p, op, bufs, outs, fl = make_problem(sc, seed)
        kl.kl_fill_ghosts(ctx, p.dtype, p.grid, bufs["u"].data_ptr(), bufs["v"].data_ptr(),
                          bufs["w"].data_ptr(), bufs["nu"].data_ptr() if "nu" in bufs else None)
        kl.kl_launch_with_config(ctx, op, "default", p.grid, fl)
        torch.cuda.synchronize()
        ref = [p.view(o).to(torch.float64).clone() for o in outs]
        scale = max(float(r.abs().max()) for r in ref)
        s = torch.cuda.current_stream()
        for cfg in configs:
            try:
                for o in outs:
                    o.zero_()
                kl.kl_launch_with_config(ctx, op, cfg, p.grid, fl, s.cuda_stream)
                torch.cuda.synchronize()
            except kl.KLError:
                out[cfg] = None
                continue
            err = max(float((p.view(o).to(torch.float64) - r).abs().max()) for o, r in zip(outs, ref))
            err /= scale
            for _ in range(warm):
                kl.kl_launch_with_config(ctx, op, cfg, p.grid, fl, s.cuda_stream)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(reps)]
            for a, b in ev:
                a.record(s)
                kl.kl_launch_with_config(ctx, op, cfg, p.grid, fl, s.cuda_stream)
                b.record(s)
            torch.cuda.synchronize()
            ms = sorted(a.elapsed_time(b) for a, b in ev)
            out[cfg] = (1e3 * ms[len(ms) // 2], err)
    finally:
        kl.kl_destroy(ctx)
    return out


def analyse(scs, tuned, logs, cross):
    """Matrix, PPM rows and histogram summaries from the two passes."""
    names = [label(s) for s in scs]
    optimum = {}
    for s in scs:
        ts = [v[0] for v in cross[label(s)].values() if v is not None and v[1] <= TOL[PRECISIONS[s[2]]]]
        optimum[label(s)] = min(ts)
    def frac(cfg, s):
        v = cross[label(s)].get(cfg)
        if v is None or v[1] > TOL[PRECISIONS[s[2]]]:
            return None
        return optimum[label(s)] / v[0]
    matrix = {n: {m: frac(tuned[n], s) for m, s in zip(names, scs)} for n in names}
    default = {m: frac("default", s) for m, s in zip(names, scs)}
    ppm_rows = {}
    for k in sorted({s[0] for s in scs}):
        ks = [s for s in scs if s[0] == k]
        rows = [("(default configuration)", [default[label(s)] for s in ks])]
        for s in ks:
            rows.append((f"tuned for {label(s)}", [matrix[label(s)][label(t)] for t in ks]))
        rows.append(("run-time selection (own record)", [1.0] * len(ks)))
        ppm_rows[k] = [{"config": r, "best": max((f for f in fs if f), default=0.0),
                        "worst": min((f if f else 0.0) for f in fs), "ppm": ppm(fs)} for r, fs in rows]
    hist = {}
    for s in scs:
        n = label(s)
        rand = [t for _, t in logs[n]["random"] if t]
        best = min(rand + [t for _, t in logs[n]["bayes"] if t])
        fr = [best / t for t in rand]
        hist[n] = {"evals": len(logs[n]["random"]), "ok": len(rand), "bins": histogram(fr),
                   "within_10pct": sum(f >= 1 / 1.1 for f in fr) / max(1, len(fr)),
                   "median_fraction": sorted(fr)[len(fr) // 2] if fr else None,
                   "default_fraction": default[n],
                   "ref_config_fraction": matrix[names[0]][n]}
    return {"scenarios": names, "tuned": tuned, "optimum_us": optimum, "matrix": matrix,
            "default": default, "ppm": ppm_rows, "histograms": hist}


def markdown(res) -> str:
    names = res["scenarios"]
    f = lambda x: "-" if x is None else f"{x:.2f}"
    out = ["## Tuned configurations (bayes) and best-known times", "",
           "| scenario | tuned configuration | best-known (us) |", "|---|---|---|"]
    for n in names:
        out.append(f"| {n} | `{res['tuned'][n]}` | {res['optimum_us'][n]:.1f} |")
    out += ["", "## Random-search distributions (fraction of optimum)", "",
            f"| scenario | evaluated | within 10 % | median | default | tuned for {names[0]} | "
            "histogram 0.0-0.1 ... 0.9-1.0 |", "|---|---|---|---|---|---|---|"]
    for n in names:
        h = res["histograms"][n]
        out.append(f"| {n} | {h['ok']} | {100 * h['within_10pct']:.1f} % | {f(h['median_fraction'])} | "
                   f"{f(h['default_fraction'])} | {f(h['ref_config_fraction'])} | "
                   f"{' '.join(str(c) for c in h['bins'])} |")
    out += ["", "## Portability matrix (row: tuned for; column: run on; fraction of best-known)", "",
            "| tuned for \\ run on | " + " | ".join(names) + " |",
            "|---|" + "---|" * len(names)]
    for n in names:
        out.append(f"| {n} | " + " | ".join(f(res["matrix"][n][m]) for m in names) + " |")
    out.append("| (default) | " + " | ".join(f(res["default"][m]) for m in names) + " |")
    for k, rows in res["ppm"].items():
        out += ["", f"## PPM, kernel {k}", "", "| configuration | best | worst | PPM |",
                "|---|---|---|---|"]
        for r in rows:
            out.append(f"| {r['config']} | {r['best']:.2f} | {r['worst']:.2f} | {r['ppm']:.2f} |")
    return "\n".join(out)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--kernels", default=",".join(KERNELS))
    ap.add_argument("--grids", default=",".join(GRIDS))
    ap.add_argument("--precisions", default=",".join(PRECISIONS))
    ap.add_argument("--random-evals", type=int, default=200)
    ap.add_argument("--bayes-evals", type=int, default=120)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--out", default=None)
    args = ap.parse_args(argv)
    scs = scenarios(args.kernels.split(","), args.grids.split(","), args.precisions.split(","))
    work = tempfile.mkdtemp()
    logs, tuned = {}, {}
    for s in scs:
        logs[label(s)] = tune_pass(s, args.seed, work, args.random_evals, args.bayes_evals)
        ok = [(t, c) for c, t in logs[label(s)]["random"] + logs[label(s)]["bayes"] if t]
        tuned[label(s)] = min(ok)[1]
        print(f"{label(s)}: tuned {tuned[label(s)]} ({min(ok)[0]:.1f} us)", flush=True)
    configs = ["default"] + sorted(set(tuned.values()))
    cross = {label(s): cross_pass(s, args.seed, configs) for s in scs}
    res = analyse(scs, tuned, logs, cross)
    res["cross"] = cross
    res["logs"] = logs
    print(markdown(res))
    if args.out:
        with open(args.out, "w") as fh:
            json.dump(res, fh)


if __name__ == "__main__":
    main()
