"""A user-defined tunable kernel end to end (Sec. 4.1-4.5 for any kernel):
define a vector add with three tunable parameters and a restriction, capture
one launch, tune it, and launch it again through run-time selection of the
wisdom record; report default and tuned times against the HBM roofline.

    python -m paper_2303_12374_gb300.def_example --n 134217728 --peak-gbs 6786

The kernel moves 12 bytes per element (two f32 reads, one f32 write), so the
algorithmic bandwidth of a launch is 12 n / t.
"""

from __future__ import annotations

import argparse
import json
import os
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

SOURCE = r"""
extern "C" __global__ void vadd(const float *a, const float *b, float *c, long n)
{
    // ELEMS chunks of BLOCK consecutive elements per block, VEC floats per access
    long base = ((long)blockIdx.x * BLOCK * ELEMS + threadIdx.x) * VEC;
#pragma unroll
    for (int e = 0; e < ELEMS; ++e) {
        long i = base + (long)e * BLOCK * VEC;
        if (VEC == 4 && i + 3 < n) {
            float4 x = *(const float4 *)(a + i), y = *(const float4 *)(b + i);
            *(float4 *)(c + i) = make_float4(x.x + y.x, x.y + y.y, x.z + y.z, x.w + y.w);
        } else {
            for (int v = 0; v < VEC; ++v)
                if (i + v < n) c[i + v] = a[i + v] + b[i + v];
        }
    }
}
"""


def definition():
    from paper_2303_12374_gb300 import kl
    d = kl.KernelDef("vadd_example", SOURCE, "vadd")
    d.param("BLOCK", [64, 128, 256, 512, 1024], 256)
    d.param("ELEMS", [1, 2, 4, 8], 1)
    d.param("VEC", [1, 4], 1)
    d.restrict("BLOCK * ELEMS * VEC <= 16384")
    d.geometry(block=("BLOCK",), grid=("div_ceil(problem_x, BLOCK * ELEMS * VEC)",))
    return d


def time_launch(fn, reps=20):
    import torch
    for _ in range(3):
        fn()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(reps)]
    for a, b in ev:
        a.record()
        fn()
        b.record()
    torch.cuda.synchronize()
    ms = sorted(a.elapsed_time(b) for a, b in ev)
    return 1e3 * ms[len(ms) // 2]


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--n", type=int, default=1 << 27)
    ap.add_argument("--strategy", default="exhaustive")
    ap.add_argument("--peak-gbs", type=float, default=None, help="HBM copy bandwidth for the fraction")
    args = ap.parse_args(argv)
    import torch
    from paper_2303_12374_gb300 import kl
    n = args.n
    g = torch.Generator(device="cuda").manual_seed(0)
    a = torch.randn(n, generator=g, device="cuda")
    b = torch.randn(n, generator=g, device="cuda")
    c = torch.empty(n, device="cuda")
    argl = [("in", a), ("in", b), ("out", c), ("i64", n)]
    d = definition()
    work = tempfile.mkdtemp()
    ctx = kl.kl_create(0, work)
    try:
        cap = os.path.join(work, "vadd.klcap")
        d.capture(ctx, (n,), argl, cap)
        log = os.path.join(work, "tune.jsonl")
        d.tune(ctx, cap, f"strategy={args.strategy} max_evals=200 log={log}",
               os.path.join(work, "vadd_example.wisdom"))
        os.remove(cap)
        evals = [json.loads(l) for l in open(log)]
        rec = [l for l in open(os.path.join(work, "vadd_example.wisdom")) if not l.startswith("#")][-1]
        t_def = time_launch(lambda: d.launch_config(ctx, "default", (n,), argl))
        t_sel = time_launch(lambda: d.launch(ctx, (n,), argl))
        torch.cuda.synchronize()
        assert torch.equal(c, a + b)
        cfg, rule = d.selected()
        out = {"n": n, "evals": len(evals), "ok": sum(e["ok"] for e in evals),
               "default_us": t_def, "selected_us": t_sel, "selected": cfg, "rule": rule,
               "default_gbs": 12 * n / t_def / 1e3, "selected_gbs": 12 * n / t_sel / 1e3,
               "tune_s": float(rec.split("tune_s=")[1].split()[0])}
        if args.peak_gbs:
            out["default_frac"] = out["default_gbs"] / args.peak_gbs
            out["selected_frac"] = out["selected_gbs"] / args.peak_gbs
        print(json.dumps(out))
    finally:
        kl.kl_destroy(ctx)


if __name__ == "__main__":
    main()
