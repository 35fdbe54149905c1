"""Throughput of the stencil tendency path on GB300.

One step = ghost fill + fused u, v, w tendency (kl_step = kl_fill_ghosts_op
followed by kl_launch; timed as those two calls so the kernel has its own events)
over one grid: 256^3 interior, 3 ghost cells, periodic x and y, free-slip
walls in z, 5th-order upwind-biased flux-form advection + constant-nu
diffusion (nu = 1e-3), f32 storage and arithmetic, seeded synthetic Fourier +
noise fields.  The configuration comes from the committed wisdom files
(tuned); the untuned default of Table 2 and the f64 build are timed beside it.

Prints ONE JSON line.  Under torchrun (N > 1) every rank runs its own
replica of the grid (weak scaling, no collective on the data path); the time
is the maximum over ranks.

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (the reference arm: there is no reference implementation to run).
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gpts/s & HBM GB/s vs ~8 TB/s: tuned vs default, FP64/FP32/16-bit-store"
WORKLOAD = "walls256_adv5_diff"
NX = NY = NZ = 256
G = 3
NU = 1e-3


def kernel_source_hash() -> str:
    import hashlib
    src = os.path.join(ROOT, "paper_2303_12374_gb300", "csrc", "kl_stencil.cuh")
    return hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="kl", choices=["kl", "reference"])
    ap.add_argument("--dtype", default="f32", choices=["f32", "f64", "bf16", "f16"])
    ap.add_argument("--no-extras", action="store_true", help="skip default/f64 side timings")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    return ap.parse_args()


def dist_init(n):
    import torch
    import torch.distributed as dist
    if n > 1 or "RANK" in os.environ:
        rank = int(os.environ.get("RANK", 0))
        local = int(os.environ.get("LOCAL_RANK", 0))
        world = int(os.environ.get("WORLD_SIZE", 1))
        if world > 1:
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        return rank, local, world
    return 0, 0, 1


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.rows = []
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        for line in out.splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def summary(self):
        rows = getattr(self, "rows", [])
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[3:]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def setup(dtype_name, device):
    import torch
    from paper_2303_12374_gb300 import kl, synth
    from paper_2303_12374_gb300.problem import Problem
    spec = synth.WORKLOADS[WORKLOAD]
    f = synth.velocity_fields(NX, NY, NZ, seed=synth.seed_of(spec["index"]), walls=True)
    p = Problem(NX, NY, NZ, g=G, dtype=dtype_name, walls=True, dz=1.0 / NZ, nu=NU,
                device=device)
    ins = [p.upload(f[k]) for k in ("u", "v", "w")]
    outs = [p.empty() for _ in range(3)]
    torch.cuda.synchronize()
    return p, f, ins, outs


def time_steps(ctx, p, ins, outs, op, config, steps, warmup, stream, per_kernel=True):
    """Run warmup + steps; returns (total_ms, mean tendency-kernel ms)."""
    import torch
    from paper_2303_12374_gb300 import kl
    fl = kl.Fields(*[t.data_ptr() for t in ins], None, *[t.data_ptr() for t in outs])
    sp = stream.cuda_stream
    ptrs = [t.data_ptr() for t in ins]

    def step(ev=None):
        if config is None:      # the fill the selected configuration reads
            kl.kl_fill_ghosts_op(ctx, op, p.grid, fl, sp)
        else:
            kl.kl_fill_ghosts(ctx, p.dtype, p.grid, ptrs[0], ptrs[1], ptrs[2], None, sp)
        if ev is not None:
            ev[0].record(stream)
        if config is None:
            kl.kl_launch(ctx, op, p.grid, fl, sp)
        else:
            kl.kl_launch_with_config(ctx, op, config, p.grid, fl, sp)
        if ev is not None:
            ev[1].record(stream)

    with torch.cuda.stream(stream):
        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)] if per_kernel else None
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for s in range(steps):
            step(evs[s] if per_kernel else None)
        t1.record(stream)
        torch.cuda.synchronize()
    total = t0.elapsed_time(t1)
    kern = statistics.fmean(a.elapsed_time(b) for a, b in evs) if per_kernel else None
    return total, kern


def cpu_baseline(seconds_target):
    """The FP64 oracle as it stands on a bounded sample (z levels) of the workload."""
    import oracle
    from paper_2303_12374_gb300 import synth
    oracle.build()
    spec = synth.WORKLOADS[WORKLOAD]
    f = synth.velocity_fields(NX, NY, NZ, seed=synth.seed_of(spec["index"]), walls=True)
    # probe with 2 levels, then size the sample to about seconds_target
    t = time.perf_counter()
    oracle.tendencies(f["u"], f["v"], f["w"], adv=5, diff=1, g=G, walls=True, dx=1 / NX,
                      dy=1 / NY, zh=f["zh"], nu=NU, levels=(0, 2))
    probe = time.perf_counter() - t
    levels = max(2, min(NZ, int(seconds_target / max(probe / 2, 1e-6))))
    t = time.perf_counter()
    oracle.tendencies(f["u"], f["v"], f["w"], adv=5, diff=1, g=G, walls=True, dx=1 / NX,
                      dy=1 / NY, zh=f["zh"], nu=NU, levels=(0, levels))
    dt = time.perf_counter() - t
    pts = NX * NY * levels
    return {"value": pts / dt / 1e9, "unit": "Gpts/s", "cores": 1, "kind": "oracle",
            "sample": f"levels 0..{levels - 1} of the 256^3 grid ({pts} points, FP64, "
                      f"single thread, {dt:.1f} s incl. ghost padding)"}, dt


def precision_sweep(ctx, f, device, stream, reps):
    """Tuned and default kernel time per storage type on the same 256^3 fields."""
    import torch
    from paper_2303_12374_gb300 import kl
    from paper_2303_12374_gb300.problem import Problem
    out = {}
    for name in ("f64", "f32", "bf16", "f16"):
        p = Problem(NX, NY, NZ, g=G, dtype=name, walls=True, dz=1.0 / NZ, nu=NU, device=device)
        ins = [p.upload(f[k]) for k in ("u", "v", "w")]
        outs = [p.empty() for _ in range(3)]
        op = kl.Op(5, 1, p.dtype, 0)
        es = {0: 8, 1: 4, 2: 2, 3: 2}[p.dtype]
        row = {"bytes_per_point": 6 * es}
        n = reps if name != "f64" else max(3, reps // 20)
        for label, cfg in (("tuned", None), ("default", "default")):
            _, k_ms = time_steps(ctx, p, ins, outs, op, cfg, n, 2, stream)
            row[label] = {"kernel_us": k_ms * 1e3, "gpts": NX * NY * NZ / (k_ms * 1e-3) / 1e9,
                          "hbm_gbs": 6 * es * NX * NY * NZ / (k_ms * 1e-3) / 1e9}
            if cfg is None:
                row[label]["config"] = json.loads(kl.kl_stats(ctx))["last_config"]
        row["speedup"] = row["default"]["kernel_us"] / row["tuned"]["kernel_us"]
        out[name] = row
        del ins, outs
        torch.cuda.empty_cache()
    return out


def batched_run(ctx, device, stream, reps=20):
    """64 uneven grids: one batched call (tuned size classes) vs 64 default launches."""
    import torch
    from paper_2303_12374_gb300 import kl, synth
    from paper_2303_12374_gb300.problem import Problem
    spec = synth.WORKLOADS["batch64_uneven"]
    sizes = synth.batch_sizes(synth.seed_of(spec["index"]), spec["count"])
    probs = []
    for q, (nx, ny, nz) in enumerate(sizes):
        f = synth.velocity_fields(nx, ny, nz, seed=synth.seed_of(spec["index"]) * 1000 + q,
                                  walls=True)
        p = Problem(nx, ny, nz, g=G, dtype="f32", walls=True, dz=1.0 / nz, nu=NU, device=device)
        bufs = [p.upload(f[k]) for k in ("u", "v", "w")]
        outs = [p.empty() for _ in range(3)]
        fl = kl.Fields(*[b.data_ptr() for b in bufs], None, *[o.data_ptr() for o in outs])
        probs.append((p, bufs, outs, fl))
    pts = sum(nx * ny * nz for nx, ny, nz in sizes)
    op = kl.Op(5, 1, 1, 0)
    grids = [pr[0].grid for pr in probs]
    fields = [pr[3] for pr in probs]
    sp = stream.cuda_stream
    with torch.cuda.stream(stream):
        for p, bufs, outs, fl in probs:
            kl.kl_fill_ghosts(ctx, p.dtype, p.grid, *[b.data_ptr() for b in bufs], None, sp)

        def batched():
            kl.kl_launch_batched(ctx, op, grids, fields, sp)

        def separate():
            for p, bufs, outs, fl in probs:
                kl.kl_launch_with_config(ctx, op, "default", p.grid, fl, sp)

        res = {}
        for label, fn in (("batched_tuned", batched), ("separate_default", separate)):
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                fn()
            b.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b) / reps
            res[label] = {"ms": ms, "gpts": pts / (ms * 1e-3) / 1e9,
                          "hbm_gbs": 24 * pts / (ms * 1e-3) / 1e9}
    res["grids"] = len(sizes)
    res["points"] = pts
    res["speedup"] = res["separate_default"]["ms"] / res["batched_tuned"]["ms"]
    return res


def launch_overhead(local, wisdom, device, calls=1000):
    """Sec. 5.6: the four stages of a first launch and the cost of a cached launch."""
    import torch
    from paper_2303_12374_gb300 import kl
    from paper_2303_12374_gb300.problem import Problem
    ctx = kl.kl_create(local, wisdom)
    try:
        n = 32
        p = Problem(n, n, n, g=G, dtype="f32", walls=True, dz=1.0 / n, nu=NU, device=device)
        bufs = [p.empty() for _ in range(3)]
        outs = [p.empty() for _ in range(3)]
        fl = kl.Fields(*[b.data_ptr() for b in bufs], None, *[o.data_ptr() for o in outs])
        op = kl.Op(5, 1, p.dtype, 0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        kl.kl_launch(ctx, op, p.grid, fl)
        first_ms = (time.perf_counter() - t0) * 1e3
        stages = json.loads(kl.kl_stats(ctx))["stage_ms"]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(calls):
            kl.kl_launch(ctx, op, p.grid, fl)
        host_us = (time.perf_counter() - t0) / calls * 1e6
        torch.cuda.synchronize()
        return {"first_launch_ms": first_ms, "stage_ms": stages,
                "cached_launch_host_us": host_us,
                "note": "host time per kl_launch call through the ctypes binding, 32^3 grid"}
    finally:
        kl.kl_destroy(ctx)


def run_reference(args):
    rank = int(os.environ.get("RANK", 0))
    if rank != 0:
        return
    per_step = max(1.0, args.cpu_seconds / max(1, args.steps))
    vals = []
    cb = None
    for _ in range(args.warmup if args.warmup < 1 else 1):
        pass
    for s in range(args.steps):
        cb, dt = cpu_baseline(per_step)
        vals.append(cb["value"])
    value = statistics.fmean(vals)
    cb["value"] = value
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Gpts/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": NX * NY * NZ / (value * 1e9) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": "256x256x256", "ghosts": G,
                       "bc": "periodic x,y; walls z", "op": "adv5 + const-nu diffusion"},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "Gpts/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import torch.distributed as dist
    from paper_2303_12374_gb300 import kl

    rank, local, world = dist_init(args.gpus)
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    wisdom = os.path.join(ROOT, "paper_2303_12374_gb300", "wisdom")
    ctx = kl.kl_create(local, wisdom)
    stream = torch.cuda.Stream(device)
    p, f, ins, outs = setup(args.dtype, device)
    op = kl.Op(5, 1, p.dtype, 0)
    pts = NX * NY * NZ
    es = {0: 8, 1: 4, 2: 2, 3: 2}[p.dtype]

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # --- tuned (wisdom-selected) configuration: the headline
    barrier()
    with Clocks(local) as clk:
        total_ms, kern_ms = time_steps(ctx, p, ins, outs, op, None, args.steps, args.warmup,
                                       stream)
    barrier()
    if world > 1:
        t = torch.tensor([total_ms], device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    stats = json.loads(kl.kl_stats(ctx))
    tuned_cfg = stats["last_config"]
    ms_step = total_ms / args.steps
    value = world * pts * args.steps / (total_ms * 1e-3) / 1e9

    peaks = measured_peaks()
    peak_gbs = peaks.get("hbm_gbs") or 6800.0
    alg_bytes = 6 * es * pts
    achieved = alg_bytes / (kern_ms * 1e-3) / 1e9
    traffic = None
    tp = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tp):
        # DRAM bytes per launch from an ncu capture, valid only for the kernel
        # source it was taken with
        tr = json.load(open(tp))
        key = f"{WORKLOAD}:{args.dtype}:{tuned_cfg}:{kernel_source_hash()}"
        traffic = tr.get(key)

    extras = {}
    if not args.no_extras and rank == 0:
        k2 = max(50, args.steps // 10)
        d_total, d_kern = time_steps(ctx, p, ins, outs, op, "default", k2, 5, stream)
        extras["default_config"] = {
            "config": "default (Table 2)", "value": pts * k2 / (d_total * 1e-3) / 1e9,
            "kernel_us": d_kern * 1e3,
            "kernel_hbm_gbs": alg_bytes / (d_kern * 1e-3) / 1e9}
        extras["tuned_config"] = {"config": tuned_cfg, "kernel_us": kern_ms * 1e3,
                                  "speedup_vs_default": d_kern / kern_ms}
        extras["precision"] = precision_sweep(ctx, f, device, stream, max(20, args.steps // 20))
        extras["batched"] = batched_run(ctx, device, stream)
        extras["launch_overhead"] = launch_overhead(local, wisdom, device)

    # --- end to end through the public API with pinned host buffers
    e2e = None
    if rank == 0:
        host_in = [torch.empty(p.extent, dtype=p.tdtype, pin_memory=True) for _ in range(3)]
        host_out = [torch.empty(p.extent, dtype=p.tdtype, pin_memory=True) for _ in range(3)]
        for h, d in zip(host_in, ins):
            h.copy_(d)
        fl = kl.Fields(*[t.data_ptr() for t in ins], None, *[t.data_ptr() for t in outs])
        ke = max(5, args.steps // 100)
        with torch.cuda.stream(stream):
            def e2e_step():
                for h, d in zip(host_in, ins):
                    d.copy_(h, non_blocking=True)
                kl.kl_step(ctx, op, p.grid, fl, stream.cuda_stream)
                for h, d in zip(host_out, outs):
                    h.copy_(d, non_blocking=True)
            for _ in range(2):
                e2e_step()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(ke):
                e2e_step()
            b.record(stream)
            torch.cuda.synchronize()
        e_ms = a.elapsed_time(b) / ke
        nbytes = 3 * p.extent * es
        e2e = {"value": pts / (e_ms * 1e-3) / 1e9, "unit": "Gpts/s",
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
               "ms_per_step": e_ms}

    cb = None
    if rank == 0 and world == 1:
        cb, _ = cpu_baseline(args.cpu_seconds)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "Gpts/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": args.dtype, "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": "256x256x256", "ghosts": G,
                       "bc": "periodic x,y; free-slip walls z",
                       "op": "adv5 + const-nu diffusion, u,v,w fused",
                       "step": "kl_fill_ghosts_op + kl_launch (= kl_step)",
                       "selected_config": tuned_cfg,
                       "l2": "inputs larger than L2 (3 x %.0f MB read, 3 x %.0f MB written)"
                             % (p.extent * es / 1e6, p.extent * es / 1e6),
                       "parallelism": f"replicas x{world}"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak_gbs,
                         "unit": "GB/s", "frac": achieved / peak_gbs, "traffic": traffic,
                         "kernel": "kl_tendency", "kernel_us": kern_ms * 1e3,
                         "alg_bytes_per_launch": alg_bytes,
                         "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)"
                                        if peaks.get("hbm_gbs") else "fallback"},
            "clocks": clk.summary(),
            "gpu_launches": 2 * args.steps,
            "e2e": e2e,
            "cpu_baseline": cb,
            "extras": extras,
        }
        print(json.dumps(line))
    kl.kl_destroy(ctx)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
