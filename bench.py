"""Throughput of the stencil tendency path on GB300.

One step = kl_step (the ghost fill the selected configuration reads, then the
fused u, v, w tendency kernel; timed as kl_fill_ghosts_op + kl_launch so that
the kernel has its own events) over one grid: 512 x 512 x 256 interior points
(67.1 M), 3 ghost cells, periodic x and y, free-slip walls in z, 5th-order
upwind-biased flux-form advection + constant-nu diffusion (nu = 1e-3), f32
storage and arithmetic, seeded synthetic Fourier + noise fields.  It is the
largest single grid of the workloads (the 1024 x 1024 x 64 LES grid has the
same point count; it is reported in the extras).  The configuration comes from
the committed wisdom files (tuned); the untuned default of Table 2, the other
storage types, the other workloads and the batch are timed beside it.

Prints ONE JSON line.  Under torchrun (N > 1) every rank runs its own
replica of the grid (weak scaling, no collective on the data path); the time
is the maximum over ranks.

--impl reference times the FP64 CPU oracle on the host cores, on bounded
samples of z levels of the same workload (the reference arm: there is no
reference implementation to run).
"""

from __future__ import annotations

import argparse
import json
import math
import os
import shutil
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gpts/s & HBM GB/s vs ~8 TB/s: tuned vs default, FP64/FP32/16-bit-store"
WORKLOAD = "walls512x512x256_precision"
G = 3
NU = 1e-3
REF_SECONDS = 120.0      # reference arm: CPU time of warm-up + timed samples
# FP32 (or FP64) operations per interior point of the fused tendency with each
# face flux formed once, an FMA counted as one: 9 faces x 14 (advecting
# velocity 1, the upwind differences and sums 5, I6 3, D6 2, U*I6 + |U|*D6 2,
# folded diffusion 1) + 3 tendencies x 6 (3 differences, 1 product, 2 FMAs)
OPS_PER_POINT = 144


def extents(workload=None):
    from paper_2303_12374_gb300 import synth
    spec = synth.WORKLOADS[workload or WORKLOAD]
    return spec["nx"], spec["ny"], spec["nz"]


def kernel_source_hash() -> str:
    import hashlib
    src = os.path.join(ROOT, "paper_2303_12374_gb300", "csrc", "kl_stencil.cuh")
    return hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=600)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="kl", choices=["kl", "reference"])
    ap.add_argument("--dtype", default="f32", choices=["f32", "f64", "bf16", "f16"])
    ap.add_argument("--no-extras", action="store_true", help="skip default/f64 side timings")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    return ap.parse_args()


def dist_init(n, backend=None):
    """(rank, local rank, world) from the torchrun environment; joins the
    process group when world > 1 (NCCL on the GPUs; `backend` overrides, e.g.
    gloo for the CPU tests of this path)."""
    import torch
    import torch.distributed as dist
    if n > 1 or "RANK" in os.environ:
        rank = int(os.environ.get("RANK", 0))
        local = int(os.environ.get("LOCAL_RANK", 0))
        world = int(os.environ.get("WORLD_SIZE", 1))
        if world > 1:
            if backend is None:
                torch.cuda.set_device(local)
                dist.init_process_group("nccl", device_id=torch.device("cuda", local))
            else:
                dist.init_process_group(backend)
        return rank, local, world
    return 0, 0, 1


def max_over_ranks(x, world, device):
    """The maximum of a per-rank scalar over all ranks (the job's time)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, pts, steps, total_ms):
    """Whole-job throughput in Gpts/s: every rank steps its own replica of the
    grid (weak scaling), the job takes the slowest rank's time."""
    return world * pts * steps / (total_ms * 1e-3) / 1e9


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


def workload_fields(workload=None):
    from paper_2303_12374_gb300 import synth
    spec = synth.WORKLOADS[workload or WORKLOAD]
    nx, ny, nz = extents(workload)
    return synth.velocity_fields(nx, ny, nz, seed=synth.seed_of(spec["index"]), walls=True)


def setup(dtype_name, device, f=None):
    import torch
    from paper_2303_12374_gb300.problem import Problem
    nx, ny, nz = extents()
    f = f if f is not None else workload_fields()
    p = Problem(nx, ny, nz, g=G, dtype=dtype_name, walls=True, dz=1.0 / nz, nu=NU,
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


class OracleSample:
    """The FP64 oracle as it stands, timed on z levels of the bench workload.

    Levels [k0, k0 + L) with 3 <= k0 and k0 + L <= nz - 3 are computed from a
    slab of the fields with the stencil's 3-level reach on each side, so only
    the slab is padded; the result is the full grid's on those levels.
    threads > 1 runs the oracle's OpenMP timing build (same results)."""

    def __init__(self, f=None):
        import oracle
        from paper_2303_12374_gb300 import synth
        oracle.build()
        self.oracle, self.synth = oracle, synth
        self.nx, self.ny, self.nz = extents()
        self.f = f if f is not None else workload_fields()

    def run(self, k0, nlev, threads=1):
        """Seconds the oracle takes for interior levels [k0, k0 + nlev)."""
        assert G <= k0 and k0 + nlev <= self.nz - G
        lo, hi = k0 - G, k0 + nlev + G
        sl = {k: np.ascontiguousarray(self.f[k][lo:hi]) for k in ("u", "v", "w")}
        zh = self.synth.zfaces(hi - lo, (hi - lo) / self.nz)
        t = time.perf_counter()
        self.oracle.tendencies(sl["u"], sl["v"], sl["w"], adv=5, diff=1, g=G, walls=False,
                               dx=1 / self.nx, dy=1 / self.ny, zh=zh, nu=NU,
                               levels=(G, G + nlev), threads=threads)
        return time.perf_counter() - t


def host_threads() -> int:
    """Host cores the oracle's OpenMP build runs on (1 without that build)."""
    import oracle
    return (os.cpu_count() or 1) if oracle.omp_available() else 1


def cpu_baseline(seconds_target, sampler=None):
    """The oracle on bounded samples (about seconds_target each) of the
    workload: single-threaded, and on every host core (OpenMP build)."""
    sampler = sampler or OracleSample()
    nx, ny, nz = sampler.nx, sampler.ny, sampler.nz
    out = {}
    for label, threads in (("single_thread", 1), ("all_cores", host_threads())):
        per_level = sampler.run(G, 2, threads) / 2
        levels = max(2, min(nz - 2 * G, int(seconds_target / max(per_level, 1e-6))))
        dt = sampler.run(G, levels, threads)
        pts = nx * ny * levels
        out[label] = {"value": pts / dt / 1e9, "unit": "Gpts/s", "cores": threads,
                      "sample": f"levels {G}..{G + levels - 1} of the {nx}x{ny}x{nz} grid "
                                f"({pts} points, FP64, {threads} thread(s), {dt:.1f} s incl. "
                                f"padding of the slab)"}
    best = out["all_cores"]
    return {"value": best["value"], "unit": "Gpts/s", "cores": best["cores"], "kind": "oracle",
            "sample": best["sample"], "single_thread": out["single_thread"],
            "host_cpus": os.cpu_count()}, None


def e2e_run(ctx, p, f, op, device, steps, overlap=True):
    """Steps from host data to host results through the public API.

    Every step copies the interior of u, v, w from pinned host memory into the
    padded device buffers (kl_copy_in: one strided DMA copy per field), runs
    kl_step (ghost fill + tendencies) and copies the interior of ut, vt, wt
    back to pinned host memory (kl_copy_out).  overlap=True runs
    the three stages of consecutive steps on three streams with two device
    buffer sets (step i's copy-in overlaps step i-1's kernels and step i-2's
    copy-out); overlap=False runs them one after the other on one stream.
    Returns (ms per step, bytes copied per direction per step)."""
    import torch
    from paper_2303_12374_gb300 import kl
    host_in = [torch.from_numpy(np.ascontiguousarray(f[k])).to(p.tdtype).pin_memory()
               for k in ("u", "v", "w")]
    host_out = [torch.empty((p.nz, p.ny, p.nx), dtype=p.tdtype).pin_memory() for _ in range(3)]
    nbuf = 2 if overlap else 1
    dev_in = [[p.empty() for _ in range(3)] for _ in range(nbuf)]
    dev_out = [[p.empty() for _ in range(3)] for _ in range(nbuf)]
    fields = [kl.Fields(*[t.data_ptr() for t in dev_in[b]], None,
                        *[t.data_ptr() for t in dev_out[b]]) for b in range(nbuf)]
    if overlap:
        s_in, s_c, s_out = (torch.cuda.Stream(device) for _ in range(3))
    else:
        s_in = s_c = s_out = torch.cuda.Stream(device)
    ev_in = [torch.cuda.Event() for _ in range(nbuf)]
    ev_c = [torch.cuda.Event() for _ in range(nbuf)]
    ev_out = [torch.cuda.Event() for _ in range(nbuf)]

    def issue(i):
        b = i % nbuf
        with torch.cuda.stream(s_in):
            if i >= nbuf:
                s_in.wait_event(ev_c[b])        # step i - nbuf's kernels read dev_in[b]
            for h, d in zip(host_in, dev_in[b]):
                kl.kl_copy_in(p.dtype, p.grid, h.data_ptr(), d.data_ptr(), s_in.cuda_stream)
            ev_in[b].record(s_in)
        with torch.cuda.stream(s_c):
            s_c.wait_event(ev_in[b])
            if i >= nbuf:
                s_c.wait_event(ev_out[b])       # step i - nbuf's results left dev_out[b]
            kl.kl_step(ctx, op, p.grid, fields[b], s_c.cuda_stream)
            ev_c[b].record(s_c)
        with torch.cuda.stream(s_out):
            s_out.wait_event(ev_c[b])
            for h, d in zip(host_out, dev_out[b]):
                kl.kl_copy_out(p.dtype, p.grid, d.data_ptr(), h.data_ptr(), s_out.cuda_stream)
            ev_out[b].record(s_out)

    for i in range(2 * nbuf):                   # warm-up (allocator, module, pinned paths)
        issue(i)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(s_in)
    for i in range(steps):
        issue(i)
    b.record(s_out)
    torch.cuda.synchronize()
    es = host_in[0].element_size()
    return a.elapsed_time(b) / steps, 3 * p.nx * p.ny * p.nz * es


def link_bound_ms(p, device, reps=5):
    """The host link's own time for one e2e step's traffic: three interior
    fields host -> device and three device -> host as plain contiguous copies
    from and to pinned memory, the two directions at once on two streams."""
    import torch
    shape = (p.nz, p.ny, p.nx)
    h_in = [torch.empty(shape, dtype=p.tdtype).pin_memory() for _ in range(3)]
    h_out = [torch.empty(shape, dtype=p.tdtype).pin_memory() for _ in range(3)]
    d_in = [torch.empty(shape, dtype=p.tdtype, device=device) for _ in range(3)]
    d_out = [torch.empty(shape, dtype=p.tdtype, device=device) for _ in range(3)]
    s1, s2 = torch.cuda.Stream(device), torch.cuda.Stream(device)

    def once():
        with torch.cuda.stream(s1):
            for h, d in zip(h_in, d_in):
                d.copy_(h, non_blocking=True)
        with torch.cuda.stream(s2):
            for h, d in zip(h_out, d_out):
                h.copy_(d, non_blocking=True)

    once()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        once()
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) / reps * 1e3
    del h_in, h_out, d_in, d_out
    return ms


def alu_peaks_live():
    """FP32 (packed and scalar) and FP64 FMA rates measured now (alu_peaks)."""
    from paper_2303_12374_gb300 import alu_peaks
    out = {}
    for kind in ("f32x2", "f64"):
        r = alu_peaks.measure(kind, target_ms=20.0, reps=5)
        out[kind] = {"tflops": r["tflops"], "fma_per_sm_per_clk": r.get("fma_per_sm_per_clk"),
                     "sm_mhz": r["clocks"]["sm_mhz"]}
    return out


def roof(us, pts, nbytes, peak_gbs, op_peak):
    """HBM and ALU roofline fractions of one kernel time.  op_peak: the FMA
    pipe's measured rate in operations per second (an FMA is one operation)."""
    gbs = nbytes / us / 1e3
    ops = OPS_PER_POINT * pts / (us * 1e-6)
    return {"hbm_gbs": gbs, "hbm_frac": gbs / peak_gbs,
            "alu_tops": ops / 1e12, "alu_frac": ops / op_peak if op_peak else None}


def precision_sweep(ctx, f, device, stream, reps, peak_gbs, op_peaks):
    """Tuned and default kernel time per storage type on the bench grid, each
    against both roofs: HBM at its bytes per point, and the FMA pipe of its
    arithmetic (FP64 for f64 storage, FP32 otherwise)."""
    import torch
    from paper_2303_12374_gb300 import kl
    from paper_2303_12374_gb300.problem import Problem
    nx, ny, nz = extents()
    pts = nx * ny * nz
    out = {}
    for name in ("f64", "f32", "bf16", "f16"):
        p = Problem(nx, ny, nz, g=G, dtype=name, walls=True, dz=1.0 / nz, nu=NU, device=device)
        ins = [p.upload(f[k]) for k in ("u", "v", "w")]
        outs = [p.empty() for _ in range(3)]
        op = kl.Op(5, 1, p.dtype, 0)
        es = {0: 8, 1: 4, 2: 2, 3: 2}[p.dtype]
        row = {"bytes_per_point": 6 * es}
        n = reps if name != "f64" else 3
        op_peak = op_peaks.get("f64" if name == "f64" else "f32")
        for label, cfg in (("tuned", None), ("default", "default")):
            _, k_ms = time_steps(ctx, p, ins, outs, op, cfg, n, 2, stream)
            us = k_ms * 1e3
            row[label] = {"kernel_us": us, "gpts": pts / us / 1e3}
            row[label].update(roof(us, pts, 6 * es * pts, peak_gbs, op_peak))
            if cfg is None:
                row[label]["config"] = json.loads(kl.kl_stats(ctx))["last_config"]
        row["speedup"] = row["default"]["kernel_us"] / row["tuned"]["kernel_us"]
        row["bound"] = ("alu" if row["tuned"]["alu_frac"] and
                        row["tuned"]["alu_frac"] > row["tuned"]["hbm_frac"] else "hbm")
        out[name] = row
        del ins, outs
        torch.cuda.empty_cache()
    return out


def workload_sweep(ctx, device, stream, reps, peak_gbs, op_peaks):
    """Kernel time, tuned (wisdom) vs default, on the other seeded workloads:
    256^3 walls f32 (the grid of the paper's 256^3 tuning), 64^3 periodic 2nd
    order f64, 1024x1024x64 stretched with variable nu f32 (ghosts filled
    once, then kernel launches only)."""
    import torch
    from paper_2303_12374_gb300 import kl, synth
    from paper_2303_12374_gb300.tune_cli import build_problem
    out = {}
    for wl, dt in (("walls256_adv5_diff", "f32"), ("periodic64_adv2_f64", "f64"),
                   ("les1024x1024x64_stretched_varnu", "f32")):
        p, op, bufs, outs, fl = build_problem(wl, dt)
        spec = synth.WORKLOADS[wl]
        pts = p.nx * p.ny * p.nz
        es = {0: 8, 1: 4, 2: 2, 3: 2}[p.dtype]
        nbytes = (6 + (1 if spec["diff"] == 2 else 0)) * es * pts
        sp = stream.cuda_stream
        with torch.cuda.stream(stream):
            kl.kl_fill_ghosts(ctx, p.dtype, p.grid, bufs["u"].data_ptr(), bufs["v"].data_ptr(),
                              bufs["w"].data_ptr(), bufs["nu"].data_ptr() if "nu" in bufs else None,
                              sp)
            row = {"grid": f"{p.nx}x{p.ny}x{p.nz}", "dtype": dt, "points": pts,
                   "alg_bytes": nbytes}
            for label, cfg in (("tuned", None), ("default", "default")):
                def launch():
                    if cfg is None:
                        kl.kl_launch(ctx, op, p.grid, fl, sp)
                    else:
                        kl.kl_launch_with_config(ctx, op, cfg, p.grid, fl, sp)
                for _ in range(3):
                    launch()
                torch.cuda.synchronize()
                n = max(3, reps * 16_777_216 // pts) if dt != "f64" else max(10, reps)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                for _ in range(n):
                    launch()
                b.record(stream)
                torch.cuda.synchronize()
                us = a.elapsed_time(b) / n * 1e3
                row[label] = {"kernel_us": us, "gpts": pts / us / 1e3, "hbm_gbs": nbytes / us / 1e3,
                              "hbm_frac": nbytes / us / 1e3 / peak_gbs}
                if cfg is None:
                    row[label]["config"] = json.loads(kl.kl_stats(ctx))["last_config"]
            row["speedup"] = row["default"]["kernel_us"] / row["tuned"]["kernel_us"]
        out[wl] = row
        del bufs, outs
        torch.cuda.empty_cache()
    return out


def diag_timing(ctx, p, outs, stream, reps=20, ins=None):
    """kl_diag (FP64 max, rms, sums, metric-weighted sum) on one tendency of the
    bench grid, without and with an FP64 reference field.  Per call: `us` the
    wall time including the 48-byte read-back it synchronises on and the host
    round trip; `device_us` the stream time between events recorded around
    each call (the reduction kernels and the read-back only)."""
    import torch
    from paper_2303_12374_gb300 import kl
    ref = torch.zeros(p.extent, dtype=torch.float64, device=outs[0].device)
    p.view(ref).copy_(p.view(outs[0]).to(torch.float64) * (1.0 + 1e-6))
    res = {}
    for label, rp in (("no_reference", None), ("fp64_reference", ref.data_ptr())):
        out = None
        for _ in range(3):
            out = kl.kl_diag(ctx, p.dtype, p.grid, 0, outs[0].data_ptr(), rp, stream.cuda_stream)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(reps)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for a, b in evs:
            a.record(stream)
            kl.kl_diag(ctx, p.dtype, p.grid, 0, outs[0].data_ptr(), rp, stream.cuda_stream)
            b.record(stream)
        wall = (time.perf_counter() - t0) / reps * 1e6
        torch.cuda.synchronize()
        dev = statistics.fmean(a.elapsed_time(b) for a, b in evs) * 1e3
        nbytes = p.nx * p.nz * p.ny * (outs[0].element_size() + (8 if rp else 0))
        res[label] = {"us": wall, "device_us": dev, "read_gbs_device": nbytes / dev / 1e3,
                      "values": list(out)}
    del ref
    if ins is not None:
        # kinetic-energy tendency of the step (three FP64 inner products)
        t0 = time.perf_counter()
        energy = sum(kl.kl_dot(ctx, p.dtype, p.grid, lv, x.data_ptr(), y.data_ptr(), stream.cuda_stream)
                     for lv, x, y in ((0, ins[0], outs[0]), (0, ins[1], outs[1]), (1, ins[2], outs[2])))
        res["energy_tendency"] = energy
        res["energy_host_us"] = (time.perf_counter() - t0) * 1e6
    return res


def les_step(ctx, stream, peak_gbs, reps=20, cs=0.1):
    """The LES step on the 1024x1024x64 stretched workload, f32: ghost fill of
    u, v, w, Smagorinsky nu (with its own ghost fill), then 5th-order advection
    + variable-nu diffusion with that nu.  The nu kernel alone is reported
    against its roofline: 16 B/pt (read u, v, w, write nu)."""
    import torch
    from paper_2303_12374_gb300 import kl
    from paper_2303_12374_gb300.tune_cli import build_problem
    p, op, bufs, outs, fl = build_problem("les1024x1024x64_stretched_varnu", "f32")
    pts = p.nx * p.ny * p.nz
    sp = stream.cuda_stream
    uvw = [bufs[k].data_ptr() for k in ("u", "v", "w")]
    nu = bufs["nu"].data_ptr()
    parts = {
        "smagorinsky": lambda: kl.kl_smagorinsky(ctx, p.dtype, p.grid, cs, *uvw, nu, False, sp),
        "tendency": lambda: kl.kl_launch(ctx, op, p.grid, fl, sp),
        "step": lambda: (kl.kl_fill_ghosts(ctx, p.dtype, p.grid, *uvw, None, sp),
                         kl.kl_smagorinsky(ctx, p.dtype, p.grid, cs, *uvw, nu, True, sp),
                         kl.kl_launch(ctx, op, p.grid, fl, sp)),
    }
    res = {"grid": f"{p.nx}x{p.ny}x{p.nz}", "dtype": "f32", "cs": cs, "points": pts}
    with torch.cuda.stream(stream):
        kl.kl_fill_ghosts(ctx, p.dtype, p.grid, *uvw, None, sp)
        for name, fn in parts.items():
            for _ in range(3):
                fn()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                fn()
            b.record(stream)
            torch.cuda.synchronize()
            res[name + "_us"] = a.elapsed_time(b) / reps * 1e3
    res["smagorinsky_gbs"] = 16 * pts / res["smagorinsky_us"] / 1e3
    res["smagorinsky_frac"] = res["smagorinsky_gbs"] / peak_gbs
    res["step_gpts"] = pts / res["step_us"] / 1e3
    res["tendency_config"] = json.loads(kl.kl_stats(ctx))["last_config"]
    del bufs, outs
    torch.cuda.empty_cache()
    return res


def batched_run(ctx, device, stream, peak_gbs, reps=20):
    """64 uneven grids: one batched call (the batch's wisdom configuration,
    one CUDA graph) vs 64 separate launches, each with its own nearest-size
    record (tuned), and vs 64 separate default launches."""
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

        def separate_tuned():
            for p, bufs, outs, fl in probs:
                kl.kl_launch(ctx, op, p.grid, fl, sp)

        res = {}
        for label, fn in (("batched_tuned", batched), ("separate_tuned", separate_tuned),
                          ("separate_default", separate)):
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
            gbs = 24 * pts / (ms * 1e-3) / 1e9
            res[label] = {"ms": ms, "gpts": pts / (ms * 1e-3) / 1e9, "hbm_gbs": gbs,
                          "hbm_frac": gbs / peak_gbs}
    res["grids"] = len(sizes)
    res["points"] = pts
    res["speedup"] = res["separate_default"]["ms"] / res["batched_tuned"]["ms"]
    res["speedup_vs_separate_tuned"] = res["separate_tuned"]["ms"] / res["batched_tuned"]["ms"]
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
        res = {"first_launch_ms": first_ms, "stage_ms": stages,
               "cached_launch_host_us": host_us,
               "note": "host time per kl_launch call through the ctypes binding, 32^3 grid"}
        # the same first launch with an on-disk cubin cache: an empty directory
        # (NVRTC, then the cubin is written) and a second context that reads it
        d = tempfile.mkdtemp()
        try:
            for which in ("empty", "filled"):
                c2 = kl.kl_create(local, wisdom)
                try:
                    kl.kl_set_cache_dir(c2, d)
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    kl.kl_launch(c2, op, p.grid, fl)
                    res[f"first_launch_ms_disk_cache_{which}"] = (time.perf_counter() - t0) * 1e3
                    st = json.loads(kl.kl_stats(c2))
                    res[f"stage_ms_disk_cache_{which}"] = dict(st["stage_ms"],
                                                               disk_read=st["disk_cache"]["read_ms"])
                finally:
                    kl.kl_destroy(c2)
        finally:
            shutil.rmtree(d, ignore_errors=True)
        return res
    finally:
        kl.kl_destroy(ctx)


def run_reference(args):
    """The reference arm: the oracle on the host cores (its OpenMP timing
    build on every core), each step a sample of z levels of the workload sized
    so that warm-up plus timed steps take about REF_SECONDS (one level at
    least); rank 0 only."""
    rank = int(os.environ.get("RANK", 0))
    if rank != 0:
        return
    sampler = OracleSample()
    nx, ny, nz = sampler.nx, sampler.ny, sampler.nz
    threads = host_threads()
    per_level = sampler.run(G, 2, threads) / 2
    nsamp = max(1, args.steps + args.warmup)
    nlev = max(1, min(nz - 2 * G, int(REF_SECONDS / nsamp / max(per_level, 1e-6))))
    span = nz - 2 * G - nlev + 1
    for s in range(args.warmup):
        sampler.run(G + (s * nlev) % span, nlev, threads)
    total = 0.0
    for s in range(args.steps):
        total += sampler.run(G + (s * nlev) % span, nlev, threads)
    pts = nx * ny * nlev * args.steps
    value = pts / total / 1e9
    cb = {"value": value, "unit": "Gpts/s", "cores": threads, "kind": "oracle",
          "sample": f"{args.steps} steps of {nlev} z level(s) of the {nx}x{ny}x{nz} grid each "
                    f"({pts} points, FP64, {threads} thread(s), {total:.1f} s)"}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Gpts/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": nx * ny * nz / (value * 1e9) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": f"{nx}x{ny}x{nz}", "ghosts": G,
                       "bc": "periodic x,y; walls z", "op": "adv5 + const-nu diffusion"},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "Gpts/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def committed_alu_peaks():
    """The FMA rates of profiles/alu_peaks.json (measured by alu_peaks)."""
    try:
        d = json.load(open(os.path.join(ROOT, "profiles", "alu_peaks.json")))
        return {k: {"tflops": d[k]["tflops"], "fma_per_sm_per_clk": d[k].get("fma_per_sm_per_clk"),
                    "sm_mhz": d[k]["clocks"]["sm_mhz"]} for k in ("f32x2", "f64")}
    except (OSError, KeyError, ValueError):
        return {}


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
    f = workload_fields()
    p, f, ins, outs = setup(args.dtype, device, f)
    op = kl.Op(5, 1, p.dtype, 0)
    nx, ny, nz = extents()
    pts = nx * ny * nz
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
    kl.kl_check(ctx, stream.cuda_stream)       # no device wait gave up while timed
    total_ms = max_over_ranks(total_ms, world, device)
    stats = json.loads(kl.kl_stats(ctx))
    tuned_cfg = stats["last_config"]
    ms_step = total_ms / args.steps
    value = job_value(world, pts, args.steps, total_ms)

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
    alu = committed_alu_peaks()
    alu_source = "profiles/alu_peaks.json (measured)" if alu else None
    if not args.no_extras and rank == 0:
        try:
            alu = alu_peaks_live()
            alu_source = "measured in this run (alu_peaks)"
        except Exception as e:      # keep the committed figures
            extras["alu_peaks_error"] = str(e)
        extras["alu_peaks"] = alu
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    # FMA-pipe operation rates (an FMA is one operation) at the maximum clock
    op_peaks = {}
    if alu:
        op_peaks["f32"] = alu["f32x2"]["tflops"] / 2 * 1e12
        op_peaks["f64"] = alu["f64"]["tflops"] / 2 * 1e12

    if not args.no_extras and rank == 0:
        k2 = max(50, args.steps // 10)
        d_total, d_kern = time_steps(ctx, p, ins, outs, op, "default", k2, 5, stream)
        extras["default_config"] = {
            "config": "default (Table 2)", "value": pts * k2 / (d_total * 1e-3) / 1e9,
            "kernel_us": d_kern * 1e3,
            "kernel_hbm_gbs": alg_bytes / (d_kern * 1e-3) / 1e9,
            "kernel_hbm_frac": alg_bytes / (d_kern * 1e-3) / 1e9 / peak_gbs}
        extras["tuned_config"] = {"config": tuned_cfg, "kernel_us": kern_ms * 1e3,
                                  "speedup_vs_default": d_kern / kern_ms}
        extras["precision"] = precision_sweep(ctx, f, device, stream, max(20, args.steps // 30),
                                              peak_gbs, op_peaks)
        extras["workloads"] = workload_sweep(ctx, device, stream, max(20, args.steps // 30),
                                             peak_gbs, op_peaks)
        extras["batched"] = batched_run(ctx, device, stream, peak_gbs)
        extras["launch_overhead"] = launch_overhead(local, wisdom, device)
        extras["diag"] = diag_timing(ctx, p, outs, stream, ins=ins)
        extras["les_step"] = les_step(ctx, stream, peak_gbs)

    # --- end to end through the public API with pinned host buffers (every rank)
    # three repeats each, the median reported: the host link and host memory
    # are shared with the other GPUs of the machine, so single runs vary
    barrier()
    e_runs = [e2e_run(ctx, p, f, op, device, max(10, args.steps // 60), overlap=True)
              for _ in range(3)]
    s_runs = [e2e_run(ctx, p, f, op, device, max(5, args.steps // 200), overlap=False)
              for _ in range(3)]
    link_ms = link_bound_ms(p, device)
    barrier()
    e_ms, e_bytes = statistics.median(r[0] for r in e_runs), e_runs[0][1]
    s_ms = statistics.median(r[0] for r in s_runs)
    e_ms = max_over_ranks(e_ms, world, device)
    s_ms = max_over_ranks(s_ms, world, device)
    e2e = {"value": job_value(world, pts, 1, e_ms), "unit": "Gpts/s",
           "h2d_bytes_per_step": e_bytes, "d2h_bytes_per_step": e_bytes,
           "ms_per_step": e_ms,
           "api": "kl_copy_in (u, v, w), kl_step, kl_copy_out (ut, vt, wt)",
           "pipeline": "copy-in, kl_step and copy-out of consecutive steps overlap on three "
                       "streams (two device buffer sets)",
           "link_bound": {"ms_per_step": link_ms, "frac": link_ms / e_ms,
                          "note": "the same bytes as plain contiguous copies, both directions "
                                  "at once: the host link's time for one step"},
           "repeats_ms": [r[0] for r in e_runs],
           "serial": {"value": job_value(world, pts, 1, s_ms), "ms_per_step": s_ms,
                      "repeats_ms": [r[0] for r in s_runs]}}

    cb = None
    if rank == 0 and world == 1:
        cb, _ = cpu_baseline(args.cpu_seconds, OracleSample(f))

    if rank == 0:
        ops = OPS_PER_POINT * pts / (kern_ms * 1e-3)
        alu_roof = None
        if "f32" in op_peaks and args.dtype != "f64":
            alu_roof = {"achieved": ops / 1e12, "peak": op_peaks["f32"] / 1e12, "unit": "Top/s",
                        "frac": ops / op_peaks["f32"], "ops_per_point": OPS_PER_POINT,
                        "peak_source": alu_source,
                        "note": "FP32 FMA-pipe operations (an FMA is one) per point of the "
                                "algorithm, each face flux formed once; peak = measured packed "
                                "FMA rate"}
        line = {
            "metric": METRIC, "value": value, "unit": "Gpts/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": args.dtype, "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": f"{nx}x{ny}x{nz}", "ghosts": G,
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
                                        if peaks.get("hbm_gbs") else "fallback",
                         "alu": alu_roof, "sms": sms},
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
