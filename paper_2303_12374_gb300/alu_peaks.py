"""Arithmetic peaks of the GPU's CUDA cores, measured (the ALU roofs).

The tendency kernels do plain FP32 (or FP64) arithmetic on the CUDA cores, not
tensor-core work, so the roof that can bind them beside HBM is the FMA rate of
those cores.  This module measures it with independent FMA chains:

  * f32    -- scalar fma.rn.f32 (one FMA per thread instruction)
  * f32x2  -- packed fma.rn.f32x2 (two FMAs per thread instruction)
  * f64    -- fma.rn.f64

Each thread runs CH independent chains x <- x * a + b for `iters` rounds, on
enough warps to fill every SM (`blocks_per_sm` blocks of 256 threads).  The
kernels are compiled through the library's own definitions (NVRTC, sm_103a)
and timed with CUDA events after warm-up; nvidia-smi samples the SM clock
while they run, so the rate is also given per SM and clock cycle (FMA lanes).

    python -m paper_2303_12374_gb300.alu_peaks

Prints one JSON object: per kind the TFLOP/s (2 flops per FMA), the FMAs per
SM per cycle at the sampled median clock, and the clock record.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

SOURCE = r"""
extern "C" __global__ void fma_f32(float *out, int iters, float a, float b)
{
    float x[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < CH; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < CH; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

extern "C" __global__ void fma_f32x2(float *out, int iters, float a, float b)
{
    unsigned long long x[CH], av, bv;
    asm("mov.b64 %0, {%1, %1};" : "=l"(av) : "f"(a));
    asm("mov.b64 %0, {%1, %1};" : "=l"(bv) : "f"(b));
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        float lo = (float)(threadIdx.x + c) * 1e-3f, hi = lo + 0.5f;
        asm("mov.b64 %0, {%1, %2};" : "=l"(x[c]) : "f"(lo), "f"(hi));
    }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < CH; ++c)
            asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(x[c]) : "l"(x[c]), "l"(av), "l"(bv));
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[c]));
        s += lo + hi;
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

extern "C" __global__ void fma_f64(double *out, int iters, double a, double b)
{
    double x[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) x[c] = (double)(threadIdx.x + c) * 1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < CH; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < CH; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
"""

# FMAs per thread instruction of each kind
KINDS = {"f32": ("fma_f32", 1, "f32"), "f32x2": ("fma_f32x2", 2, "f32"), "f64": ("fma_f64", 1, "f64")}


class ClockSampler:
    """nvidia-smi samples of the SM clock and the throttle reasons."""

    def __init__(self, index=0):
        self.index, self.proc, self.rows = index, None, []

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out = ""
        for line in out.splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 6 and parts[0].replace(".", "").isdigit():
                self.rows.append(parts)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        return {"sm_mhz": statistics.median(float(r[0]) for r in self.rows),
                "sm_max_mhz": max(float(r[1]) for r in self.rows),
                "reasons": sorted({n for r in self.rows for n, v in zip(names, r[2:])
                                   if v.lower() == "active"}),
                "samples": len(self.rows)}


def measure(kind, chains=8, blocks_per_sm=8, target_ms=40.0, reps=10):
    import torch
    from paper_2303_12374_gb300 import kl
    fn, per_inst, dt = KINDS[kind]
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    nblk, nthr = sms * blocks_per_sm, 256
    d = kl.KernelDef(f"alu_{kind}", SOURCE, fn)
    d.param("CH", [chains], chains)
    d.geometry(block=(str(nthr),), grid=("problem_x",))
    tdt = torch.float32 if dt == "f32" else torch.float64
    out = torch.empty(nblk * nthr, dtype=tdt, device="cuda")
    a, b = 0.9999999, 1e-7
    scal = "f32" if dt == "f32" else "f64"
    work = tempfile.mkdtemp()
    ctx = kl.kl_create(0, work)
    try:
        def launch(iters):
            d.launch_config(ctx, "default", (nblk,), [("out", out), ("i32", iters), (scal, a), (scal, b)])

        iters = 256
        launch(iters)
        torch.cuda.synchronize()
        # grow the loop until one launch takes about target_ms
        while True:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            launch(iters)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            if ms >= target_ms / 4 or iters >= 1 << 24:
                break
            iters *= 4
        iters = max(1, int(iters * target_ms / max(ms, 1e-3)))
        for _ in range(3):
            launch(iters)
        torch.cuda.synchronize()
        with ClockSampler() as clk:
            times = []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                launch(iters)
                e1.record()
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
        ms = statistics.median(times)
        fmas = float(nblk) * nthr * chains * iters * per_inst
        c = clk.summary()
        res = {"tflops": 2 * fmas / (ms * 1e-3) / 1e12, "ms": ms, "iters": iters, "chains": chains,
               "blocks": nblk, "threads": nthr, "clocks": c}
        if c["sm_mhz"]:
            res["fma_per_sm_per_clk"] = fmas / (ms * 1e-3) / (sms * c["sm_mhz"] * 1e6)
            if c["sm_max_mhz"]:
                res["tflops_at_max_clock"] = res["tflops"] * c["sm_max_mhz"] / c["sm_mhz"]
        return res
    finally:
        kl.kl_destroy(ctx)
        d.close()


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--kinds", default="f32,f32x2,f64")
    ap.add_argument("--chains", type=int, default=8)
    ap.add_argument("--blocks-per-sm", type=int, default=8)
    ap.add_argument("--target-ms", type=float, default=40.0)
    args = ap.parse_args(argv)
    import torch
    props = torch.cuda.get_device_properties(0)
    res = {"device": props.name, "sms": props.multi_processor_count}
    for k in args.kinds.split(","):
        res[k] = measure(k, args.chains, args.blocks_per_sm, args.target_ms)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
