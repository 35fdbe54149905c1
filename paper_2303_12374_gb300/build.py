"""Build libkl.so in-tree with nvcc for sm_103a (no cmake).

The tendency kernels themselves are compiled at run time by NVRTC; their
source (csrc/kl_stencil.cuh) is embedded into the library as a string.  The
ghost-fill and diagnostic kernels are compiled here by nvcc.
"""

from __future__ import annotations

import hashlib
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libkl.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
CUDA_LIB = "/usr/local/cuda/lib64"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["kl_api.cpp", "kl_config.cpp", "kl_tune.cpp", "kl_bayes.cpp", "kl_def.cpp", "kl_device.cu"]


def _embed_source() -> str:
    """Write the NVRTC source as a raw string literal include."""
    src = open(os.path.join(CSRC, "kl_stencil.cuh")).read()
    inc = os.path.join(OUT, "kl_source.inc")
    body = 'R"KLSRC(' + src + ')KLSRC"\n'
    if not os.path.exists(inc) or open(inc).read() != body:
        with open(inc, "w") as f:
            f.write(body)
    return inc


def _digest() -> str:
    h = hashlib.sha256()
    for name in sorted(os.listdir(CSRC)):
        with open(os.path.join(CSRC, name), "rb") as f:
            h.update(name.encode() + f.read())
    with open(os.path.join(ROOT, "include", "kl.h"), "rb") as f:
        h.update(f.read())
    h.update(" ".join(ARCH).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    stamp = os.path.join(OUT, "libkl.stamp")
    dig = _digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read() == dig:
        return LIB
    _embed_source()
    inc = ["-I", os.path.join(ROOT, "include"), "-I", CSRC, "-I", OUT]
    common = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-Wall"] + ARCH + inc

    def compile_one(src: str) -> str:
        obj = os.path.join(OUT, os.path.splitext(src)[0] + ".o")
        cmd = [NVCC] + common + ["-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cu"):
            cmd += ["-Xptxas", "-v"] if verbose else []
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + objs + [
        "-L" + CUDA_LIB, "-lnvrtc", "-lpthread", "-Xlinker", "-rpath," + CUDA_LIB]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(dig)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
