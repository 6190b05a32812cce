"""Builds libecl.so in-tree with nvcc for sm_103a (no torch extension machinery).

Each .cu file is compiled to an object in parallel, then the objects are
linked into one shared library next to this file.  The Mandelbrot and
ray-tracing units are compiled with -fmad=false (their results must match a
correctly rounded host evaluation bit for bit).  The NBody unit is compiled
with -ftz=true: every FP32 value there is far from the subnormal range
(r^2 >= eps^2 > 0), and without subnormal handling rsqrtf is the bare
hardware reciprocal square root instead of a range check, a scaling and the
root.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libecl.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

# source -> extra flags
SOURCES = {
    "runtime.cu": [],
    "registry.cu": [],
    "k_mandelbrot.cu": ["-fmad=false"],
    "k_gaussian.cu": [],
    "k_nbody.cu": ["-ftz=true"],
    "k_binomial.cu": [],
    "k_gemm.cu": [],
    "k_gemm6.cu": [],
    "k_ray.cu": ["-fmad=false"],
    "k_probe.cu": [],
}
HEADERS = ["ecl_internal.h", "sched.cuh", "f32x2.cuh", "tc.cuh"]
LFACT = "lfact_table.inc"  # generated into _build: ln k! for k = 0..2048 as FP32 (hi, lo) pairs


def write_lfact_table(path: str, kmax: int = 2048) -> None:
    """ln k! (math.lgamma(k + 1), double precision) split into two FP32
    values hi + lo, written as C hex-float initialisers for the binomial
    kernel's closed-form leaf weights.  hi is the value rounded to a multiple
    of 2^-10 (below 2^14 for k <= 2048, so exact in FP32), so that sums of hi
    parts are exact in FP32; lo (at most 2^-11) is the FP32 remainder."""
    import math
    import struct

    def f32(x: float) -> float:
        return struct.unpack("<f", struct.pack("<f", x))[0]

    lines = []
    for k in range(kmax + 1):
        v = math.lgamma(k + 1.0)
        hi = round(v * 1024.0) / 1024.0
        assert f32(hi) == hi and abs(hi) < 2.0 ** 14
        lo = f32(v - hi)
        lines.append("{%sf, %sf}," % (float.hex(hi), float.hex(lo)))
    text = "\n".join(lines) + "\n"
    if not os.path.exists(path) or open(path).read() != text:
        with open(path, "w") as f:
            f.write(text)


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _stale(obj: str, deps) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, force: bool = False, jobs: int = 8) -> str:
    os.makedirs(OBJ, exist_ok=True)
    write_lfact_table(os.path.join(OBJ, LFACT))
    cc = nvcc()
    inc = os.path.join(os.path.dirname(HERE), "include")
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(inc, "ecl.h"), __file__]
    common = [cc, *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
              "-I", inc, "-I", OBJ, "--expt-relaxed-constexpr"]
    cmds = []
    objs = []
    for src, extra in SOURCES.items():
        s = os.path.join(CSRC, src)
        o = os.path.join(OBJ, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + hdrs):
            cmds.append(common + extra + ["-c", s, "-o", o])

    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n%s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, flush=True)

    if cmds:
        with ThreadPoolExecutor(max_workers=jobs) as ex:
            list(ex.map(run, cmds))
    if force or cmds or not os.path.exists(LIB) or _stale(LIB, objs):
        tmp = LIB + ".tmp%d" % os.getpid()
        run([cc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
