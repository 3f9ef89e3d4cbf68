"""Build ``libpolar_gb300.so`` in-tree with nvcc for sm_103a.

Eight objects compile in parallel: the host runtime, the list kernels in four
parts (float / int8 x plain / batched form, one source compiled with
-DPOLAR_KPART=0..3), the wide-list kernel and the two L = 1 kernels (many
frames: a lane each; small batches: a warp each). They are linked
into one shared library next to this file. No CMake, no torch extension
machinery: the library has a plain C ABI (include/polar.h).
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libpolar_gb300.so")
SOURCES = ["polar_capi.cu", "polar_kernels.cu", "polar_wide.cu", "polar_sc1.cu", "polar_sc1w.cu"]
# (source, object, extra flags): the list kernels compile once per part
UNITS = [("polar_capi.cu", "polar_capi.o", []),
         *[("polar_kernels.cu", f"polar_kernels_p{p}.o", [f"-DPOLAR_KPART={p}", "-diag-suppress", "177"])
           for p in range(4)],   # a part leaves the other parts' helpers unused
         ("polar_wide.cu", "polar_wide.o", []),
         ("polar_sc1.cu", "polar_sc1.o", []),
         ("polar_sc1w.cu", "polar_sc1w.o", [])]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "-DPOLAR_BUILD"]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(os.path.dirname(HERE), "include", "polar.h"))
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    bdir = os.path.join(HERE, "_build")
    os.makedirs(bdir, exist_ok=True)
    procs, objs = [], []
    for src, o, extra in UNITS:
        obj = os.path.join(bdir, o)
        cmd = [NVCC, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((subprocess.Popen(cmd), src))
        objs.append(obj)
    for p, src in procs:
        if p.wait() != 0:
            raise RuntimeError(f"nvcc failed on {src}")
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.run([NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"], check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
