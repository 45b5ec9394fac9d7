"""Build libhfx.so in-tree with nvcc for sm_103a (GB300).

Five translation units compiled in parallel: the FP64 kernels, the
split-precision kernels, the tcgen05 first-product kernel, the split-precision
kernels for wide blocks and the C++ host planner/ABI.  The result is written next to this file.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libhfx.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def build(verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    inc = ["-I", os.path.join(ROOT, "include"), "-I", CSRC]
    units = {
        "hfx_kernels.o": [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", *inc,
                          "-c", os.path.join(CSRC, "hfx_kernels.cu")],
        "hfx_mixed.o": [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", *inc,
                        "-c", os.path.join(CSRC, "hfx_mixed.cu")],
        "hfx_t1umma.o": [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", *inc,
                         "-c", os.path.join(CSRC, "hfx_t1umma.cu")],
        "hfx_wide.o": [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", *inc,
                       "-c", os.path.join(CSRC, "hfx_wide.cu")],
        "hfx_host.o": [nvcc, *ARCH, "-O2", "-std=c++17", "-Xcompiler", "-fPIC", *inc,
                       "-x", "cu", "-c", os.path.join(CSRC, "hfx_host.cpp")],
    }
    procs = []
    for obj, cmd in units.items():
        cmd = cmd + ["-o", os.path.join(BUILD, obj)]
        if verbose:
            print(" ".join(cmd), flush=True)
        procs.append((obj, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
    failed = []
    for obj, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append(f"{obj}:\n{out}")
        elif verbose and out.strip():
            print(out)
    if failed:
        raise RuntimeError("nvcc failed\n" + "\n".join(failed))
    link = [nvcc, *ARCH, "-shared", "-o", LIB + ".tmp"] + [os.path.join(BUILD, o) for o in units]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed\n" + r.stdout + r.stderr)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
