"""Build libdgf.so in-tree for sm_103a (nvcc + g++, no cmake).

Translation units compile in parallel; the shared library links the CUDA
runtime statically.  Run as ``python -m paper_2502_12620_gb300.build``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libdgf.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def sources():
    cu = sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))
    cpp = sorted(f for f in os.listdir(CSRC) if f.endswith(".cpp"))
    return cu, cpp


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def build(verbose=False, ptxas_info=False, jobs=None):
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    cu, cpp = sources()
    cmds = []
    objs = []
    for f in cu:
        o = os.path.join(BUILD, f[:-3] + ".o")
        objs.append(o)
        c = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
             "--expt-relaxed-constexpr", "-c", os.path.join(CSRC, f), "-o", o]
        if "_f32" in f:
            # FP32 kernels: hardware-approximate divide and square root (a few
            # ulp, far inside the FP32 parity bar; denormals are kept)
            c[1:1] = ["-prec-div=false", "-prec-sqrt=false"]
        # extra -D flags for tuning sweeps (e.g. DGF_NVCC_DEFINES="-DDGF_STAGE_NT_F32=576")
        c[1:1] = os.environ.get("DGF_NVCC_DEFINES", "").split()
        if ptxas_info:
            c.insert(1, "-Xptxas=-v")
        cmds.append(c)
    for f in cpp:
        o = os.path.join(BUILD, f[:-4] + ".o")
        objs.append(o)
        cmds.append(["g++", "-O2", "-std=c++17", "-fPIC", "-c", os.path.join(CSRC, f), "-o", o])
    jobs = jobs or min(len(cmds), os.cpu_count() or 4)
    logs = []
    with cf.ThreadPoolExecutor(jobs) as ex:
        for out in ex.map(_run, cmds):
            logs.append(out)
    tmp = LIB + ".tmp"
    _run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"])
    os.replace(tmp, LIB)
    if verbose:
        for l in logs:
            if l.strip():
                print(l)
    return LIB


if __name__ == "__main__":
    build(verbose=True, ptxas_info="--ptxas" in sys.argv)
    print(LIB)
