"""Builds librteaal.so in-tree for sm_103a (no cmake; translation units in parallel)."""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT = os.path.join(HERE, "librteaal.so")
BUILD = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for c in [os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"]:
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def sources():
    return [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC))
            if f.endswith((".cu", ".cpp", ".cuh", ".hpp", ".h"))] + [os.path.join(INCLUDE, "rteaal.h")]


def up_to_date() -> bool:
    if not os.path.exists(OUT):
        return False
    t = os.path.getmtime(OUT)
    return all(os.path.getmtime(s) <= t for s in sources() + [os.path.abspath(__file__)])


def build(force: bool = False, verbose: bool = False, ptxas_v: bool = False) -> str:
    if not force and up_to_date():
        return OUT
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    common = ["-O3", "-std=c++17", "-I", INCLUDE, "-I", CSRC]
    jobs = []
    objs = []
    # the persistent-kernel variants are instantiated in their own units so that
    # they compile in parallel with the runtime
    units = ["rteaal.cu"] + sorted(f for f in os.listdir(CSRC) if f.startswith("variants_") and f.endswith(".cu")) + [
        "lower.cpp", "inspect.cpp", "specialize.cpp"]
    for f in units:
        src = os.path.join(CSRC, f)
        obj = os.path.join(BUILD, f + ".o")
        cmd = [nvcc] + ARCH + common + ["-lineinfo", "-Xcompiler", "-fPIC,-fvisibility=hidden",
                                         "-c", src, "-o", obj]
        if f.endswith(".cu"):
            cmd += ["--expt-relaxed-constexpr"]
            if ptxas_v:
                cmd += ["-Xptxas", "-v"]
        jobs.append(subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True))
        objs.append(obj)
    logs = []
    for j in jobs:
        out, _ = j.communicate()
        logs.append(out)
        if j.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + out)
    tmp = OUT + ".tmp%d" % os.getpid()
    cuda_lib = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "lib64")
    link = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-L" + cuda_lib, "-lnvrtc",
                                                            "-Xlinker", "-rpath," + cuda_lib]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout)
    os.replace(tmp, OUT)
    if verbose:
        sys.stdout.write("".join(logs))
    return OUT


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_v="-v" in sys.argv)
    print(OUT)
