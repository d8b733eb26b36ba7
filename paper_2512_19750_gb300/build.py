"""Builds libgace.so in-tree for sm_103a (GB300) with nvcc, one process per
translation unit, then links them.  Used by ``__graft_entry__.build()``."""
from __future__ import annotations

import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libgace.so")
OBJDIR = os.path.join(HERE, "_build")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CUDA_SOURCES = ["gace_probe.cu", "gace_hll_join.cu", "gace_noalloc.cu", "gace_batch.cu", "gace_sample.cu"]
HOST_SOURCES = ["gace_capi.cpp", "gace_batch_host.cpp", "gace_serve.cpp", "gace_gate.cpp", "gace_resident.cpp"]


def cuda_home() -> str:
    env = os.environ.get("CUDA_HOME") or os.environ.get("CUDA_PATH")
    if env and os.path.isdir(env):
        return env
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    return "/usr/local/cuda"


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "gace.h"))
    return files


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in _inputs())


def build(force: bool = False, verbose: bool = False, ptxas_verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    home = cuda_home()
    nvcc = os.path.join(home, "bin", "nvcc")
    if not os.path.exists(nvcc):
        nvcc = "nvcc"
    os.makedirs(OBJDIR, exist_ok=True)
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]
    procs = []
    objs = []
    for src in CUDA_SOURCES:
        obj = os.path.join(OBJDIR, src + ".o")
        cmd = [nvcc, *ARCH, "-lineinfo", *common, "-c", os.path.join(CSRC, src), "-o", obj]
        if ptxas_verbose:
            cmd += ["-Xptxas", "-v"]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    for src in HOST_SOURCES:
        obj = os.path.join(OBJDIR, src + ".o")
        cmd = [nvcc, *common, "-x", "cu", "-c", os.path.join(CSRC, src), "-o", obj, *ARCH]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        text = out.decode(errors="replace")
        if p.returncode != 0:
            failed.append(" ".join(cmd) + "\n" + text)
        elif verbose or ptxas_verbose:
            print(text, end="")
    if failed:
        raise RuntimeError("libgace build failed:\n" + "\n".join(failed))
    libdir = os.path.join(home, "lib64")
    tmp = LIB + ".tmp"
    link = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "shared",
            "-Xlinker", "-rpath," + libdir]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("libgace link failed:\n" + r.stdout.decode(errors="replace"))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys

    print(build(force=True, verbose=True, ptxas_verbose="-v" in sys.argv))
