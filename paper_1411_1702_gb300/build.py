"""Build the CUDA library libpf_gb300.so in-tree for sm_103a (GB300).

Each translation unit under ``csrc/`` is compiled by nvcc in parallel, then
linked into one shared library that exports the C ABI of ``include/pf.h``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libpf_gb300.so")
# probes outside the C ABI, in a library of their own: the benchmark's FP64 FMA
# probe and the device side of the test of the table-driven math routines
PROBE_SRCS = [os.path.join(CSRC, "probe", f) for f in ("fp64_fma_probe.cu", "math_probe.cu")]
PROBE_LIB = os.path.join(HERE, "libpf_fp64_probe.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--threads", "1"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpf_gb300.so")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _deps():
    out = [os.path.join(ROOT, "include", "pf.h")]
    out += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    return out


def stale() -> bool:
    for lib, deps in ((LIB, sources() + _deps()), (PROBE_LIB, PROBE_SRCS + _deps())):
        if not os.path.exists(lib):
            return True
        t = os.path.getmtime(lib)
        if any(os.path.getmtime(p) > t for p in deps + [__file__]):
            return True
    return False


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not stale():
        return LIB
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    probe_tmp = PROBE_LIB + f".tmp{os.getpid()}"
    probe = subprocess.Popen([nvcc, *ARCH, *FLAGS, "-shared", *PROBE_SRCS, "-o", probe_tmp],
                             stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    procs = []
    objs = []
    for src in sources():
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        objs.append(obj)
        cmd = [nvcc, *ARCH, *FLAGS, "-c", src, "-o", obj]
        if verbose:
            cmd += ["-Xptxas", "-v"]
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode != 0:
            sys.stderr.write(out.decode(errors="replace"))
        if p.returncode != 0:
            failed.append(src)
    out, _ = probe.communicate()
    if verbose or probe.returncode != 0:
        sys.stderr.write(out.decode(errors="replace"))
    if probe.returncode != 0:
        failed.append(" ".join(PROBE_SRCS))
    if failed:
        raise RuntimeError("nvcc failed on: " + ", ".join(failed))
    os.replace(probe_tmp, PROBE_LIB)
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
