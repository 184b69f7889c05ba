"""Build of the native library ``_build/liblskum.so`` (sm_103a) and the probe.

Translation units are compiled in parallel: the CUDA files with nvcc for
``sm_103a`` only, the host set-up with g++ (``-ffp-contract=off``: the
split-stencil membership must be decided on exact FP64 products), then linked
into one shared library with a C ABI (``include/lskum.h``).
"""

from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liblskum.so")
PROBE = os.path.join(BUILD, "pipe_peaks")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CUDA_SOURCES = ["lskum_kernels.cu", "lskum_kernels_mixed.cu", "lskum_api.cu", "lskum_noalloc.cu",
                "mlp_kernels.cu"]
HOST_SOURCES = ["lskum_setup.cpp"]
HEADERS = ["lskum_internal.h", "lskum_kernels.cuh", "math_tables.h", "device_math.cuh"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblskum")


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, fmad: bool = True) -> str:
    """Compile (if stale) and return the path of ``liblskum.so``."""
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    inc = os.path.join(os.path.dirname(HERE), "include")
    headers = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(inc, "lskum.h"),
                                                           os.path.join(inc, "lskum_mlp.h")]
    cuda_flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", inc,
                         "--fmad=true" if fmad else "--fmad=false"]
    jobs = []
    objs = []
    for src in CUDA_SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src + ".o")
        objs.append(o)
        if force or _stale(o, [s] + headers):
            jobs.append([nvcc] + cuda_flags + ["-c", s, "-o", o])
    for src in HOST_SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src + ".o")
        objs.append(o)
        if force or _stale(o, [s] + headers):
            jobs.append(["g++", "-O2", "-ffp-contract=off", "-fPIC", "-fopenmp", "-std=c++17",
                         "-I", inc, "-c", s, "-o", o])
    probe_src = os.path.join(CSRC, "pipe_peaks.cu")
    if force or _stale(PROBE, [probe_src]):
        jobs.append([nvcc] + ARCH + ["-O3", "-o", PROBE, probe_src])
    procs = [(j, subprocess.Popen(j, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)) for j in jobs]
    failed = []
    for j, p in procs:
        out, _ = p.communicate()
        if verbose and out:
            sys.stdout.write(out.decode(errors="replace"))
        if p.returncode != 0:
            failed.append((j, out.decode(errors="replace")))
    if failed:
        msg = "\n".join(" ".join(j) + "\n" + o for j, o in failed)
        raise RuntimeError("liblskum build failed:\n" + msg)
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-Xcompiler", "-fopenmp"],
                       check=True)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
