"""Build libmirres.so in-tree with nvcc for sm_103a (GB300).

The translation units are compiled in parallel and linked into one shared library with the
CUDA runtime linked dynamically (the process shares one runtime with PyTorch).
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libmirres.so")
UNITS = ["abi.cu", "bvh.cu", "wbvh.cu", "env.cu", "render.cu", "wave.cu", "noalloc.cu", "denoise.cu",
         "regular.cu", "peaks.cu"]
HEADERS = ["device.cuh", "path.cuh", "internal.h", "render.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _inputs():
    files = [os.path.join(CSRC, f) for f in UNITS + HEADERS] + [os.path.join(INCLUDE, h)
                                                               for h in ("mirres.h", "mirres_peaks.h")]
    return files


STAMP = os.path.join(BUILD, "flags.txt")


def extra_flags() -> list:
    """MIRRES_NVCC_FLAGS: extra nvcc flags, e.g. the launch knobs -DMR_SHADE_MINB=3."""
    return os.environ.get("MIRRES_NVCC_FLAGS", "").split()


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    if not os.path.exists(STAMP) or open(STAMP).read() != " ".join(extra_flags()):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in _inputs())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-v",
                    "-I", CSRC, "-I", INCLUDE] + extra_flags()
    procs, objs = [], []
    for u in UNITS:
        obj = os.path.join(BUILD, u.replace(".cu", ".o"))
        log = open(os.path.join(BUILD, u.replace(".cu", ".log")), "w")
        p = subprocess.Popen([nvcc()] + flags + ["-c", os.path.join(CSRC, u), "-o", obj], stdout=log,
                             stderr=subprocess.STDOUT)
        procs.append((u, p, log))
        objs.append(obj)
    failed = []
    for u, p, log in procs:
        p.wait()
        log.close()
        if p.returncode != 0:
            failed.append(u)
    if failed:
        msgs = []
        for u in failed:
            msgs.append(open(os.path.join(BUILD, u.replace(".cu", ".log"))).read()[-4000:])
        raise RuntimeError("nvcc failed for %s:\n%s" % (failed, "\n".join(msgs)))
    tmp = LIB + ".tmp%d" % os.getpid()
    subprocess.run([nvcc()] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs, check=True)
    os.replace(tmp, LIB)
    with open(STAMP, "w") as f:
        f.write(" ".join(extra_flags()))
    if verbose:
        for u in UNITS:
            sys.stdout.write(open(os.path.join(BUILD, u.replace(".cu", ".log"))).read())
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
