"""Compile libsd.so (the CUDA library behind include/sd.h) for sm_103a.

In-tree build: objects and the library go to paper_2108_10480_gb300/_build/.
Each translation unit compiles in its own nvcc process, in parallel.
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
LIB = os.path.join(BUILD, "libsd.so")
INCLUDE = os.path.join(ROOT, "include")

SOURCES = ["sd_api.cu", "sd_build.cu", "sd_query.cu", "sd_pose.cu", "sd_mlp.cu", "sd_mesh.cu", "sd_trace.cu", "sd_peak.cu", "sd_weights_host.cpp"]
HEADERS = ["sd_common.cuh", "sd_sort.cuh", "sd_pairs.cuh", "sd_wtab.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


def _stale(lib=LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, s) for s in SOURCES + HEADERS] + [os.path.join(INCLUDE, "sd.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False, tag: str = "", defines=()) -> str:
    """Build libsd.so; with a tag, a separate library _build/libsd_<tag>.so
    compiled with the extra -D `defines` (test-only builds, e.g. with the
    device-side wait limits lowered)."""
    lib = os.path.join(BUILD, f"libsd_{tag}.so") if tag else LIB
    objdir = os.path.join(BUILD, tag) if tag else BUILD
    if not force and not _stale(lib):
        return lib
    os.makedirs(objdir, exist_ok=True)
    nvcc = _nvcc()
    common = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]
    common += ["-D" + d for d in defines]
    procs = []
    objs = []
    for s in SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(objdir, os.path.splitext(s)[0] + ".o")
        objs.append(obj)
        if s.endswith(".cu"):
            cmd = [nvcc] + ARCH + common + ["-c", src, "-o", obj]
        else:
            cmd = [nvcc] + common + ["-x", "c++", "-c", src, "-o", obj]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if verbose and out:
            sys.stdout.write(out.decode(errors="replace"))
        if p.returncode != 0:
            failed.append((" ".join(cmd), out.decode(errors="replace")))
    if failed:
        raise RuntimeError("libsd build failed:\n" + "\n".join(f"$ {c}\n{o}" for c, o in failed))
    tmp = lib + f".{os.getpid()}.tmp"
    cmd = [nvcc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("libsd link failed:\n" + r.stdout.decode(errors="replace"))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
