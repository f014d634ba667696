"""Build libgdr.so (the CUDA library behind include/gdr.h) in-tree for sm_103a.

    python -m paper_0707_0502_gb300.build [--force] [--verbose]

Each translation unit is compiled by nvcc in parallel into ``_build/``; the
objects are linked into ``paper_0707_0502_gb300/libgdr.so`` (CUDA runtime
linked statically).  A rebuild happens only when a source or header is newer
than the library.
"""
from __future__ import annotations

import os
import platform
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libgdr.so")
SOURCES = ["ops.cu", "krylov.cu", "sweep.cu", "dense.cu", "solver.cu", "capi.cu", "noalloc.cu", "tune.cu",
           "tc_proj.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC] + ARCH


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "gdr.h"))
    return files


def _elf_machine(path):
    with open(path, "rb") as f:
        head = f.read(20)
    return int.from_bytes(head[18:20], "little") if head[:4] == b"\x7fELF" else None


_MACHINES = {"x86_64": 62, "aarch64": 183, "arm64": 183}


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    if _elf_machine(LIB) != _MACHINES.get(platform.machine()):
        return False  # built on another architecture
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def _run(cmd, verbose):
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed ({r.returncode}): {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return r.stderr


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    objs = [os.path.join(BUILD, os.path.splitext(s)[0] + ".o") for s in SOURCES]
    cmds = [[NVCC] + FLAGS + ["-c", os.path.join(CSRC, s), "-o", o] for s, o in zip(SOURCES, objs)]
    with ThreadPoolExecutor(max_workers=len(cmds)) as ex:
        list(ex.map(lambda c: _run(c, verbose), cmds))
    tmp = LIB + ".tmp"
    _run([NVCC] + ARCH + ["-shared", "-o", tmp] + objs, verbose)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="--verbose" in sys.argv))
