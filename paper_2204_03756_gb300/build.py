"""In-tree build of the CUDA library ``libmtpt.so`` for sm_103a (GB300).

One translation unit (``csrc/mtpt.cu``) compiled by nvcc with
``-gencode arch=compute_103a,code=sm_103a``; the shared object lands in
``paper_2204_03756_gb300/_lib/`` next to the package, so the process that
imports the package loads it from the source tree.  A second object,
``libmtpt_checked.so``, is the same source with ``-DMTPT_CHECKED`` (run-time
bounds checks of the kernels' index invariants, for the tests); both compile
in parallel.
"""
from __future__ import annotations

import os
import shutil
import subprocess

PKG_DIR = os.path.dirname(os.path.abspath(__file__))
SRC_DIR = os.path.join(PKG_DIR, "csrc")
INCLUDE_DIR = os.path.join(os.path.dirname(PKG_DIR), "include")
LIB_DIR = os.path.join(PKG_DIR, "_lib")
LIB_PATH = os.path.join(LIB_DIR, "libmtpt.so")
LIB_CHECKED_PATH = os.path.join(LIB_DIR, "libmtpt_checked.so")
VARIANTS = ((LIB_PATH, ()), (LIB_CHECKED_PATH, ("-DMTPT_CHECKED",)))
ARCH_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _sources():
    out = [os.path.join(INCLUDE_DIR, "mtpt.h")]
    for name in sorted(os.listdir(SRC_DIR)):
        if name.endswith((".cu", ".cuh", ".h")):
            out.append(os.path.join(SRC_DIR, name))
    return out


def nvcc_path() -> str:
    home = os.environ.get("CUDA_HOME") or os.environ.get("CUDA_PATH") or "/usr/local/cuda"
    cand = os.path.join(home, "bin", "nvcc")
    if os.path.exists(cand):
        return cand
    found = shutil.which("nvcc")
    if not found:
        raise RuntimeError("nvcc not found: set CUDA_HOME or put nvcc on PATH")
    return found


def build_command(out_path: str = LIB_PATH, extra=()) -> list:
    # host code without contraction into fused multiply-adds: the same host
    # arithmetic (grid and tile tables) on x86 and Arm builds
    return [nvcc_path(), *ARCH_FLAGS, "-O3", "-lineinfo", "-std=c++17",
            "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off", "-shared", "-I",
            INCLUDE_DIR, *extra,
            "-o", out_path, os.path.join(SRC_DIR, "mtpt.cu")]


def needs_build(path: str = LIB_PATH) -> bool:
    if not os.path.exists(path):
        return True
    t = os.path.getmtime(path)
    return any(os.path.getmtime(s) > t for s in _sources())


def start_build(force: bool = False):
    """Launch nvcc for every out-of-date variant in the background; returns
    the list of (Popen, temporary path, final path)."""
    os.makedirs(LIB_DIR, exist_ok=True)
    jobs = []
    for path, extra in VARIANTS:
        if not force and not needs_build(path):
            continue
        tmp = path + f".tmp{os.getpid()}"
        proc = subprocess.Popen(build_command(tmp, extra), stdout=subprocess.PIPE,
                                stderr=subprocess.STDOUT, text=True)
        jobs.append((proc, tmp, path))
    return jobs


def finish_build(jobs) -> str:
    errors = []
    for proc, tmp, path in jobs or ():
        out, _ = proc.communicate()
        if proc.returncode != 0:
            errors.append(f"nvcc failed for {os.path.basename(path)} ({proc.returncode}):\n{out}")
            continue
        os.replace(tmp, path)
    if errors:
        raise RuntimeError("\n".join(errors))
    return LIB_PATH


def build(force: bool = False) -> str:
    return finish_build(start_build(force))


if __name__ == "__main__":
    print(build(force=True))
