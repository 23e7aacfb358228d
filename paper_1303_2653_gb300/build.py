"""In-tree build of the package's native libraries.

- ``liblbdps.so``: the CUDA library behind ``include/lbdps.h`` (sm_103a).
- ``libworkloads.so``: the seeded input generator (plain C).
"""
from __future__ import annotations

import concurrent.futures as _cf
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")
BUILD_DIR = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _newer(out, srcs):
    if not os.path.exists(out):
        return False
    t = os.path.getmtime(out)
    return all(os.path.getmtime(s) <= t for s in srcs)


def build_workloads(force: bool = False) -> str:
    src = os.path.join(CSRC, "workloads.c")
    out = os.path.join(HERE, "libworkloads.so")
    if force or not _newer(out, [src]):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, src, "-lm"],
                       check=True)
        os.replace(tmp, out)
    return out
