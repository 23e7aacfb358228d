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


CU_SOURCES = ["lbm_kernels.cu", "particle_kernels.cu", "stats_kernels.cu", "lbdps_api.cu",
              "lbdps_server.cu", "noalloc_sort.cu", "bubble_kernels.cu", "contact_kernels.cu"]
HEADERS = ["lbdps_internal.cuh", "particle_common.cuh"]


def nvcc_flags(extra=()):
    return ["-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC,-O2",
            f"-I{INCLUDE}", f"-I{CSRC}", *extra]


def build_lbdps(force: bool = False, verbose_ptxas: bool = False, jobs: int = 4) -> str:
    """Compile the CUDA library into ``liblbdps.so`` next to this file."""
    out = os.path.join(HERE, "liblbdps.so")
    srcs = [os.path.join(CSRC, s) for s in CU_SOURCES]
    deps = srcs + [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(INCLUDE, "lbdps.h")]
    if not force and _newer(out, deps):
        return out
    os.makedirs(BUILD_DIR, exist_ok=True)
    extra = ["-Xptxas", "-v"] if verbose_ptxas else []

    def compile_one(src):
        obj = os.path.join(BUILD_DIR, os.path.basename(src) + ".o")
        cmd = ["nvcc", *nvcc_flags(extra), "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with _cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        results = list(ex.map(compile_one, srcs))
    if verbose_ptxas:
        for _, log in results:
            print(log)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["nvcc", *ARCH, "-shared", "-o", tmp, *[o for o, _ in results], "-lcudart"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build_all(force: bool = False) -> None:
    build_workloads(force)
    build_lbdps(force)


if __name__ == "__main__":
    import sys
    build_workloads(force=True)
    print(build_lbdps(force=True, verbose_ptxas="-v" in sys.argv))
