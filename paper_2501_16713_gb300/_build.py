"""Build the in-tree CUDA library libnrsense.so for sm_103a with nvcc.

Each translation unit is compiled in parallel into paper_2501_16713_gb300/_build/
and linked with cuFFT into paper_2501_16713_gb300/libnrsense.so.  The build is
incremental: a source newer than its object (or a header newer than any
object) triggers a recompile.
"""

from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libnrsense.so")
INCLUDE = os.path.join(ROOT, "include")

SOURCES = [
    "kb_host.cu",
    "plan.cu",
    "apply.cu",
    "kernels_image.cu",
    "kernels_kspace.cu",
    "kernels_spread.cu",
    "solver.cu",
    "noalloc.cu",
    "cnn.cu",
    "fista.cu",
    "motion.cu",
    "fft_pruned.cu",
    "spread_home.cu",
]
HEADERS = ["common.cuh", "plan_internal.h", "kb_host.h"]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libnrsense")
    return cand


def _cuda_lib_dir(nvcc):
    root = os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    for sub in ("lib64", "lib", "targets/sbsa-linux/lib", "targets/x86_64-linux/lib"):
        d = os.path.join(root, sub)
        if os.path.exists(os.path.join(d, "libcufft.so")):
            return d
    return os.path.join(root, "lib64")


def _mtime(path):
    try:
        return os.path.getmtime(path)
    except OSError:
        return -1.0


def build(verbose: bool = False, force: bool = False, extra_flags=None) -> str:
    """Compile (if needed) and return the path of libnrsense.so."""
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    hdr_time = max(_mtime(os.path.join(CSRC, h)) for h in HEADERS)
    hdr_time = max(hdr_time, _mtime(os.path.join(INCLUDE, "nrsense.h")))
    flags = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE,
             "--expt-relaxed-constexpr"] + ARCH + list(extra_flags or [])
    jobs = []
    objs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _mtime(o) < max(_mtime(s), hdr_time):
            jobs.append([nvcc, "-c", s, "-o", o] + flags)
    if jobs:
        def run(cmd):
            r = subprocess.run(cmd, capture_output=True, text=True)
            return cmd, r
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            for cmd, r in ex.map(run, jobs):
                if verbose or r.returncode != 0:
                    sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
                if r.returncode != 0:
                    raise RuntimeError(f"nvcc failed on {cmd[2]}")
    if force or jobs or _mtime(LIB) < max(_mtime(o) for o in objs):
        libdir = _cuda_lib_dir(nvcc)
        cmd = [nvcc, "-shared", "-o", LIB] + objs + ARCH + [
            "-L", libdir, "-lcufft", "-Xlinker", "-rpath," + libdir]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if verbose or r.returncode != 0:
            sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError("linking libnrsense.so failed")
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
