"""Builds librrg.so, the CUDA library behind include/rrg.h, for sm_103a.

Each translation unit is compiled by nvcc in parallel, then linked into one
shared object next to this file (in-tree, git-ignored).  The CUDA runtime is
linked statically so the library loads without a toolkit on the loader path.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import platform
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build", platform.machine())
LIB = os.path.join(HERE, "librrg.so")
SOURCES = ("rrg_kernels.cu", "rrg_capi.cu", "rrg_static.cu", "rrg_adjoint.cu", "rrg_batch.cu",
           "rrg_peaks.cu", "rrg_error.cu")
HEADERS = ("rrg_device.cuh", "rrg_internal.h", "rrg_lane.cuh")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# -ftz=true: the binary32 rollouts never meet subnormal values, and flushing
# lets lg2/ex2/rcp issue as single MUFU operations on the critical path
# -ffp-contract=off for the host compiler: host code folds constants the
# device folds too (fold_rhs) and must not fuse them differently
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-ftz=true", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
              "-Xcompiler", "-ffp-contract=off",
              "-Xcompiler", "-fvisibility=hidden", "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build librrg")


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags=(), out: str = None,
          build_dir: str = None) -> str:
    """Compiles and links librrg.so (or `out`, with objects in `build_dir`)."""
    lib_path = out or LIB
    bdir = build_dir or BUILD
    stamp = os.path.join(bdir, "librrg.stamp")
    os.makedirs(bdir, exist_ok=True)
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", "rrg.h")]
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(bdir, src + ".o")
        if force or _stale(o, [s] + hdrs):
            jobs.append([nvcc(), *ARCH, *NVCC_FLAGS, *extra_flags, "-c", s, "-o", o])

    def run(cmd):
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError("nvcc failed:\n%s\n%s" % (" ".join(cmd), p.stdout + p.stderr))
        if verbose and (p.stdout or p.stderr):
            print(p.stdout + p.stderr, file=sys.stderr)

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        list(ex.map(run, jobs))
    objs = [os.path.join(bdir, s + ".o") for s in SOURCES]
    # the stamp records which machine linked librrg.so, so a library copied
    # from another architecture is relinked from this machine's objects
    if force or jobs or _stale(lib_path, objs) or not os.path.exists(stamp):
        tmp = lib_path + ".tmp%d" % os.getpid()
        run([nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs])
        os.replace(tmp, lib_path)
        with open(stamp, "w") as f:
            f.write(platform.machine() + "\n")
    return lib_path


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
