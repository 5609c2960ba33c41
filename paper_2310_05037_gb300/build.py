"""Builds librawalign_dtw.so in-tree for sm_103a (nvcc, one -gencode).

Each .cu under csrc/ compiles to an object in parallel; the objects link into
paper_2310_05037_gb300/librawalign_dtw.so.  No fast-math: IEEE FP32 with
round-to-nearest, no flush-to-zero, and -fmad=false so no multiply-add can be
contracted anywhere in device code (-ffp-contract=off does the same for the
host compiler).
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
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "librawalign_dtw.so")
BUILD = os.path.join(PKG, "_build")
# the checked build (-DRAWALIGN_CHECKED): the same library with device-side
# checks of every planned work item (extents inside their arrays, ring large
# enough); a failing item is reported (poll returns RA_EDEVICE) and skipped
LIB_CHECKED = os.path.join(PKG, "librawalign_dtw_checked.so")
BUILD_CHECKED = os.path.join(PKG, "_build_checked")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ["-O3", "-lineinfo", "-std=c++17", "-fmad=false", "-Xcompiler", "-fPIC",
           "-Xcompiler", "-fno-fast-math", "-Xcompiler", "-ffp-contract=off", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    p = os.path.join(home, "bin", "nvcc")
    return p if os.path.exists(p) else (shutil.which("nvcc") or "nvcc")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _stale(lib=LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = sources() + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    deps.append(os.path.join(INCLUDE, "rawalign_dtw.h"))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra=(), checked: bool = False) -> str:
    lib, bdir = (LIB_CHECKED, BUILD_CHECKED) if checked else (LIB, BUILD)
    if checked:
        extra = tuple(extra) + ("-DRAWALIGN_CHECKED",)
    if not force and not _stale(lib):
        return lib
    os.makedirs(bdir, exist_ok=True)

    def comp(src):
        obj = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc(), *ARCH, *NVFLAGS, *extra, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        if verbose:
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=max(2, os.cpu_count() or 2)) as ex:
        objs = list(ex.map(comp, sources()))
    tmp = lib + ".%d.tmp" % os.getpid()
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                extra=(["-Xptxas", "-v"] if "--ptxas" in sys.argv else []), checked="--checked" in sys.argv))
