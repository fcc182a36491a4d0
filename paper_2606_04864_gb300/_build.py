"""Build the AMS CUDA library (libams.so) in-tree for sm_103a.

Compiles every translation unit under ``csrc/`` with nvcc in parallel and
links them into ``paper_2606_04864_gb300/libams.so``.  Object files go to
``_build/`` at the repository root.  A source is recompiled only when it,
or a header it may include, is newer than its object.

``build(debug=True)`` makes the checking variant ``libams_debug.so`` from
the same sources with ``-DAMS_DEBUG`` (objects under ``_build/debug/``):
device-side index checks on the gathers record the failing site in an
error word and skip the access; the host API turns a recorded site into
AMS_ERR_CUDA.  The package loads it instead of libams.so when the
environment variable AMS_LIBRARY is ``debug``.
"""

from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libams.so")
LIB_DEBUG = os.path.join(PKG, "libams_debug.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O3",
         "-I", os.path.join(ROOT, "include")]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the AMS library needs the CUDA toolkit to build")


def _cuda_lib_dir(nvcc: str) -> str:
    return os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "lib64")


def _compile(nvcc: str, src: str, obj: str, extra: tuple = ()) -> tuple[str, int, str]:
    cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
    p = subprocess.run(cmd, capture_output=True, text=True)
    return src, p.returncode, (p.stdout + p.stderr)


def build(verbose: bool = False, force: bool = False, debug: bool = False) -> str:
    nvcc = _nvcc()
    bdir = os.path.join(BUILD, "debug") if debug else BUILD
    lib = LIB_DEBUG if debug else LIB
    extra = ("-DAMS_DEBUG",) if debug else ()
    os.makedirs(bdir, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))
    hdrs = glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(ROOT, "include", "*.h"))
    hdr_time = max((os.path.getmtime(h) for h in hdrs), default=0.0)
    jobs, objs = [], []
    for s in srcs:
        o = os.path.join(bdir, os.path.basename(s) + ".o")
        objs.append(o)
        if force or not os.path.exists(o) or os.path.getmtime(o) < max(os.path.getmtime(s), hdr_time):
            jobs.append((s, o))
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
            for src, rc, out in ex.map(lambda j: _compile(nvcc, *j, extra), jobs):
                if verbose or rc != 0:
                    sys.stderr.write(out)
                if rc != 0:
                    raise RuntimeError(f"nvcc failed on {os.path.basename(src)}")
    if jobs or not os.path.exists(lib) or force:
        libdir = _cuda_lib_dir(nvcc)
        cmd = [nvcc, *ARCH, "-shared", "-o", lib, *objs, "-L", libdir, "-lcudart", "-ldl",
               "-Xlinker", "-rpath", "-Xlinker", libdir]
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            sys.stderr.write(p.stdout + p.stderr)
            raise RuntimeError(f"linking {os.path.basename(lib)} failed")
    return lib


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv, debug="--debug" in sys.argv))
