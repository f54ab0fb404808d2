"""Builds libnncandelinc.so in-tree from csrc/*.cu for sm_103a with nvcc.

Each translation unit is compiled in parallel; the objects are linked into
paper_1909_07570_gb300/_lib/libnncandelinc.so. A unit is rebuilt when its
source or any header under csrc/ or include/ is newer than its object.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
OBJDIR = os.path.join(LIBDIR, "obj")
LIBNAME = "libnncandelinc.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "-I" + os.path.join(ROOT, "include")]


def nvcc_path() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libnncandelinc.so")


def lib_path() -> str:
    return os.path.join(LIBDIR, LIBNAME)


def _newest_header() -> float:
    hdrs = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(ROOT, "include", "*.h"))
    return max((os.path.getmtime(h) for h in hdrs), default=0.0)


def _compile(nvcc: str, src: str, extra: list) -> str:
    obj = os.path.join(OBJDIR, os.path.basename(src)[:-3] + ".o")
    stamp = max(os.path.getmtime(src), _newest_header())
    if os.path.exists(obj) and os.path.getmtime(obj) >= stamp and not extra:
        return obj
    cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{res.stdout}\n{res.stderr}")
    if extra and res.stderr:
        sys.stderr.write(res.stderr)
    return obj


def build(verbose: bool = False, extra_flags: list | None = None) -> str:
    """Compile every csrc/*.cu and link the shared library; returns its path."""
    nvcc = nvcc_path()
    os.makedirs(OBJDIR, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    extra = list(extra_flags or [])
    with ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda s: _compile(nvcc, s, extra), srcs))
    out = lib_path()
    if (not os.path.exists(out) or extra
            or any(os.path.getmtime(o) > os.path.getmtime(out) for o in objs)):
        tmp = out + ".tmp"
        cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
        os.replace(tmp, out)
    if verbose:
        print(out)
    return out


if __name__ == "__main__":
    flags = sys.argv[1:]
    build(verbose=True, extra_flags=flags)
