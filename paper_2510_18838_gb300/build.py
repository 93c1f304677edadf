"""Build libpcms.so (the C-ABI CUDA library) in-tree for sm_103a.

Each .cu translation unit under csrc/ is compiled in parallel with
``nvcc -gencode arch=compute_103a,code=sm_103a -O3 -lineinfo`` and linked into
``paper_2510_18838_gb300/_lib/libpcms.so`` against the shared CUDA runtime, so that the
library shares the runtime (streams, memory pool) of the PyTorch process that loads it.
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
INCLUDE = os.path.join(ROOT, "include")
OBJ = os.path.join(PKG, "_build")
LIBDIR = os.path.join(PKG, "_lib")
LIB = os.path.join(LIBDIR, "libpcms.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return (_sources() + glob.glob(os.path.join(CSRC, "*.cuh")) +
            [os.path.join(INCLUDE, "pcms.h"), os.path.abspath(__file__)])


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src: str, verbose_ptxas: bool) -> tuple[str, str]:
    obj = os.path.join(OBJ, os.path.basename(src)[:-3] + ".o")
    deps = [src] + glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(INCLUDE, "pcms.h"),
                                                           os.path.abspath(__file__)]
    if not _stale(obj, deps):
        return obj, ""
    cmd = [nvcc(), *ARCH, *NVCC_FLAGS, "-c", src, "-o", obj + ".tmp"]
    if verbose_ptxas:
        cmd += ["-Xptxas", "-v"]
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{p.stdout}\n{p.stderr}")
    os.replace(obj + ".tmp", obj)
    return obj, p.stderr


def build(force: bool = False, jobs: int | None = None, verbose_ptxas: bool = False,
          quiet: bool = True) -> str:
    """Compile every csrc/*.cu for sm_103a and link _lib/libpcms.so. Returns its path."""
    os.makedirs(OBJ, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    if force:
        for o in glob.glob(os.path.join(OBJ, "*.o")):
            os.remove(o)
    if not force and not verbose_ptxas and not _stale(LIB, _deps()):
        return LIB
    srcs = _sources()
    jobs = jobs or min(len(srcs), os.cpu_count() or 4)
    logs = []
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        futs = {ex.submit(_compile, s, verbose_ptxas): s for s in srcs}
        objs = []
        for f in cf.as_completed(futs):
            o, log = f.result()
            objs.append(o)
            if log:
                logs.append((futs[f], log))
    cmd = [nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", LIB + ".tmp", *sorted(objs),
           "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
    subprocess.run(cmd, check=True, capture_output=quiet)
    os.replace(LIB + ".tmp", LIB)
    if verbose_ptxas:
        for s, log in logs:
            print(f"== {os.path.basename(s)}\n{log}", file=sys.stderr)
    return LIB


if __name__ == "__main__":
    t = build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv)
    print(t)
