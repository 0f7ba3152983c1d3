"""Build libstag.so (the CUDA kernels and the C ABI) in-tree with nvcc.

Every translation unit under ``csrc/`` is compiled for sm_103a in parallel,
then linked into ``_build/libstag.so``.  A unit is recompiled when it, or any
header it can include, is newer than its object file.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libstag.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "--expt-relaxed-constexpr", "-Xptxas", "-warn-spills"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libstag")


def nccl_paths():
    """(include dir, library file) of an NCCL the build can use, or None.
    The NCCL of the nvidia-nccl wheel (the one torch loads) comes first."""
    cands = []
    try:
        import nvidia.nccl as nn  # noqa: F401
        base = os.path.dirname(nn.__file__) if getattr(nn, "__file__", None) else list(nn.__path__)[0]
        cands.append((os.path.join(base, "include"), os.path.join(base, "lib")))
    except Exception:
        pass
    cands += [("/usr/include", d) for d in sorted(glob.glob("/usr/lib/*-linux-gnu")) + ["/usr/lib64", "/usr/lib"]]
    for inc, libdir in cands:
        lib = os.path.join(libdir, "libnccl.so.2")
        if os.path.exists(os.path.join(inc, "nccl.h")) and os.path.exists(lib):
            return inc, lib
    return None


def _headers():
    return (glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
            + glob.glob(os.path.join(ROOT, "include", "*.h")))


def _stale(obj: str, src: str, newest_header: float) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return t < os.path.getmtime(src) or t < newest_header


def build(verbose: bool = False, force: bool = False, jobs: int | None = None) -> str:
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    sources = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    newest = max((os.path.getmtime(h) for h in _headers()), default=0.0)
    objs = []
    todo = []
    for src in sources:
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        if force or _stale(obj, src, newest):
            todo.append((src, obj))

    nccl = nccl_paths()
    nccl_flags = ["-DSTAG_HAVE_NCCL", "-I", nccl[0]] if nccl else []
    # the NCCL choice is part of the communicator's object: rebuild it when it changes
    stamp = os.path.join(BUILD, "nccl.txt")
    want = repr(nccl)
    old = open(stamp).read() if os.path.exists(stamp) else None
    if old != want:
        todo = [t for t in todo if not t[0].endswith("comm_nccl.cu")]
        todo.append((os.path.join(CSRC, "comm_nccl.cu"), os.path.join(BUILD, "comm_nccl.o")))
        with open(stamp, "w") as f:
            f.write(want)

    def compile_one(item):
        src, obj = item
        tmp = obj + f".tmp{os.getpid()}"
        extra = nccl_flags if src.endswith("comm_nccl.cu") else []
        cmd = [cc, *NVCC_FLAGS, *extra, "-I", os.path.join(ROOT, "include"), "-c", src, "-o", tmp]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
        os.replace(tmp, obj)
        return r.stderr

    if todo:
        with cf.ThreadPoolExecutor(max_workers=jobs or min(len(todo), os.cpu_count() or 4)) as ex:
            for log in ex.map(compile_one, todo):
                if verbose and log.strip():
                    print(log, file=sys.stderr)
    stale = not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs)
    if todo or stale:
        tmp = LIB + f".tmp{os.getpid()}"
        link = ["-Xlinker", nccl[1], f"-Xlinker=-rpath={os.path.dirname(nccl[1])}"] if nccl else []
        cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, *link]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link of libstag.so failed:\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv))
