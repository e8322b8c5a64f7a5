"""Build the LOWD CUDA library (liblowd.so) in-tree for sm_103a with nvcc.

Each translation unit under csrc/ is compiled in parallel to an object file, then linked
into ``paper_2307_15969_gb300/_lib/liblowd.so``.  A unit is rebuilt when it or any
header it can include is newer than its object.
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
OBJ = os.path.join(HERE, "_build")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "liblowd.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-Xptxas", "-warn-spills"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _headers():
    return glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(ROOT, "include", "*.h"))


def _stale(src: str, obj: str, newest_header: float) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return os.path.getmtime(src) > t or newest_header > t


def build(verbose: bool = False, force: bool = False, extra_flags=None) -> str:
    nvcc = _nvcc()
    os.makedirs(OBJ, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    hdr_t = max([os.path.getmtime(p) for p in _headers()] + [0.0])
    flags = NVCC_FLAGS + list(extra_flags or [])
    jobs = []
    for s in srcs:
        o = os.path.join(OBJ, os.path.basename(s)[:-3] + ".o")
        if force or _stale(s, o, hdr_t):
            cmd = [nvcc] + ARCH + flags + ["-I", os.path.join(ROOT, "include"), "-c", s, "-o", o]
            jobs.append((s, cmd))

    def run(job):
        s, cmd = job
        p = subprocess.run(cmd, capture_output=True, text=True)
        return s, cmd, p

    failed = []
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            for s, cmd, p in ex.map(run, jobs):
                out = (p.stdout + p.stderr).strip()
                if verbose and out:
                    print(f"[{os.path.basename(s)}]\n{out}", file=sys.stderr)
                if p.returncode != 0:
                    failed.append((s, " ".join(cmd), out))
    if failed:
        msg = "\n\n".join(f"{s}\n{c}\n{o}" for s, c, o in failed)
        raise RuntimeError("nvcc failed:\n" + msg)
    objs = [os.path.join(OBJ, os.path.basename(s)[:-3] + ".o") for s in srcs]
    if force or jobs or not os.path.exists(LIB):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError("link failed:\n" + " ".join(cmd) + "\n" + p.stdout + p.stderr)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv))
