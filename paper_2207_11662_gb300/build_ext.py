"""Compile the CUDA library ``libhomln.so`` in-tree for sm_103a (nvcc, no cmake).

Each translation unit in ``csrc/`` is compiled in parallel into ``_build/``,
then linked into ``paper_2207_11662_gb300/libhomln.so``. A unit is rebuilt only
when it or a header is newer than its object file. Processes that build at the same
time (test workers, spawned pools) take turns on a lock file in ``_build/``: the first
compiles, the others then find everything up to date.
"""
from __future__ import annotations

import fcntl
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libhomln.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
              "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]


def _nvcc() -> str:
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hs.append(os.path.join(ROOT, "include", "homln.h"))
    return hs


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def build(force: bool = False, verbose: bool = False) -> str:
    """Build the library. HOMLN_NVCC_EXTRA (environment) adds nvcc flags, e.g. the kernel's
    compile-time knobs -DHOMLN_GATHER_UNROLL=8 or -DHOMLN_BFS_MIN_BLOCKS=3; a change of
    these flags rebuilds everything."""
    os.makedirs(BUILD, exist_ok=True)
    with open(os.path.join(BUILD, ".lock"), "w") as lock:
        fcntl.flock(lock, fcntl.LOCK_EX)  # released when the file is closed
        return _build_locked(force, verbose)


def _build_locked(force: bool, verbose: bool) -> str:
    nvcc = _nvcc()
    extra = os.environ.get("HOMLN_NVCC_EXTRA", "").split()
    stamp = os.path.join(BUILD, "flags.txt")
    want = " ".join(ARCH + NVCC_FLAGS + extra)
    try:
        with open(stamp) as f:
            force = force or f.read() != want
    except OSError:
        force = True
    newest_header = max(os.path.getmtime(h) for h in _headers())
    jobs = []
    for src in sources():
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        stale = (force or not os.path.exists(obj) or os.path.getmtime(obj) < max(os.path.getmtime(src), newest_header))
        jobs.append((src, obj, stale))

    def compile_one(job):
        src, obj, stale = job
        if not stale:
            return None
        tmp = obj + f".tmp{os.getpid()}"
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, *extra, "-c", src, "-o", tmp]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            return f"{' '.join(cmd)}\n{r.stdout}\n{r.stderr}"
        os.replace(tmp, obj)
        if verbose:
            print(r.stderr)
        return None

    with ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
        errs = [e for e in ex.map(compile_one, jobs) if e]
    if errs:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errs))
    objs = [o for _, o, _ in jobs]
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(want)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
