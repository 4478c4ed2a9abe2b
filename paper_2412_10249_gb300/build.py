"""Builds libimask.so in-tree (paper_2412_10249_gb300/_build/) with nvcc for sm_103a."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libimask.so")
SOURCES = ["kernels.cu", "api.cu"]
HEADERS = ["imask_internal.h", os.path.join("..", "..", "include", "imask.h")]

NVCC_FLAGS = [
    "-gencode", "arch=compute_103a,code=sm_103a",
    "-lineinfo", "-O3", "-std=c++17",
    "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


# index-checked variant of the same library (kernels check their computed
# indices and record failures instead of accessing out of bounds)
CHECKED_OUT = os.path.join(OUT, "checked")
CHECKED_LIB = os.path.join(CHECKED_OUT, "libimask.so")


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, s) for s in SOURCES] + [os.path.join(CSRC, h) for h in HEADERS]
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(out_dir: str, lib: str, extra: list, verbose: bool):
    """Starts the compiles of one variant; returns (processes, link step)."""
    os.makedirs(out_dir, exist_ok=True)
    procs, objs = [], []
    for s in SOURCES:
        obj = os.path.join(out_dir, s.replace(".cu", ".o"))
        objs.append(obj)
        cmd = [nvcc(), *NVCC_FLAGS, *extra, "-c", os.path.join(CSRC, s), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))

    def link():
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-o", tmp, *objs]
        r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
        if r.returncode != 0:
            sys.stderr.write(r.stdout.decode(errors="replace"))
            raise RuntimeError("nvcc link failed")
        os.replace(tmp, lib)

    return procs, link


def _finish(procs, link, verbose: bool):
    for cmd, pr in procs:
        out, _ = pr.communicate()
        if verbose or pr.returncode != 0:
            sys.stderr.write(out.decode(errors="replace"))
        if pr.returncode != 0:
            raise RuntimeError(f"nvcc failed: {' '.join(cmd)}")
    link()


def build(force: bool = False, verbose: bool = False, extra: list | None = None,
          checked: bool = True) -> str:
    """Compile the CUDA sources in parallel and link the shared library (and,
    with `checked`, its index-checked variant, in parallel with it)."""
    jobs = []
    if force or _stale(LIB):
        jobs.append(_compile(OUT, LIB, list(extra or []), verbose))
    if checked and (force or _stale(CHECKED_LIB)):
        jobs.append(_compile(CHECKED_OUT, CHECKED_LIB, ["-DIMASK_BOUNDS_CHECK", *(extra or [])],
                             verbose))
    for procs, link in jobs:
        _finish(procs, link, verbose)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None))
