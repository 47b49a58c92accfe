"""Build libme.so (the CUDA kernels and the C-ABI) in-tree for sm_103a.

Each translation unit is compiled by nvcc in parallel, then linked into
``paper_0806_0689_gb300/_build/libme.so``.  No cmake, no setuptools.
"""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libme.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-I", INCLUDE, "-I", CSRC]


def nvcc():
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libme")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _deps():
    return sources() + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cuh")] + [
        os.path.join(INCLUDE, "me.h")]


# Library variants: the default build, and "check", whose DCDS tile kernel
# bounds-checks every shared-memory access and records a violation in the
# status word instead of making it (a stand-in for a memory sanitizer).
VARIANTS = {"": [], "check": ["-DME_CHECK"]}


def variant() -> str:
    """The variant this process loads: $ME_LIB_VARIANT, default ""."""
    v = os.environ.get("ME_LIB_VARIANT", "")
    if v not in VARIANTS:
        raise ValueError(f"ME_LIB_VARIANT must be one of {sorted(VARIANTS)}, not {v!r}")
    return v


def paths(v: str = ""):
    """(build directory, library path) of variant v."""
    d = BUILD if not v else os.path.join(HERE, f"_build_{v}")
    return d, os.path.join(d, "libme.so")


def is_stale(v: str = "") -> bool:
    lib = paths(v)[1]
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in _deps())


def build(force: bool = False, verbose: bool = False, extra_flags=(), variant_name=None) -> str:
    v = variant() if variant_name is None else variant_name
    bdir, lib = paths(v)
    if not force and not is_stale(v):
        return lib
    os.makedirs(bdir, exist_ok=True)
    cc = nvcc()
    objs = []
    flags = [*VARIANTS[v], *extra_flags]

    def compile_one(src):
        obj = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
        cmd = [cc, *ARCH, *NVCC_FLAGS, *flags, "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr, file=sys.stderr)
        return obj

    with concurrent.futures.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        objs = list(ex.map(compile_one, sources()))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
