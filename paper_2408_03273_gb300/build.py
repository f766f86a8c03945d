"""Build the sm_103a shared library ``_build/libqmmm_gb300.so`` in-tree.

Each translation unit under ``csrc/`` is compiled by nvcc in parallel for
``-gencode arch=compute_103a,code=sm_103a`` (the sweep sources once per angular class) and the
objects are linked into one shared library with a plain C ABI (include/qmmm.h).  A rebuild happens only when a source or header is newer
than the library.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import re
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libqmmm_gb300.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--extended-lambda", "-Xcompiler", "-fPIC",
              "-I" + os.path.join(ROOT, "include")]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _nclass() -> int:
    """Number of angular classes (l_A >= l_B), from LMAX in device_common.cuh."""
    with open(os.path.join(CSRC, "device_common.cuh")) as f:
        m = re.search(r"constexpr int LMAX = (\d+);", f.read())
    if not m:
        raise RuntimeError("LMAX not found in device_common.cuh")
    lmax = int(m.group(1))
    return (lmax + 1) * (lmax + 2) // 2


def _units():
    """(source, object, extra flags) per compilation: a source that mentions QMMM_SPLIT_CLASS is
    compiled once per angular class plus once for its dispatcher; the highest classes first,
    since they take longest."""
    units, split = [], []
    for src in _sources():
        base = os.path.join(BUILD, os.path.basename(src)[:-3])
        with open(src) as f:
            is_split = "QMMM_SPLIT_CLASS" in f.read()
        units.append((src, base + ".o", []))
        if is_split:
            split += [(src, f"{base}.c{c}.o", [f"-DQMMM_SPLIT_CLASS={c}"]) for c in range(_nclass())]
    split.sort(key=lambda u: -int(u[1].rsplit(".c", 1)[1][:-2]))
    return split + units


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) +
                  glob.glob(os.path.join(ROOT, "include", "*.h")))


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in _sources() + _headers() + [__file__])


def build(force: bool = False, verbose: bool = False, jobs: int | None = None) -> str:
    """Compile every CUDA translation unit for sm_103a and link the shared library."""
    if not force and not needs_build():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    hdr_t = max(os.path.getmtime(f) for f in _headers() + [__file__])

    def compile_one(unit):
        src, obj, extra = unit
        if (not force and os.path.exists(obj) and os.path.getmtime(obj) > os.path.getmtime(src)
                and os.path.getmtime(obj) > hdr_t):
            return obj
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, *extra, "-c", src, "-o", obj + ".tmp"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr[-4000:]}")
        if verbose and r.stderr:
            print(r.stderr)
        os.replace(obj + ".tmp", obj)
        return obj

    units = _units()
    jobs = jobs or min(len(units), max(2, os.cpu_count() or 2))
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        objs = list(ex.map(compile_one, units))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr[-4000:]}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
