"""Build step of the CUDA library: compiles csrc/*.cu for sm_103a with nvcc (one
object per translation unit, in parallel) and links librpr.so in _build/.

    python -m paper_1803_00430_gb300.build [--force] [--verbose] [--checked]

--checked builds the bounds-checked variant (RP_CHECKED) in _build/checked/.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "librpr.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I", os.path.join(ROOT, "include")]


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return (_sources() + glob.glob(os.path.join(CSRC, "*.cuh"))
            + [os.path.join(ROOT, "include", "rpr.h"), __file__])


def lib_path(checked: bool = False) -> str:
    """The library, or its bounds-checked build (RP_CHECKED) in _build/checked/."""
    return os.path.join(OUT, "checked", "librpr.so") if checked else LIB


def up_to_date(checked: bool = False) -> bool:
    lib = lib_path(checked)
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Compile every translation unit and link the shared library.  checked=True
    builds the bounds-checked variant (-DRP_CHECKED) beside the normal one."""
    lib = lib_path(checked)
    if not force and up_to_date(checked):
        return lib
    out = os.path.dirname(lib)
    os.makedirs(os.path.join(out, "obj"), exist_ok=True)
    nvcc = NVCC if os.path.exists(NVCC) else "nvcc"
    extra = (["-Xptxas", "-v"] if verbose else []) + (["-DRP_CHECKED"] if checked else [])

    def compile_one(src):
        obj = os.path.join(out, "obj", os.path.basename(src) + ".o")
        cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        objs = list(ex.map(compile_one, _sources()))
    tmp = lib + f".{os.getpid()}.tmp"
    r = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stderr)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="--verbose" in sys.argv, checked="--checked" in sys.argv))
