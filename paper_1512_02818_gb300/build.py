"""Build libpdd.so in-tree with nvcc for sm_103a (GB300).

The translation units under ``csrc/`` are compiled in parallel to objects in
``_build/`` and linked into ``libpdd.so`` next to this file.  Rebuilds only
when a source or header is newer than the library.

``build(bounds=True)`` builds the bounds-checked variant ``libpdd_bounds.so``
(objects in ``_build_bounds/``, compiled with -DPDD_DEBUG_BOUNDS=1): the same
library whose kernels check their index arithmetic against their buffers and
report a violation as PDD_ERR_BOUNDS instead of touching memory out of range.
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
LIB = os.path.join(HERE, "libpdd.so")
LIB_BOUNDS = os.path.join(HERE, "libpdd_bounds.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_path() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _inputs() -> list[str]:
    return (sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
            + glob.glob(os.path.join(ROOT, "include", "*.h")) + [os.path.abspath(__file__)])


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib) or os.environ.get("PDD_NVCC_FLAGS"):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _inputs())


def compile_flags(verbose_ptxas: bool = False) -> list[str]:
    # -ftz=true: FP32 denormals flush to zero, so the SFU intrinsics need no
    # denormal fix-up code (no quantity of the method comes near 1e-38).
    f = ["-O3", "-std=c++17", *ARCH, "-lineinfo", "-ftz=true", "-Xcompiler", "-fPIC",
         "-Xcompiler", "-O2", "-I", os.path.join(ROOT, "include")]
    # extra flags for build experiments, e.g. PDD_NVCC_FLAGS="-DPDD_MIN_BLOCKS=6"
    f += os.environ.get("PDD_NVCC_FLAGS", "").split()
    if verbose_ptxas:
        f += ["-Xptxas", "-v"]
    return f


def build(force: bool = False, verbose_ptxas: bool = False, jobs: int | None = None,
          bounds: bool = False) -> str:
    lib = LIB_BOUNDS if bounds else LIB
    bdir = BUILD + "_bounds" if bounds else BUILD
    if not force and up_to_date(lib):
        return lib
    os.makedirs(bdir, exist_ok=True)
    nvcc = nvcc_path()
    flags = compile_flags(verbose_ptxas) + (["-DPDD_DEBUG_BOUNDS=1"] if bounds else [])
    srcs = sources()

    def one(src: str) -> str:
        obj = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc, *flags, "-c", src, "-o", obj]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{res.stdout}\n{res.stderr}")
        if verbose_ptxas and res.stderr:
            sys.stderr.write(res.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=jobs or min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(one, srcs))
    tmp = lib + f".tmp{os.getpid()}"
    res = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv,
                bounds="--bounds" in sys.argv))
