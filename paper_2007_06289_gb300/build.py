"""Builds ``libfbp.so`` in-tree for sm_103a with nvcc (no cmake, no torch extension).

Each CUDA translation unit is compiled in parallel to an object file under ``_build/``,
then linked into ``libfbp.so`` next to this file (the CUDA runtime is linked statically,
so the library depends on nothing but the driver).  A rebuild happens only when a source
or header is newer than the library.
"""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(HERE, "libfbp.so")
# the same sources with FBP_BOUNDS_CHECK: range checks on every pipeline access, reported
# through the plan's status word (slower; for testing)
CHECKED_BUILD_DIR = os.path.join(HERE, "_build_checked")
CHECKED_LIB_PATH = os.path.join(HERE, "libfbp_checked.so")
SOURCES = ("fbp_api.cu", "iir_ramp.cu", "fht.cu", "direct.cu", "noalloc.cu", "volume.cu", "adjoint.cu", "cnn.cu", "sirt.cu")
ARCH = ("-gencode", "arch=compute_103a,code=sm_103a")
FLAGS = ("-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE,
         "--expt-relaxed-constexpr")


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    return files


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(f) > t for f in _deps())


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False,
          bounds_check: bool = False) -> str:
    """Compile and link libfbp.so (bounds_check: libfbp_checked.so) if needed; returns its
    path."""
    lib = CHECKED_LIB_PATH if bounds_check else LIB_PATH
    if not force and not _stale(lib):
        return lib
    nvcc = _nvcc()
    bdir = CHECKED_BUILD_DIR if bounds_check else BUILD_DIR
    os.makedirs(bdir, exist_ok=True)
    extra = ["-DFBP_BOUNDS_CHECK"] if bounds_check else []

    def compile_one(src):
        obj = os.path.join(bdir, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        if ptxas_info:
            cmd += ["-Xptxas", "-v"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with concurrent.futures.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


def build_all(force: bool = False) -> None:
    """Both libraries, compiled concurrently."""
    with concurrent.futures.ThreadPoolExecutor(max_workers=2) as ex:
        futs = [ex.submit(build, force), ex.submit(build, force, bounds_check=True)]
        for f in futs:
            f.result()


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv,
                bounds_check="--checked" in sys.argv))
