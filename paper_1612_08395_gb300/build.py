"""Build the CUDA library libbem_gb300.so (sm_103a) in-tree.

Each translation unit under csrc/ is compiled by nvcc in parallel, then the
objects are linked into paper_1612_08395_gb300/_build/libbem_gb300.so.  Only
the sm_103a target is generated.  Rebuilds when a source or header is newer
than the library.

With debug_checks (or BEM_DEBUG_CHECKS=1 in the environment) the sources are
compiled with -DBEM_DEBUG_CHECKS into _build_debug/libbem_gb300.so instead:
the kernels then bounds-check their index arithmetic on the transposed
spectrum workspace and report a failed check as a solver error instead of
touching memory out of range.  The binding loads that library when
BEM_DEBUG_CHECKS=1 is set.
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
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(OUT_DIR, "libbem_gb300.so")
DEBUG_OUT_DIR = os.path.join(PKG, "_build_debug")
DEBUG_LIB = os.path.join(DEBUG_OUT_DIR, "libbem_gb300.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "-I", CSRC, "-I", INCLUDE, "-diag-suppress", "128"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) \
        + glob.glob(os.path.join(INCLUDE, "*.h"))


def debug_requested() -> bool:
    return os.environ.get("BEM_DEBUG_CHECKS", "0") == "1"


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, debug_checks: bool | None = None) -> str:
    if debug_checks is None:
        debug_checks = debug_requested()
    out_dir, lib = (DEBUG_OUT_DIR, DEBUG_LIB) if debug_checks else (OUT_DIR, LIB)
    if not force and up_to_date(lib):
        return lib
    os.makedirs(out_dir, exist_ok=True)
    cc = nvcc()
    extra = ["-DBEM_DEBUG_CHECKS"] if debug_checks else []

    def compile_one(src):
        obj = os.path.join(out_dir, os.path.basename(src)[:-3] + ".o")
        cmd = [cc, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        results = list(ex.map(compile_one, _sources()))
    objs = [o for o, _ in results]
    if verbose:
        for _, err in results:
            sys.stderr.write(err)
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                debug_checks=True if "--debug-checks" in sys.argv else None))
