"""In-tree build of libsbse.so for sm_103a (GB300): one nvcc per translation unit, in parallel, then
one shared-library link. No cmake. Run `python -m paper_2205_06690_gb300.build` or call build()."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OBJ = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libsbse.so")
# the debug build: every translation unit with SBSE_DEBUG_BOUNDS (device-side index checks that
# record instead of faulting, read by sbse_debug_bounds), linked as libsbse_dbg.so
OBJ_DBG = os.path.join(PKG, "_build_dbg")
LIB_DBG = os.path.join(PKG, "libsbse_dbg.so")
SOURCES = ["sbse_api.cu", "tdh_kernels.cu", "fft_fast.cu", "fft_split.cu", "contract.cu", "eig.cu", "noalloc.cu", "umma_gemm.cu", "fno.cu", "spectrum.cu", "finite_box.cu", "localized.cu", "mixed.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsbse.so")
    return exe


def _compile(src: str, extra: list[str], obj_dir: str = OBJ) -> str:
    obj = os.path.join(obj_dir, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if r.stderr.strip():
        sys.stderr.write(r.stderr)
    return obj


def build(verbose_ptxas: bool = False, debug_bounds: bool = False) -> str:
    """Compile every CUDA source for sm_103a and link libsbse.so (libsbse_dbg.so with the debug
    bounds checks) next to this file."""
    obj_dir, lib = (OBJ_DBG, LIB_DBG) if debug_bounds else (OBJ, LIB)
    os.makedirs(obj_dir, exist_ok=True)
    extra = ["-Xptxas", "-v"] if verbose_ptxas else []

    def one(k_src):
        k, src = k_src
        dbg = ["-DSBSE_DEBUG_BOUNDS", f"-DSBSE_TU={k + 1}"] if debug_bounds else []
        return _compile(src, extra + dbg, obj_dir)

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(one, enumerate(SOURCES)))
    cmd = [nvcc(), *ARCH, "-shared", "-o", lib, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link of {os.path.basename(lib)} failed:\n{r.stdout}\n{r.stderr}")
    return lib


if __name__ == "__main__":
    print(build(verbose_ptxas="-v" in sys.argv, debug_bounds="--debug-bounds" in sys.argv))
