"""Build libtflbm (the CUDA kernels and the C ABI of include/tflbm.h) in-tree.

nvcc compiles each translation unit for sm_103a only, in parallel, and links
them into ``paper_1810_07642_gb300/_build/libtflbm_<machine>.so``.  Nothing is
installed outside the repository.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import platform
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, f"libtflbm_{platform.machine()}.so")
# the bounds-checked debug build (TFLBM_CHECK_BOUNDS): every index of the step
# kernels is checked; a bad one sets TF_LBM_STATUS_BOUNDS instead of trapping
LIB_CHECKED = os.path.join(BUILD, f"libtflbm_checked_{platform.machine()}.so")
SOURCES = ["tflbm_api.cu", "tflbm_aux.cu", "step_f32.cu", "step_f16.cu", "step2_f32.cu", "step2_f16.cu",
           "step2_bf16.cu", "tflbm_adjoint.cu", "tflbm_noalloc.cu", "tflbm_batch.cu"]
HEADERS = ["tflbm_internal.h", "tflbm_step.cuh", "tflbm_step2.cuh", "tflbm_adjoint_march.cuh", "tflbm_handle.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
         f"-I{os.path.join(ROOT, 'include')}"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libtflbm")


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, s) for s in SOURCES + HEADERS]
    deps.append(os.path.join(ROOT, "include", "tflbm.h"))
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Compile the library (or, with checked=True, its bounds-checked debug
    variant) if a source is newer than it; return its path."""
    lib = LIB_CHECKED if checked else LIB
    if not force and not _stale(lib):
        return lib
    os.makedirs(BUILD, exist_ok=True)
    nv = nvcc()
    objs = []
    tag = "_checked" if checked else ""
    extra = ["-DTFLBM_CHECK_BOUNDS"] if checked else []

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.splitext(src)[0] + f"{tag}_{platform.machine()}.o")
        cmd = [nv, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + f".tmp{os.getpid()}"
    r = subprocess.run([nv, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, checked="--checked" in sys.argv))
