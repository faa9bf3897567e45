"""Builds libqb.so (the C ABI of include/qb.h) for sm_103a with nvcc, in-tree.

The translation units compile in parallel; the result lands in
paper_2111_00050_gb300/_build/libqb.so.  Rebuilds only when a source changed.
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
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libqb.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["qb_host.cpp", "qb_kernels.cu", "qb_adjoint.cu", "qb_stage_m5.cu", "qb_stage_m7.cu", "qb_stage_m9.cu", "qb_stage_m11.cu",
           "qb_stage_any.cu", "qb_diag.cu", "qb_observe.cu"]
HEADERS = ["qb_internal.h", "qb_device.cuh", "qb_stage.cuh", os.path.join("..", "..", "include", "qb.h"),
           os.path.join("..", "..", "include", "qb_diag.h")]


def _nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found")
    return p


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, s) for s in SOURCES + HEADERS] + [os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False, out_dir: str = None,
          defines=()) -> str:
    """Compiles libqb.so into `out_dir` (default: the in-tree _build/).  `defines`
    are extra -D macros (tuning switches of the stage kernel)."""
    global OUT_DIR, LIB
    if out_dir is not None:
        OUT_DIR_, LIB_ = OUT_DIR, LIB
        OUT_DIR, LIB = out_dir, os.path.join(out_dir, "libqb.so")
        try:
            return build(True, verbose, ptxas_info, None, defines)
        finally:
            OUT_DIR, LIB = OUT_DIR_, LIB_
    if not force and not _stale():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    common = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]
    common += [f"-D{d}" for d in defines]

    def compile_one(src: str) -> str:
        obj = os.path.join(OUT_DIR, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc, *ARCH, *common, "-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cu"):
            cmd += ["-Xptxas", "-v"] if ptxas_info else []
        else:
            cmd += ["-x", "c++"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose or ptxas_info:
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    with concurrent.futures.ThreadPoolExecutor(min(len(SOURCES), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
