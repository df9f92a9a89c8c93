"""Build liblbm.so (the C-ABI library) in-tree with nvcc for sm_103a.

Translation units compile in parallel; the result lands in
``paper_1902_00530_gb300/_build/liblbm.so``.  Run ``python -m
paper_1902_00530_gb300.build`` or call ``build()``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
ROOT = os.path.dirname(HERE)
LIB = os.path.join(BUILD, "liblbm.so")
UNITS = ["lbm_step_f32.cu", "lbm_step_f16.cu", "lbm_step_bf16.cu", "lbm_step_q7_f32.cu", "lbm_step_q7_f16.cu",
         "lbm_step_q7_bf16.cu", "lbm_aux.cu", "lbm_api.cu", "lbm_noalloc.cu"]
HEADERS = ["lbm_device.cuh", "lbm_step.cuh", "lbm_step_staged.cuh", "lbm_step_persistent.cuh", "lbm_step_q7.cuh",
           "lbm_step_q7_staged.cuh", "lbm_internal.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"] + \
    os.environ.get("LBM_NVCC_EXTRA", "").split()


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblbm.so")


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(unit: str, verbose: bool) -> str:
    src = os.path.join(CSRC, unit)
    obj = os.path.join(BUILD, unit.replace(".cu", ".o"))
    deps = [src] + [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", "lbm.h")]
    if _stale(obj, deps):
        cmd = [nvcc(), *ARCH, *FLAGS, "-I", os.path.join(ROOT, "include"), "-c", src, "-o", obj + ".tmp"]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {unit}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stderr)
        os.replace(obj + ".tmp", obj)
    return obj


def build(force: bool = False, verbose: bool = False, build_dir: str | None = None) -> str:
    global BUILD, LIB
    if build_dir:
        BUILD, LIB = build_dir, os.path.join(build_dir, "liblbm.so")
    os.makedirs(BUILD, exist_ok=True)
    if force:
        for u in UNITS:
            p = os.path.join(BUILD, u.replace(".cu", ".o"))
            if os.path.exists(p):
                os.remove(p)
    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(lambda u: _compile(u, verbose), UNITS))
    if force or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
