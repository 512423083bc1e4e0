"""Build libmrfv.so in-tree with nvcc for sm_103a (GB300).

Translation units and their floating-point flags:
  fv_f64.cu, mr_f64.cu, mr_f32.cu : -fmad=false, IEEE division and square root, so
      the double-precision step and every multiresolution operation round exactly
      where the source says (parity with the CPU oracle; bit-exact thresholding);
  fv_f32.cu, fvt.cu : --use_fast_math (single-precision throughput path; fvt.cu is the
      TMA-staged 2D stage kernel with packed FP32x2 arithmetic);
  tree.cu, api.cu : integer work and host sequencing;
  noalloc.cu : -fmad=false (the allocation-free CFL reduction rounds like the
      double-precision one in fv_f64.cu);
  proposer.cu : the learned refinement proposer (tcgen05 inference, FP32 training).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libmrfv.so")
BUILD = os.path.join(HERE, "_build")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
          "-I", CSRC, "-I", INCLUDE]
UNITS = {
    "fv_f32.cu": ["--use_fast_math"],
    "fv_f64.cu": ["-fmad=false"],
    "mr_f32.cu": ["-fmad=false"],
    "mr_f64.cu": ["-fmad=false"],
    "tree.cu": [],
    "api.cu": [],
    "noalloc.cu": ["-fmad=false"],
    "proposer.cu": [],
    "fvt.cu": ["--use_fast_math"],
}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _sources_mtime() -> float:
    m = 0.0
    for d in (CSRC, INCLUDE):
        for f in os.listdir(d):
            m = max(m, os.path.getmtime(os.path.join(d, f)))
    return m


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    """Compile every translation unit in parallel and link libmrfv.so; returns its path."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _sources_mtime():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nv = nvcc()
    extra = list(extra or [])

    def compile_unit(name: str) -> str:
        obj = os.path.join(BUILD, name.replace(".cu", ".o"))
        cmd = [nv, *ARCH, *COMMON, *UNITS[name], *extra, "-c", os.path.join(CSRC, name), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {name}:\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(compile_unit, UNITS))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nv, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None))
