"""Build the CUDA library libfx.so in-tree for sm_103a (nvcc, translation units in parallel).

build(bounds_check=True) builds the debug variant libfx_bc.so instead: every kernel index that the
sources mark is checked against its buffer's extent, and an index outside it is reported as
FX_ERR_BOUNDS (with the site) instead of being accessed.  Load it by setting FX_LIBRARY to its path
before importing the binding."""
from __future__ import annotations

import concurrent.futures as cf
import glob
import hashlib
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfx.so")
LIB_BC = os.path.join(HERE, "libfx_bc.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


# The FP32 translation units use the hardware reciprocal and square-root approximations (a few
# ulp) and flush denormals; the FP32 form's accuracy bar is far above that.  FP64 units keep IEEE.
FP32_FLAGS = ["-prec-div=false", "-prec-sqrt=false", "-ftz=true"]


def _compile(src: str, extra: list[str]) -> str:
    fp32 = os.path.basename(src).startswith(("fx_stage_f32", "fx_adjoint_f32"))
    cmd = [_nvcc(), *ARCH, *NVCC_FLAGS, *(FP32_FLAGS if fp32 else []), *extra, "-c", src]
    tag = hashlib.sha1(" ".join(cmd[1:]).encode()).hexdigest()[:10]
    obj = os.path.join(BUILD, f"{os.path.basename(src)}.{tag}.o")
    deps = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + [
        os.path.join(HERE, "..", "include", "fx.h"), src]
    if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(d) for d in deps):
        return obj
    r = subprocess.run(cmd + ["-o", obj], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
    return obj


def build(verbose: bool = False, extra: list[str] | None = None, bounds_check: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    flags = list(extra or []) + (["-DFX_BOUNDS_CHECK"] if bounds_check else [])
    out = LIB_BC if bounds_check else LIB
    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda s: _compile(s, flags), srcs))
    tmp = out + ".tmp"
    cmd = [_nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, out)
    if verbose:
        print("built", out)
    return out


if __name__ == "__main__":
    args = sys.argv[1:]
    bc = "--bounds-check" in args
    build(verbose=True, extra=[a for a in args if a != "--bounds-check"], bounds_check=bc)
