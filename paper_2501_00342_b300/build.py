"""Builds the CUDA library paper_2501_00342_b300/libsgs.so for sm_103a (B300).

Each .cu file is compiled on its own (in parallel) into _build/, then linked with the
static CUDA runtime so that the library loads on a machine without a GPU.
"""
import concurrent.futures
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libsgs.so")
SOURCES = ["api.cu", "preprocess.cu", "binning.cu", "sort.cu", "blend.cu", "sort_noalloc.cu", "optim.cu", "probe.cu"]
HEADERS = [os.path.join(CSRC, h) for h in ("common.cuh", "colour.cuh", "kernels.h")] + \
          [os.path.join(INCLUDE, "sgs.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")


def _flags():
    # host code computes per-view single-precision constants the kernels must reproduce:
    # no contraction of a multiply and an add into one rounding there
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
                   "-I", INCLUDE, "-I", CSRC, "--expt-relaxed-constexpr"]


def _obj(src):
    return os.path.join(BUILD, src.replace(".cu", ".o"))


def _stale(src) -> bool:
    o = _obj(src)
    if not os.path.exists(o):
        return True
    t = os.path.getmtime(o)
    deps = [os.path.join(CSRC, src)] + HEADERS
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src, verbose_ptxas=False):
    cmd = [NVCC] + _flags() + ["-c", os.path.join(CSRC, src), "-o", _obj(src)]
    if verbose_ptxas:
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return r.stderr


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    todo = [s for s in SOURCES if force or verbose_ptxas or _stale(s)]
    if todo:
        with concurrent.futures.ThreadPoolExecutor(max_workers=len(todo)) as ex:
            logs = list(ex.map(lambda s: _compile(s, verbose_ptxas), todo))
        if verbose_ptxas:
            for s, log in zip(todo, logs):
                print(f"==== {s}\n{log}")
    if todo or not os.path.exists(LIB):
        cmd = [NVCC] + ARCH + ["-shared", "-cudart", "static", "-o", LIB + ".tmp"] + [_obj(s) for s in SOURCES]
        subprocess.run(cmd, check=True)
        os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="--ptxas" in sys.argv))
