"""Builds librpiv.so in-tree: nvcc for sm_103a, one object per translation unit,
compiled in parallel, then linked against the CUDA runtime."""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(os.path.dirname(HERE), "_build", "rpiv")
LIB = os.path.join(HERE, "librpiv.so")

SOURCES = ["k_pass_fp32.cu", "k_pass_tc.cu", "k_deform.cu", "k_grid.cu", "k_adjoint.cu",
           "k_static_scratch.cu", "k_pre.cu", "pass_plan.cpp", "capi.cpp"]
HEADERS = ["rpiv_internal.h", "pass_impl.cuh", "tc_pass.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", CSRC, "-I", INCLUDE,
           "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _digest() -> str:
    h = hashlib.sha256()
    for f in SOURCES + HEADERS:
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    with open(os.path.join(INCLUDE, "rpiv.h"), "rb") as fh:
        h.update(fh.read())
    h.update(" ".join(ARCH + NVFLAGS).encode())
    return h.hexdigest()[:16]


FMA_SRC = "fma_peak.cu"
FMA_LIB = os.path.join(HERE, "libfmapeak.so")


def build_fma_peak(force: bool = False) -> str:
    """The FP32 FMA-throughput microbenchmark (measurement support for the
    ALU roofline), as its own small library."""
    src = os.path.join(CSRC, FMA_SRC)
    if not force and os.path.exists(FMA_LIB) and os.path.getmtime(FMA_LIB) >= os.path.getmtime(src):
        return FMA_LIB
    tmp = FMA_LIB + f".tmp{os.getpid()}"
    r = subprocess.run([_nvcc(), *ARCH, "-O3", "-Xcompiler", "-fPIC", "-shared", src, "-o", tmp, "-lcudart"],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {FMA_SRC}:\n{r.stderr}")
    os.replace(tmp, FMA_LIB)
    return FMA_LIB


TCR_SRC = "tc_rate.cu"
TCR_LIB = os.path.join(HERE, "libtcrate.so")


def build_tc_rate(force: bool = False) -> str:
    """The tcgen05.mma issue-rate microbenchmark (measurement support), as its
    own small library."""
    src = os.path.join(CSRC, TCR_SRC)
    if not force and os.path.exists(TCR_LIB) and os.path.getmtime(TCR_LIB) >= os.path.getmtime(src):
        return TCR_LIB
    tmp = TCR_LIB + f".tmp{os.getpid()}"
    r = subprocess.run([_nvcc(), *ARCH, "-O3", "-Xcompiler", "-fPIC", "-shared", src, "-o", tmp, "-lcudart"],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {TCR_SRC}:\n{r.stderr}")
    os.replace(tmp, TCR_LIB)
    return TCR_LIB


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile (if sources changed) and return the path of librpiv.so."""
    stamp = os.path.join(BUILD, "stamp")
    dig = _digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read() == dig:
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()

    def compile_one(src: str) -> str:
        obj = os.path.join(BUILD, src + ".o")
        cmd = [nvcc, *ARCH, *NVFLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cpp"):
            cmd[1:1] = ["-x", "cu"]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    workers = min(len(SOURCES), max(2, os.cpu_count() or 2))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    r = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(stamp, "w") as fh:
        fh.write(dig)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
