"""Builds libcg.so (the CUDA library) in-tree for sm_103a with nvcc.

Each translation unit is compiled in parallel with
``-gencode arch=compute_103a,code=sm_103a`` and linked into
``paper_1407_5026_gb300/_build/libcg.so``.  Host code is compiled with
``-ffp-contract=off`` so the binary64 set-up arithmetic is never fused.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libcg.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

SOURCES = ["cg_lib.cu", "cg_pr_kernel.cu", "cg_pr_kernel3d.cu", "cg_pr_kernel_pair.cu",
           "cg_pr_kernel_pair_time.cu", "cg_pr_cluster_pair.cu", "cg_pr_kernel3d_pair.cu",
           "cg_pr_random.cu", "cg_pr_random_cluster.cu",
           "cg_aux_kernels.cu",
           "cg_microbench.cu", "cg_refresh_tc.cu", "cg_refresh_static.cu", "cg_pr_cluster.cu",
           "cg_refresh_fft.cu"]
HEADERS = ["cg_internal.h", "cg_device.cuh", "cg_pr_common.cuh", "cg_pr_persistent.cuh",
           "cg_pr_cluster.cuh", "cg_pr_random.cuh"]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
              "--expt-relaxed-constexpr"]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found")
    return cand


def _digest() -> str:
    h = hashlib.sha256()
    for name in SOURCES + HEADERS:
        with open(os.path.join(CSRC, name), "rb") as f:
            h.update(f.read())
    with open(os.path.join(INCLUDE, "cg.h"), "rb") as f:
        h.update(f.read())
    h.update(" ".join(ARCH + NVCC_FLAGS).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile and link libcg.so if the sources changed; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    stamp = os.path.join(BUILD, "libcg.stamp")
    dig = _digest()
    if (not force and os.path.exists(LIB) and os.path.exists(stamp)
            and open(stamp).read().strip() == dig):
        return LIB
    cc = nvcc()
    extra = ["-Xptxas", "-v"] if ptxas_info else []

    def compile_one(src):
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *NVCC_FLAGS, *extra, "-I", INCLUDE, "-c",
               os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose or ptxas_info:
        for _, log in results:
            sys.stderr.write(log)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *[o for o, _ in results], "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(dig + "\n")
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True,
                ptxas_info="--ptxas" in sys.argv))
