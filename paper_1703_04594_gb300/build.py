"""Build the sm_103a shared library ``_native/liblbm_d2q37.so`` from ``csrc/*.cu``.

Each translation unit is compiled by nvcc in parallel, then linked with
``nvcc -shared``.  Only one architecture is built: ``-gencode
arch=compute_103a,code=sm_103a`` (GB300).  Usage: ``python -m paper_1703_04594_gb300.build``.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_native")
LIB_NAME = "liblbm_d2q37.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-Xptxas", "-v"]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")
    return cand


def _compile(src: str, obj: str) -> str:
    # LBM_NVCC_DEFINES: extra "-DNAME=VALUE" flags (launch-bound and unroll tuning knobs)
    extra = os.environ.get("LBM_NVCC_DEFINES", "").split()
    cmd = [nvcc(), *ARCH, *NVCC_FLAGS, *extra, "-c", src, "-o", obj]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{res.stdout}\n{res.stderr}")
    return res.stderr


def build(verbose: bool = False) -> str:
    """Compile and link the library; returns its path."""
    os.makedirs(OUT_DIR, exist_ok=True)
    obj_dir = os.path.join(OUT_DIR, "obj")
    os.makedirs(obj_dir, exist_ok=True)
    sources = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    objs = [os.path.join(obj_dir, os.path.basename(s)[:-3] + ".o") for s in sources]
    with cf.ThreadPoolExecutor(max_workers=min(len(sources), os.cpu_count() or 4)) as ex:
        logs = list(ex.map(_compile, sources, objs))
    with open(os.path.join(OUT_DIR, "ptxas.log"), "w") as fh:
        for s, log in zip(sources, logs):
            fh.write(f"== {os.path.basename(s)}\n{log}\n")
    lib = os.path.join(OUT_DIR, LIB_NAME)
    tmp = lib + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", *objs, "-o", tmp, "-lcudart"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, lib)
    if verbose:
        print(open(os.path.join(OUT_DIR, "ptxas.log")).read())
    return lib


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
