"""Compile the CUDA sources of libsph.so for sm_103a (GB300), in tree."""
from __future__ import annotations

import concurrent.futures
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_DIR = os.path.join(HERE, "_lib")
LIB_PATH = os.path.join(LIB_DIR, "libsph.so")
SOURCES = ["sph_cells.cu", "sph_physics.cu", "sph_relax_pr.cu", "sph_relax_dr.cu", "sph_gather.cu", "sph_diag.cu", "sph_noalloc.cu", "sph_learned.cu", "sph_diffusion.cu", "sph_gradient.cu", "sph_persistent.cu", "sph_halfpair.cu", "sph_fsi.cu", "sph_api.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


def _flags():
    return ARCH + ["-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
                   "-I", CSRC, "-I", INCLUDE]


def _run(cmd):
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"command failed: {' '.join(cmd)}\n{res.stdout}\n{res.stderr}")
    return res.stdout + res.stderr


def build(verbose: bool = False, extra_flags=()) -> str:
    """Compile every translation unit in parallel and link libsph.so; returns its path."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    os.makedirs(LIB_DIR, exist_ok=True)
    objs = []
    cmds = []
    for src in SOURCES:
        obj = os.path.join(BUILD_DIR, src.replace(".cu", ".o"))
        objs.append(obj)
        cmds.append([NVCC, *(_flags()), *extra_flags, "-c", os.path.join(CSRC, src), "-o", obj])
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(cmds)) as ex:
        logs = list(ex.map(_run, cmds))
    tmp = LIB_PATH + ".tmp"
    logs.append(_run([NVCC, *ARCH, "-shared", "-o", tmp, *objs]))
    os.replace(tmp, LIB_PATH)
    if verbose:
        print("\n".join(l for l in logs if l.strip()))
    return LIB_PATH


if __name__ == "__main__":
    print(build(verbose=True))
