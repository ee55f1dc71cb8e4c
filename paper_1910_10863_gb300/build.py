"""Build libpfmbem.so in-tree for sm_103a (nvcc for the kernels, g++ for the host side)."""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libpfmbem.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _cuda_home():
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return c
    nv = shutil.which("nvcc")
    if nv:
        return os.path.dirname(os.path.dirname(nv))
    raise RuntimeError("nvcc not found")


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed: " + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def build(verbose: bool = False, ptxas_info: bool = False) -> str:
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    os.makedirs(BUILD, exist_ok=True)
    inc = ["-I" + CSRC, "-I" + INCLUDE, "-I" + os.path.join(cuda, "include")]
    k_obj = os.path.join(BUILD, "kernels.o")
    t_obj = os.path.join(BUILD, "m2l_tc.o")
    m_obj = os.path.join(BUILD, "mlp.o")
    f_obj = os.path.join(BUILD, "matvec_fused.o")
    h_obj = os.path.join(BUILD, "host.o")
    nv_flags = [nvcc, ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--use_fast_math=false"]
    nv_flags = [f for f in nv_flags if f != "--use_fast_math=false"]
    if ptxas_info:
        nv_flags.append("-Xptxas=-v")
    jobs = [
        nv_flags + inc + ["-c", os.path.join(CSRC, "kernels.cu"), "-o", k_obj],
        nv_flags + inc + ["-c", os.path.join(CSRC, "m2l_tc.cu"), "-o", t_obj],
        nv_flags + inc + ["-c", os.path.join(CSRC, "mlp.cu"), "-o", m_obj],
        nv_flags + inc + ["-c", os.path.join(CSRC, "matvec_fused.cu"), "-o", f_obj],
        ["g++", "-O2", "-fPIC", "-std=c++17", "-Wall", "-Wno-unused-function"] + inc
        + ["-c", os.path.join(CSRC, "host.cpp"), "-o", h_obj],
    ]
    with ThreadPoolExecutor(len(jobs)) as ex:
        logs = list(ex.map(_run, jobs))
    logs.append(_run([nvcc, ARCH, "-shared", "-Xcompiler", "-fPIC", k_obj, t_obj, m_obj, f_obj, h_obj, "-o", LIB]))
    if verbose:
        print("\n".join(l for l in logs if l.strip()))
    return "\n".join(logs)


if __name__ == "__main__":
    print(build(verbose=True, ptxas_info="-v" in sys.argv))
