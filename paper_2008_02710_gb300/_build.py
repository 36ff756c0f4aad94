"""Builds the CUDA library in-tree: csrc/rlgl.cu -> librlgl.so (sm_103a)."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = [os.path.join(HERE, "csrc", "rlgl.cu"), os.path.join(HERE, "csrc", "rlgl_noalloc.cu")]
DEPS = SRC + [os.path.join(HERE, "csrc", "rlgl_kernels.cuh"), os.path.join(HERE, "csrc", "rlgl_sweep.cuh"),
               os.path.join(HERE, "csrc", "rlgl_power.cuh"), os.path.join(HERE, "csrc", "rlgl_batch.cuh"),
               os.path.join(ROOT, "include", "rlgl.h")]
LIB = os.path.join(HERE, "librlgl.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
         "-shared", "-Xcompiler", "-fPIC", "-Xptxas", "-v"]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in DEPS)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [NVCC] + FLAGS + ["-I", os.path.join(ROOT, "include"), "-o", tmp] + SRC
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("nvcc failed building librlgl.so")
    if verbose:
        sys.stderr.write(r.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose=True)
