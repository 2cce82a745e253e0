"""Build the in-tree shared library ``lib/libhdg_gb300.so`` for sm_103a.

Every translation unit is compiled by nvcc in parallel, then linked with
``nvcc -shared``.  No CMake, no torch extension machinery: the library has a
plain C ABI (``include/hdg.h``) and is loaded with ctypes.
"""
import concurrent.futures
import hashlib
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "lib")
BUILD_DIR = os.path.join(ROOT, "_build")
LIB_PATH = os.path.join(OUT_DIR, "libhdg_gb300.so")

SOURCES = ["setup1d.cpp", "kernels.cu", "tpt_f64.cu", "tpt_f32.cu", "tpt_bf16.cu", "tpt_tile_f32.cu", "tpt_tile_f64.cu", "tpt_tile_bf16.cu", "tp_nodal.cu", "lowdim.cu", "hdg_api.cu", "hdg_static.cu", "probe.cu", "tpt_generic.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _digest(src):
    h = hashlib.sha256()
    h.update(" ".join(ARCH + FLAGS).encode())
    for name in sorted(os.listdir(CSRC)):
        if name.endswith((".h", ".cuh")) or name == src:
            with open(os.path.join(CSRC, name), "rb") as f:
                h.update(name.encode())
                h.update(f.read())
    with open(os.path.join(ROOT, "include", "hdg.h"), "rb") as f:
        h.update(f.read())
    return h.hexdigest()[:16]


def _compile(src):
    obj = os.path.join(BUILD_DIR, src + "." + _digest(src) + ".o")
    if os.path.exists(obj):
        return obj
    cmd = [_nvcc()] + ARCH + FLAGS + ["-c", os.path.join(CSRC, src), "-o", obj + ".tmp"]
    subprocess.run(cmd, check=True)
    os.replace(obj + ".tmp", obj)
    return obj


def build(jobs=None, verbose=True):
    """Compile and link; returns the path of the shared library."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    os.makedirs(OUT_DIR, exist_ok=True)
    jobs = jobs or min(len(SOURCES), os.cpu_count() or 4)
    with concurrent.futures.ThreadPoolExecutor(jobs) as ex:
        objs = list(ex.map(_compile, SOURCES))
    stamp = hashlib.sha256("".join(objs).encode()).hexdigest()[:16]
    stamp_file = LIB_PATH + ".stamp"
    if os.path.exists(LIB_PATH) and os.path.exists(stamp_file) and open(stamp_file).read() == stamp:
        return LIB_PATH
    cmd = [_nvcc()] + ARCH + ["-shared", "-o", LIB_PATH + ".tmp"] + objs
    subprocess.run(cmd, check=True)
    os.replace(LIB_PATH + ".tmp", LIB_PATH)
    with open(stamp_file, "w") as f:
        f.write(stamp)
    if verbose:
        print("built", LIB_PATH, file=sys.stderr)
    return LIB_PATH


if __name__ == "__main__":
    build()
