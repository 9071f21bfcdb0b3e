"""In-tree build of libtc.so for sm_103a (GB300) with nvcc.

Each CUDA translation unit is compiled in parallel, then linked into
paper_0711_1429_gb300/libtc.so (CUDA runtime linked statically, so the library
loads on a machine without a GPU driver; compute calls need a GB300).
"""
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libtc.so")
SOURCES = ["tc_fft_f64.cu", "tc_fft_df.cu", "tc_fft_f32.cu", "tc_line.cu", "tc_api.cu", "tc_fft.cu",
           "tc_peak.cu", "tc_noalloc.cu", "tc_serve.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
         "-Xptxas", "-O3"]


def _nvcc():
    nv = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nv):
        raise RuntimeError("nvcc not found")
    return nv


def build(verbose=False, extra_flags=()):
    os.makedirs(BUILD, exist_ok=True)
    nv = _nvcc()
    inc = ["-I", os.path.join(HERE, "..", "include"), "-I", CSRC]

    def compile_one(src):
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [nv, "-c", os.path.join(CSRC, src), "-o", obj] + ARCH + FLAGS + list(extra_flags) + inc
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{p.stdout}\n{p.stderr}")
        if verbose and (p.stdout or p.stderr):
            print(p.stdout, p.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + ".tmp"
    cmd = [nv, "-shared", "-o", tmp] + objs + ARCH + ["-Xcompiler", "-fPIC"]
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError(f"link failed:\n{p.stdout}\n{p.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
