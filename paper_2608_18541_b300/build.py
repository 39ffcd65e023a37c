"""Compile the CUDA library (libtts.so) for sm_103a, in-tree.

nvcc -gencode arch=compute_103a,code=sm_103a -O3 -lineinfo, shared, with the
CUDA runtime linked statically so the library depends only on the driver.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIB = os.path.join(HERE, "libtts.so")
OBJDIR = os.path.join(HERE, "_build")

SOURCES = ["tts_build.cpp", "tts_kernels.cu", "tts_engines.cu", "tts_runtime.cu", "tts_noalloc.cu", "tts_lattice.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "tts.h"))
    files.append(os.path.abspath(__file__))
    return files


def build(force: bool = False, verbose: bool = False) -> str:
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(f) for f in _deps())):
        return LIB
    os.makedirs(OBJDIR, exist_ok=True)
    objs = []
    for src in SOURCES:
        obj = os.path.join(OBJDIR, src + ".o")
        cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
               "-Xcompiler", "-fvisibility=hidden", "-I", INCLUDE,
               "-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cu"):
            cmd[5:5] = ["--expt-relaxed-constexpr"]
        if verbose:
            cmd.append("-Xptxas=-v")
            print(" ".join(cmd))
        subprocess.check_call(cmd)
        objs.append(obj)
    tmp = LIB + ".tmp.%d" % os.getpid()
    subprocess.check_call([NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
