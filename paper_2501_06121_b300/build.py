"""Build the CUDA library libkann.so in-tree for sm_103a.

nvcc compiles the device code for compute_103a/sm_103a only; the host
graph builder is plain C++ linked into the same shared object.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libkann.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

CU_SOURCES = ["kann_api.cu", "kann_search.cu", "kann_search_f32.cu", "kann_search_f16.cu", "kann_search_bf16.cu",
              "kann_search_e4m3.cu", "kann_search_f32_multi.cu", "kann_search_f16_multi.cu",
              "kann_search_bf16_multi.cu", "kann_search_e4m3_multi.cu", "kann_search_f32_team.cu",
              "kann_search_f16_team.cu", "kann_search_bf16_team.cu", "kann_search_e4m3_team.cu",
              "kann_exact.cu", "kann_exact_tc.cu",
              "kann_pq.cu", "kann_exact_sparse.cu", "kann_build_gpu.cu"]
CPP_SOURCES = ["kann_build.cpp"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _sources():
    names = CU_SOURCES + CPP_SOURCES + [f for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    return [os.path.join(CSRC, f) for f in names] + [os.path.join(INCLUDE, "kann.h")]


def build(force=False, verbose=False):
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(s) <= t for s in _sources()):
            return LIB
    bdir = os.path.join(HERE, "_build")
    os.makedirs(bdir, exist_ok=True)
    objs = []
    cmds = []
    for src in CU_SOURCES:
        obj = os.path.join(bdir, src + ".o")
        cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE,
               "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        cmds.append(cmd)
        objs.append(obj)
    procs = [subprocess.Popen(c) for c in cmds]
    codes = [p.wait() for p in procs]
    if any(codes):
        raise RuntimeError("nvcc failed: %s" % codes)
    for src in CPP_SOURCES:
        obj = os.path.join(bdir, src + ".o")
        subprocess.check_call(["g++", "-std=c++17", "-O3", "-fPIC", "-pthread", "-I" + INCLUDE, "-c",
                               os.path.join(CSRC, src), "-o", obj])
        objs.append(obj)
    tmp = LIB + ".tmp%d" % os.getpid()
    subprocess.check_call([NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-Xcompiler", "-pthread", "-lcudart"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
