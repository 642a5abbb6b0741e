"""Build libdg.so in-tree for sm_103a (nvcc + g++, translation units in parallel).

Run ``python -m paper_1602_07997_gb300.build`` or call :func:`build`.
"""

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libdg.so")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

CU_SOURCES = ["dg_kernels_acoustic.cu", "dg_kernels_elastic.cu", "dg_kernels_tc_acoustic.cu", "dg_strategies.cu",
              "dg_kernels_tc_elastic.cu", "dg_dispatch.cu", "rhs_noalloc.cu",
              "fp32_peak.cu", "dg_ept.cu"]
CPP_SOURCES = ["api.cpp", "refelem.cpp", "mesh.cpp", "server.cpp"]


def _run(cmd):
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError("command failed: %s\n%s%s" % (" ".join(cmd), p.stdout, p.stderr))
    return p.stdout + p.stderr


def _newer(src_list, target):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in src_list)


def build(verbose=False, force=False, ptxas_info=False):
    os.makedirs(OUT, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(HERE, "..", "include", "dg.h"))
    jobs = []
    for f in CU_SOURCES:
        src = os.path.join(CSRC, f)
        obj = os.path.join(OUT, f + ".o")
        if force or _newer([src] + headers, obj):
            cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                   "--expt-relaxed-constexpr", "-c", src, "-o", obj]
            if ptxas_info:
                cmd.insert(1, "-Xptxas=-v")
            jobs.append(cmd)
    for f in CPP_SOURCES:
        src = os.path.join(CSRC, f)
        obj = os.path.join(OUT, f + ".o")
        if force or _newer([src] + headers, obj):
            jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", "-pthread", "-I" + os.path.join(CUDA, "include"),
                         "-c", src, "-o", obj])
    with ThreadPoolExecutor(max_workers=max(2, min(8, os.cpu_count() or 2))) as ex:
        outs = list(ex.map(_run, jobs))
    if verbose:
        for o in outs:
            if o.strip():
                print(o)
    objs = [os.path.join(OUT, f + ".o") for f in CU_SOURCES + CPP_SOURCES]
    if force or jobs or not os.path.exists(LIB):
        _run([NVCC, *ARCH, "-shared", "-cudart", "shared", "-o", LIB, *objs, "-lcublas", "-lpthread",
              "-Xlinker", "-rpath=" + os.path.join(CUDA, "lib64")])
    return LIB


if __name__ == "__main__":
    build(verbose=True, force="--force" in sys.argv, ptxas_info="--ptxas" in sys.argv)
    print(LIB)
