"""Build libzmc.so in-tree (paper_1902_07916_gb300/_build/) with nvcc for sm_103a.

Translation units are compiled in parallel and linked into one shared
library with the CUDA runtime linked statically, so the library loads on any
host with the NVIDIA driver (and on hosts without one, for symbol checks).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
GEN = os.path.join(BUILD, "gen")
LIB = os.path.join(BUILD, "libzmc.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

SOURCES = ["eval_fp64.cu", "eval_fp32.cu", "eval_fp32k.cu", "batch_fp64.cu", "batch_fp32.cu",
           "batch_fp32k.cu", "batch.cu", "select.cu", "api.cu", "jit.cu", "probe.cu"]
# Device headers handed to NVRTC for expression integrands, under the names
# their #include lines use.
JIT_HEADERS = [
    ("../../include/zmc.h", os.path.join(INCLUDE, "zmc.h")),
    ("zmc_layout.h", os.path.join(CSRC, "zmc_layout.h")),
    ("zmc_device.cuh", os.path.join(CSRC, "zmc_device.cuh")),
    ("eval_kernel.cuh", os.path.join(CSRC, "eval_kernel.cuh")),
]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
         "--expt-relaxed-constexpr", "-I" + GEN, "-I" + INCLUDE]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libzmc")


def _gen_jit_sources() -> str:
    os.makedirs(GEN, exist_ok=True)
    path = os.path.join(GEN, "jit_sources.inc")
    parts = ["// generated by paper_1902_07916_gb300/build.py -- do not edit\n"]
    names, bodies = [], []
    for name, src in JIT_HEADERS:
        with open(src) as fh:
            text = fh.read()
        assert ")ZMCSRC\"" not in text
        names.append('"%s"' % name)
        bodies.append('R"ZMCSRC(%s)ZMCSRC"' % text)
    parts.append("static const int kJitNumHeaders = %d;\n" % len(names))
    parts.append("static const char* const kJitHeaderNames[] = {%s};\n" % ", ".join(names))
    parts.append("static const char* const kJitHeaders[] = {\n%s};\n" % ",\n".join(bodies))
    text = "".join(parts)
    if not os.path.exists(path) or open(path).read() != text:
        with open(path, "w") as fh:
            fh.write(text)
    return path


def _newest_input() -> float:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files += [os.path.join(INCLUDE, "zmc.h"), os.path.abspath(__file__)]
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile every translation unit and link libzmc.so; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    _gen_jit_sources()
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= _newest_input()):
        return LIB
    nvcc = _nvcc()
    extra = ["-Xptxas", "-v"] if ptxas_info else []

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose or ptxas_info:
        for _, err in results:
            sys.stderr.write(err)
    objs = [o for o, _ in results]
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-ldl", "-lpthread", "-lrt"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True,
                ptxas_info="--ptxas-info" in sys.argv))
