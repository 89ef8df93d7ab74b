"""Build libzmc.so in-tree (paper_1902_07916_gb300/_build/) with nvcc for sm_103a.

Translation units are compiled in parallel and linked into one shared
library with the CUDA runtime linked statically, so the library loads on any
host with the NVIDIA driver (and on hosts without one, for symbol checks).
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
GEN = os.path.join(BUILD, "gen")
LIB = os.path.join(BUILD, "libzmc.so")
# the bounds-guarded test build (ZMC_CHECKED): its own objects and library
BUILD_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(BUILD_CHECKED, "libzmc.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

SOURCES = ["batch.cu", "select.cu", "api.cu", "jit.cu", "probe.cu"]
# The sampling kernels, single-integral and batched, of each precision mode
# (0: FP64, 1: FP32 + FP64 accumulation, 2: FP32 Kahan) in four parts of two
# registry integrands each: one small generated translation unit per
# (kind, mode, part), so that the heavy template instantiations compile in
# parallel.
KERNEL_PARTS = 4
KERNEL_TUS = [(kind, mode, part) for kind in ("eval", "batch") for mode in (0, 1, 2)
              for part in range(KERNEL_PARTS)]
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
         "--expt-relaxed-constexpr", "-I" + GEN, "-I" + INCLUDE, "-I" + CSRC]


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


def _gen_kernel_tus() -> list:
    """Write the per-(kind, mode, part) translation units into gen/ (only when
    their text changes); returns their paths."""
    os.makedirs(GEN, exist_ok=True)
    paths = []
    for kind, mode, part in KERNEL_TUS:
        header = "eval_kernel.cuh" if kind == "eval" else "batch_kernel.cuh"
        text = ("// generated by paper_1902_07916_gb300/build.py -- do not edit\n"
                "#include \"%s\"\n#include \"zmc_internal.h\"\n\n"
                "namespace zmc {\n"
                "template <> const void* %s_kernel_part<%d, %d>(int fn, int d) {\n"
                "    return %s_kernel_pair<%d, %d>(fn, d);\n}\n"
                "}  // namespace zmc\n" % (header, kind, mode, part, kind, mode, part))
        path = os.path.join(GEN, "%s_m%d_p%d.cu" % (kind, mode, part))
        if not os.path.exists(path) or open(path).read() != text:
            with open(path, "w") as fh:
                fh.write(text)
        paths.append(path)
    return paths


def _newest_input() -> float:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files += [os.path.join(INCLUDE, "zmc.h"), os.path.abspath(__file__)]
    return max(os.path.getmtime(f) for f in files)


def _build_id(sources: list, checked: bool) -> str:
    """64-bit hash of everything that goes into the library (sources,
    headers, flags); the tuner's file cache keys its entries by it."""
    h = hashlib.sha256()
    files = sorted(set(sources) | {os.path.join(CSRC, f) for f in os.listdir(CSRC)}
                   | {os.path.join(INCLUDE, "zmc.h")})
    for f in files:
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    h.update(" ".join(ARCH + FLAGS + (["checked"] if checked else [])).encode())
    return "0x%sULL" % h.hexdigest()[:16]


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False,
          checked: bool = False) -> str:
    """Compile every translation unit and link libzmc.so; returns its path.
    checked=True builds the bounds-guarded test library instead
    (ZMC_CHECKED, two registry integrands) into _build_checked/."""
    build_dir = BUILD_CHECKED if checked else BUILD
    lib = LIB_CHECKED if checked else LIB
    os.makedirs(build_dir, exist_ok=True)
    _gen_jit_sources()
    sources = [os.path.join(CSRC, f) for f in SOURCES] + _gen_kernel_tus()
    if (not force and os.path.exists(lib)
            and os.path.getmtime(lib) >= _newest_input()):
        return lib
    nvcc = _nvcc()
    extra = ["-Xptxas", "-v"] if ptxas_info else []
    if checked:
        extra = extra + ["-DZMC_CHECKED"]
    extra = extra + ["-DZMC_BUILD_ID=" + _build_id(sources, checked)]

    def compile_one(src):
        obj = os.path.join(build_dir, os.path.splitext(os.path.basename(src))[0] + ".o")
        cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        return obj, r.stderr

    # the longest units first, so the pool's tail is short
    order = sorted(sources, key=lambda p: 0 if "_kernel_part" in p or "/gen/" in p else 1)
    with cf.ThreadPoolExecutor(max_workers=max(2, os.cpu_count() or 2)) as ex:
        results = list(ex.map(compile_one, order))
    if verbose or ptxas_info:
        for _, err in results:
            sys.stderr.write(err)
    objs = [o for o, _ in results]
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-ldl", "-lpthread", "-lrt"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True,
                ptxas_info="--ptxas-info" in sys.argv, checked="--checked" in sys.argv))
