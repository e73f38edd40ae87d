"""Build libmln.so in-tree with nvcc for sm_103a (GB300).

Each translation unit compiles in its own process, in parallel; the objects
are linked into paper_1710_09799_gb300/_build/libmln.so with the static CUDA
runtime. Nothing is installed outside the package directory.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libmln.so")

SOURCES = ["api.cu", "kernels_fp64.cu", "kernels_fp32.cu", "kernels_tc.cu", "kernels_tcr.cu", "setup.cpp", "static_scratch.cu", "batch.cu",
           "adjoint.cu", "jit.cu", "project.cu", "pstd.cu"]
HEADERS = ["kernels.cuh", "dispatch.cuh", "setup.h", "ctx.h", "adjoint.cuh", "jit.h", "tc.cuh", "tc_kernel.h",
           "pstd.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC, "-I", BUILD]


def nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    deps = [src, os.path.join(INCLUDE, "mln.h")] + [os.path.join(CSRC, h) for h in HEADERS]
    return any(os.path.getmtime(d) > t for d in deps)


def write_jit_source() -> str:
    """kernels.cuh as a C++ string literal, compiled into the library for the
    per-problem kernels it generates and compiles at run time (NVRTC)."""
    src = open(os.path.join(CSRC, "kernels.cuh")).read()
    assert ")MLNSRC" not in src
    path = os.path.join(BUILD, "jit_source.inc")
    text = "static const char *kKernelsSource = R\"MLNSRC(" + src + ")MLNSRC\";\n"
    if not os.path.exists(path) or open(path).read() != text:
        with open(path, "w") as f:
            f.write(text)
    return path


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    os.makedirs(BUILD, exist_ok=True)
    write_jit_source()
    extra = list(extra or [])
    procs = []
    objs = []
    for s in SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(BUILD, os.path.splitext(s)[0] + ".o")
        objs.append(obj)
        if not force and not _stale(obj, src):
            continue
        cmd = [nvcc()] + ARCH + FLAGS + extra + ["-c", src, "-o", obj]
        if s.endswith(".cpp"):
            cmd = [nvcc(), "-x", "c++"] + FLAGS + extra + ["-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((s, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for s, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((s, out.decode(errors="replace")))
        elif verbose and out:
            print(out.decode(errors="replace"), file=sys.stderr)
    if failed:
        msg = "\n".join(f"--- {s}\n{o}" for s, o in failed)
        raise RuntimeError(f"nvcc failed:\n{msg}")
    if force or procs or not os.path.exists(LIB):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-cudart", "static", "-ldl"]
        subprocess.check_call(cmd)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
