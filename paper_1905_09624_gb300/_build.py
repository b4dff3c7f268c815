"""Compile the CUDA library libcobs_gpu.so for sm_103a (GB300) in-tree.

One translation unit per .cu file (and per host-only .cpp file: the error
status and the serve scheduler), compiled in parallel, linked with the CUDA
runtime statically.  Output: paper_1905_09624_gb300/_lib/libcobs_gpu.so.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libcobs_gpu.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libcobs_gpu.so")


def _sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    return hs + [os.path.join(INCLUDE, "cobs_gpu.h")]


def _digest(paths, extra):
    h = hashlib.sha256(extra.encode())
    for p in sorted(paths):
        with open(p, "rb") as f:
            h.update(p.encode())
            h.update(f.read())
    return h.hexdigest()


def build(verbose: bool = False, ptxas_verbose: bool = False, extra_flags=(), lib_path: str = LIB,
          link_flags=()) -> str:
    """Build (or reuse) the library; returns its path.  lib_path / extra_flags /
    link_flags build a variant elsewhere (the tests build one whose host code
    runs under AddressSanitizer + UBSan)."""
    nvcc = _nvcc()
    flags = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
             "-I", INCLUDE, "-I", CSRC] + ARCH + list(extra_flags)
    # compile-time kernel geometry for experiments, e.g. "-DCOBS_PIPE_G=16 -DCOBS_PIPE_D=3"
    flags += os.environ.get("COBS_EXTRA_NVCC_FLAGS", "").split()
    if ptxas_verbose:
        flags += ["-Xptxas", "-v"]
    srcs = _sources()
    stamp_val = _digest(srcs + _headers(), " ".join(flags) + " ".join(link_flags) + nvcc)
    stamp = lib_path + ".stamp"
    if os.path.exists(lib_path) and os.path.exists(stamp) and open(stamp).read() == stamp_val:
        return lib_path
    libdir = os.path.dirname(lib_path)
    os.makedirs(libdir, exist_ok=True)
    objs = [os.path.join(libdir, os.path.splitext(os.path.basename(s))[0] + ".o") for s in srcs]

    def compile_one(src_obj):
        src, obj = src_obj
        cmd = [nvcc, "-c", src, "-o", obj] + flags
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
        return r.stdout + r.stderr

    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        logs = list(ex.map(compile_one, zip(srcs, objs)))
    if verbose or ptxas_verbose:
        for s, log in zip(srcs, logs):
            if log.strip():
                print(f"== {os.path.basename(s)}\n{log}")
    tmp = lib_path + f".{os.getpid()}.tmp"
    cmd = [nvcc, "-shared", "-o", tmp] + objs + ARCH + ["-Xcompiler", "-fPIC", "-lpthread", "-ldl"] + list(link_flags)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib_path)
    with open(stamp, "w") as f:
        f.write(stamp_val)
    return lib_path


if __name__ == "__main__":
    import sys
    print(build(verbose=True, ptxas_verbose="-v" in sys.argv))
