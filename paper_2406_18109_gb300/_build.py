"""Builds the in-tree shared library ``_lib/libdiffuse.so`` for sm_103a.

Steps: embed ``csrc/dfs_device.cuh`` as a string for NVRTC, compile the host
runtime (C++17) and the ahead-of-time device translation units (nvcc,
``-gencode arch=compute_103a,code=sm_103a``) in parallel, link against NVRTC
and the static CUDA runtime.  The driver API is reached through
``cudaGetDriverEntryPointByVersion``, so the library loads on machines without
a GPU driver (the analysis-only context and symbol checks still work there).
"""
from __future__ import annotations

import concurrent.futures as cf
import fcntl
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
OBJDIR = os.path.join(HERE, "_build")
LIB = os.path.join(LIBDIR, "libdiffuse.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

HOST_SOURCES = ["runtime.cpp", "fusion.cpp", "codegen.cpp", "batchgen.cpp", "jit.cpp", "partition.cpp"]
DEVICE_SOURCES = ["dfs_check.cu", "noalloc.cu", "gather.cu"]
GENCODE = "arch=compute_103a,code=sm_103a"


def cuda_home() -> str:
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return c
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(nvcc))
    raise RuntimeError("CUDA toolkit (nvcc) not found")


def _embed_device_header() -> None:
    src = open(os.path.join(CSRC, "dfs_device.cuh")).read()
    assert ')DFSRAW"' not in src
    text = f'static const char kDeviceSourceText[] = R"DFSRAW({src})DFSRAW";\n'
    out = os.path.join(CSRC, "dfs_device_src.inc")
    if not os.path.exists(out) or open(out).read() != text:
        with open(out, "w") as f:
            f.write(text)


def _inputs_digest() -> str:
    h = hashlib.sha256()
    for name in sorted(os.listdir(CSRC)):
        if name.endswith((".cpp", ".hpp", ".cu", ".cuh")):
            h.update(name.encode())
            h.update(open(os.path.join(CSRC, name), "rb").read())
    h.update(open(os.path.join(INCLUDE, "diffuse.h"), "rb").read())
    h.update(open(__file__, "rb").read())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False) -> str:
    """Compiles libdiffuse.so if its sources changed; returns its path.
    Processes that build at once (one per rank) take turns on a file lock, so
    the later ones find the library up to date."""
    os.makedirs(LIBDIR, exist_ok=True)
    with open(os.path.join(LIBDIR, ".build.lock"), "w") as lk:
        fcntl.flock(lk, fcntl.LOCK_EX)
        try:
            return _build_locked(force, verbose)
        finally:
            fcntl.flock(lk, fcntl.LOCK_UN)


def _build_locked(force: bool, verbose: bool) -> str:
    cuda = cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    os.makedirs(OBJDIR, exist_ok=True)
    _embed_device_header()
    digest = _inputs_digest()
    stamp = os.path.join(LIBDIR, "libdiffuse.stamp")
    if not force and os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read() == digest:
        return LIB
    common = ["-std=c++17", "-O2", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]
    jobs = []
    for s in HOST_SOURCES:
        obj = os.path.join(OBJDIR, s + ".o")
        jobs.append([nvcc, *common, "-c", os.path.join(CSRC, s), "-o", obj])
    for s in DEVICE_SOURCES:
        obj = os.path.join(OBJDIR, s + ".o")
        jobs.append([nvcc, *common, "-gencode", GENCODE, "-lineinfo", "-Xptxas", "-v" if verbose else "-O3",
                     "-c", os.path.join(CSRC, s), "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r.stdout + r.stderr

    with cf.ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
        logs = list(ex.map(run, jobs))
    if verbose:
        for lg in logs:
            if lg.strip():
                print(lg)
    objs = [os.path.join(OBJDIR, s + ".o") for s in HOST_SOURCES + DEVICE_SOURCES]
    tmp = LIB + ".tmp"
    run([nvcc, "-shared", "-gencode", GENCODE, "-o", tmp, *objs, "-cudart", "static",
         "-L", os.path.join(cuda, "lib64"), "-lnvrtc",
         "-Xlinker", "-rpath," + os.path.join(cuda, "lib64"), "-Xlinker", "--no-undefined"])
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(digest)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
