"""Build the native library (libgfs.so) in-tree for sm_103a.

nvcc compiles the CUDA translation units for `-gencode arch=compute_103a,code=sm_103a`
and the host translation units as C++17; the objects are linked into
paper_2109_05366_gb300/libgfs.so (static cudart).  The device-side file API of
include/gfs_device.h is compiled as relocatable device code into
paper_2109_05366_gb300/libgfs_device.a, which user kernels link with
`nvcc -rdc=true`.  Translation units compile in parallel; nothing is rebuilt when
no source changed.
"""
from __future__ import annotations

import hashlib
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIB = os.path.join(PKG, "libgfs.so")
DEVLIB = os.path.join(PKG, "libgfs_device.a")
BUILD_DIR = os.path.join(ROOT, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["gfs_scan_wide.cu", "gfs_scan_narrow.cu", "gfs_kernels.cu", "gfs_serve.cu", "gfs_apps.cu", "gfs_host.cpp",
           "gfs_service.cpp"]
DEVAPI_SOURCE = "gfs_devapi.cu"  # relocatable device code: libgfs_device.a
HEADERS = ["gfs_internal.h", "gfs_device.cuh", "gfs_scan.cuh", "gfs_host.h", "gfs_service.h", "gfs_serve.h"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgfs.so")


def _digest() -> str:
    h = hashlib.sha256()
    for name in SOURCES + [DEVAPI_SOURCE] + HEADERS:
        with open(os.path.join(CSRC, name), "rb") as f:
            h.update(name.encode() + b"\0" + f.read())
    for name in ("gfs.h", "gfs_device.h"):
        with open(os.path.join(ROOT, "include", name), "rb") as f:
            h.update(f.read())
    h.update(" ".join(ARCH).encode())
    return h.hexdigest()


# The sources the stride-scan kernel is compiled from (its device code); profiles
# taken on one build stay valid while these are unchanged.
KERNEL_SOURCES = ["gfs_scan.cuh", "gfs_scan_wide.cu", "gfs_scan_narrow.cu", "gfs_kernels.cu", "gfs_device.cuh",
                  "gfs_internal.h"]


def _code_only(text: bytes) -> bytes:
    """C/C++ source without comments and with whitespace collapsed (a comment edit is not a code change)."""
    import re
    t = re.sub(rb"/\*.*?\*/", b" ", text, flags=re.S)
    t = re.sub(rb"//[^\n]*", b" ", t)
    return b" ".join(t.split())


def kernel_digest() -> str:
    """Digest of the stride-scan kernel's code (device code, shared layouts, ABI header, arch)."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(CSRC, name), "rb") as f:
            h.update(name.encode() + b"\0" + _code_only(f.read()))
    with open(os.path.join(ROOT, "include", "gfs.h"), "rb") as f:
        h.update(_code_only(f.read()))
    h.update(" ".join(ARCH).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libgfs.so unless it is up to date; returns its path."""
    digest = _digest()
    stamp = LIB + ".stamp"
    if not force and os.path.exists(LIB) and os.path.exists(DEVLIB) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == digest:
                return LIB
    nvcc = _nvcc()
    os.makedirs(BUILD_DIR, exist_ok=True)
    procs = []
    objs = []
    for src in SOURCES:
        obj = os.path.join(BUILD_DIR, os.path.splitext(src)[0] + ".o")
        objs.append(obj)
        cmd = [nvcc, "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cu"):
            cmd[1:1] = ARCH + ["-lineinfo"]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    devobj = os.path.join(BUILD_DIR, "gfs_devapi.o")
    cmd = [nvcc] + ARCH + ["-lineinfo", "-O3", "-std=c++17", "-rdc=true", "-Xcompiler", "-fPIC", "-c",
                           os.path.join(CSRC, DEVAPI_SOURCE), "-o", devobj]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    procs.append((DEVAPI_SOURCE, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    errors = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            errors.append("%s:\n%s" % (src, out.decode(errors="replace")))
        elif verbose and out:
            print(out.decode(errors="replace"), file=sys.stderr)
    if errors:
        raise RuntimeError("libgfs build failed\n" + "\n".join(errors))
    tmp = LIB + ".%d.tmp" % os.getpid()
    subprocess.check_call([nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lpthread"])
    os.replace(tmp, LIB)
    tmp = DEVLIB + ".%d.tmp.a" % os.getpid()
    subprocess.check_call([nvcc] + ARCH + ["-lib", "-o", tmp, devobj])
    os.replace(tmp, DEVLIB)
    with open(stamp, "w") as f:
        f.write(digest + "\n")
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
