"""Compile tests/devapi_user.cu (a user's kernel calling the device API) with nvcc.

The kernel sees include/ only and links the device API library libgfs_device.a
(relocatable device code), as a library user's kernel does."""
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "devapi_user.cu")


def build_user_kernel(outdir: str) -> str:
    nvcc = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    out = os.path.join(outdir, "devapi_user.so")
    devlib = os.path.join(ROOT, "paper_2109_05366_gb300", "libgfs_device.a")
    subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17", "-rdc=true",
                           "-shared", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"), SRC, devlib,
                           "-o", out])
    return out
