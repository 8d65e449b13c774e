"""Build the in-tree host library libchem.so (C++ host code; the CUDA kernels themselves are
generated per mechanism and compiled for sm_103a by NVRTC at load time, see csrc/chem_host.cpp).

The device source csrc/ros4_device.cuh is embedded into the library as a string so that the
library is self-contained.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libchem.so")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")
SOURCES = [os.path.join(CSRC, "chem_host.cpp"), os.path.join(CSRC, "ros4_device.cuh"),
           os.path.join(ROOT, "include", "chem.h")]


def _embed(dst: str) -> None:
    src = open(os.path.join(CSRC, "ros4_device.cuh")).read()
    delim = "CHEMSRC"
    assert ")" + delim not in src
    # split into chunks below the portable string-literal limit and concatenate
    chunks = [src[i:i + 60000] for i in range(0, len(src), 60000)]
    body = "\n".join('R"%s(%s)%s"' % (delim, c, delim) for c in chunks)
    text = "static const char* const kDeviceSource =\n%s;\n" % body
    if not os.path.exists(dst) or open(dst).read() != text:
        with open(dst, "w") as fh:
            fh.write(text)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    inc = os.path.join(OUT_DIR, "device_src.inc")
    _embed(inc)
    newest = max(os.path.getmtime(p) for p in SOURCES + [inc])
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-Wall",
           "-I", os.path.join(ROOT, "include"), "-I", OUT_DIR, "-I", os.path.join(CUDA, "include"),
           os.path.join(CSRC, "chem_host.cpp"), "-o", tmp,
           "-L", os.path.join(CUDA, "lib64"),
           "-Wl,-rpath," + os.path.join(CUDA, "lib64"), "-lnvrtc", "-ldl", "-lpthread"]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
