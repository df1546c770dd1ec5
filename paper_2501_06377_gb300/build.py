"""Build libsft.so in-tree with nvcc for sm_103a (GB300).

The translation units compile in parallel; the library is rebuilt only
when a source, the header or the flags change (a stamp file records their
hash).  build(debug=True) makes libsft_debug.so instead: the same sources
with -DSFT_DEBUG, whose kernels check the indexes they derive (the checks
record a failure on the device and keep the access in bounds).
"""
from __future__ import annotations

import hashlib
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libsft.so")
LIB_DEBUG = os.path.join(PKG, "libsft_debug.so")
SOURCES = ["sft_api.cu", "sft_kernels.cu", "sft_noalloc.cu", "sfs.cu", "sfs_fused.cu", "sfs_gemm.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: libsft needs the CUDA toolkit to build")
    return cand


def _stamp(flags) -> str:
    h = hashlib.sha256()
    h.update(" ".join(flags).encode())
    headers = ["../../include/" + f for f in sorted(os.listdir(INCLUDE)) if f.endswith(".h")]
    for name in sorted(os.listdir(CSRC)) + headers:
        p = os.path.normpath(os.path.join(CSRC, name))
        if os.path.isfile(p):
            h.update(name.encode())
            with open(p, "rb") as f:
                h.update(f.read())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Compile libsft.so (libsft_debug.so with debug=True) if needed and
    return its path."""
    flags = FLAGS + ["-DSFT_DEBUG"] if debug else FLAGS
    lib = LIB_DEBUG if debug else LIB
    bdir = BUILD + "_debug" if debug else BUILD
    stamp_path = os.path.join(bdir, "stamp")
    stamp = _stamp(flags)
    if not force and os.path.exists(lib) and os.path.exists(stamp_path):
        with open(stamp_path) as f:
            if f.read() == stamp:
                return lib
    os.makedirs(bdir, exist_ok=True)
    nvcc = _nvcc()
    procs, objs = [], []
    for src in SOURCES:
        obj = os.path.join(bdir, src.replace(".cu", ".o"))
        objs.append(obj)
        cmd = [nvcc, *flags, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd))
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError("nvcc failed: %s\n%s" % (" ".join(cmd), out.decode(errors="replace")))
    tmp = lib + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
    out = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if out.returncode != 0:
        raise RuntimeError("link failed: %s\n%s" % (" ".join(cmd), out.stdout.decode(errors="replace")))
    os.replace(tmp, lib)
    with open(stamp_path, "w") as f:
        f.write(stamp)
    return lib


if __name__ == "__main__":
    print(build(verbose=True))
