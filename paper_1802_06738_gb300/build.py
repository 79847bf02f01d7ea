"""In-tree build of libpnoeom.so for sm_103a (nvcc, parallel compilation)."""
from __future__ import annotations

import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(HERE, "libpnoeom.so")
SOURCES = ["engine.cu", "sigma_kernels.cu", "build.cu", "build_program.cu", "solve.cu", "capi.cu", "noalloc.cu", "peaks.cu", "sandwich_tc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else (shutil.which("nvcc") or "nvcc")


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every CUDA source for sm_103a and link libpnoeom.so in-tree."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    nvcc = _nvcc()
    flags = ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-diag-suppress", "177"]
    objs, procs = [], []
    lib_mtime = os.path.getmtime(LIB_PATH) if os.path.exists(LIB_PATH) else -1
    newest = 0.0
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        obj = os.path.join(BUILD_DIR, src.replace(".cu", ".o"))
        objs.append(obj)
        deps = [s] + [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith(".cuh")] + \
               [os.path.join(HERE, "..", "include", "pnoeom.h")]
        m = max(os.path.getmtime(d) for d in deps)
        newest = max(newest, m)
        if force or not os.path.exists(obj) or os.path.getmtime(obj) < m:
            cmd = [nvcc] + flags + ["-c", s, "-o", obj]
            procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{out.decode()}")
        if verbose and out:
            print(out.decode())
    if force or procs or lib_mtime < newest:
        cmd = [nvcc] + ARCH + ["-shared", "-o", LIB_PATH] + objs + ["-lcusolver", "-lcublas", "-lcudart"]
        r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + r.stdout.decode())
    return LIB_PATH


if __name__ == "__main__":
    print(build(verbose=True))
