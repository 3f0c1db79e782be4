"""Compile the CUDA engine into an in-tree shared library (libsnn.so).

sm_103a only: every translation unit is compiled with
``-gencode arch=compute_103a,code=sm_103a`` and ``-fmad=false`` (no fused
multiply-add anywhere in device code), host code with ``-ffp-contract=off``.
The translation units compile in parallel; nothing here needs a GPU.
"""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD_DIR = os.path.join(PKG, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "libsnn.so")
# the checked build (-DSNN_CHECKED): every step kernel verifies its computed
# indices before use; a bad one sets the device error word (SNN_EBOUNDS) and
# the access is skipped
CHECKED_DIR = os.path.join(BUILD_DIR, "checked")
CHECKED_LIB_PATH = os.path.join(BUILD_DIR, "libsnn_checked.so")
SOURCES = ["snn_build.cu", "snn_step.cu", "snn_dense.cu", "snn_api.cu", "snn_microbench.cu"]
HEADERS = ["snn_internal.cuh"]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-fmad=false", "-Xcompiler", "-fPIC,-ffp-contract=off",
              "-I", INCLUDE, "-I", CSRC] + ARCH


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA engine cannot be built")
    return path


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags=(), checked: bool = False) -> str:
    obj_dir = CHECKED_DIR if checked else BUILD_DIR
    lib_path = CHECKED_LIB_PATH if checked else LIB_PATH
    if checked:
        extra_flags = tuple(extra_flags) + ("-DSNN_CHECKED",)
    os.makedirs(obj_dir, exist_ok=True)
    headers = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(INCLUDE, "snn.h")]
    jobs = []
    objs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(obj_dir, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + headers):
            jobs.append([nvcc(), *NVCC_FLAGS, *extra_flags, "-c", s, "-o", o])

    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r.stdout + r.stderr

    with concurrent.futures.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        for out in ex.map(run, jobs):
            if verbose and out.strip():
                print(out)
    if force or jobs or _stale(lib_path, objs):
        tmp = lib_path + ".tmp%d" % os.getpid()
        run([nvcc(), "-shared", *ARCH, "-Xcompiler", "-fPIC", "-o", tmp, *objs])
        os.replace(tmp, lib_path)
    return lib_path


def build_all(force: bool = False, verbose: bool = False):
    """The library and its checked build, compiled side by side."""
    with concurrent.futures.ThreadPoolExecutor(max_workers=2) as ex:
        a = ex.submit(build, force, verbose)
        b = ex.submit(build, force, verbose, (), True)
        return a.result(), b.result()


if __name__ == "__main__":
    import sys
    print(build_all(force="--force" in sys.argv, verbose=True))
