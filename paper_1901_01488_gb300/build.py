"""Builds libesc.so in-tree for sm_103a (nvcc + the host C++ compiler), and
libesc_checked.so, the same sources compiled with -DESC_CHECKED: kernels
that test every index they use and report ESC_EBOUNDS instead of touching
memory out of range (the stand-in for a memory checker; tests load it with
ESC_CHECKED=1 in the environment).

Usage: python -m paper_1901_01488_gb300.build [--force]
"""
from __future__ import annotations

import fcntl
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libesc.so")
LIB_CHECKED = os.path.join(HERE, "libesc_checked.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU = ["esc_scan.cu", "esc_semijoin.cu", "esc_mlp.cu"]
CPP = ["esc_host.cpp"]
HEADERS = [os.path.join(CSRC, "esc_internal.h"), os.path.join(ROOT, "include", "esc.h")]


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src: str, verbose_ptxas: bool, checked: bool = False) -> str:
    obj = os.path.join(OBJ, ("checked_" if checked else "") + os.path.splitext(src)[0] + ".o")
    path = os.path.join(CSRC, src)
    if not _stale(obj, [path] + HEADERS):
        return obj
    defs = ["-DESC_CHECKED"] if checked else []
    if src.endswith(".cu"):
        cmd = [NVCC, *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC", *defs,
               "-I", os.path.join(ROOT, "include"), "-c", path, "-o", obj]
        if verbose_ptxas:
            cmd[1:1] = ["-Xptxas", "-v"]
    else:
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-Wall", *defs, "-I", "/usr/local/cuda/include",
               "-I", os.path.join(ROOT, "include"), "-c", path, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    if verbose_ptxas and r.stderr:
        sys.stderr.write(r.stderr)
    return obj


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    """Compiles what is out of date and links libesc.so; processes that build
    at the same time (one per GPU under torchrun) take turns on a file lock,
    so the later ones find everything up to date."""
    os.makedirs(OBJ, exist_ok=True)
    with open(os.path.join(OBJ, ".lock"), "w") as lock:
        fcntl.flock(lock, fcntl.LOCK_EX)
        try:
            return _build_locked(force, verbose_ptxas)
        finally:
            fcntl.flock(lock, fcntl.LOCK_UN)


def _build_locked(force: bool, verbose_ptxas: bool) -> str:
    if force:
        for f in os.listdir(OBJ):
            if f.endswith(".o"):
                os.remove(os.path.join(OBJ, f))
    jobs = [(s, False) for s in CU + CPP] + [(s, True) for s in CU + CPP]
    with ThreadPoolExecutor(len(jobs)) as ex:
        objs = list(ex.map(lambda j: _compile(j[0], verbose_ptxas, j[1]), jobs))
    n = len(CU) + len(CPP)
    for lib, lib_objs in ((LIB, objs[:n]), (LIB_CHECKED, objs[n:])):
        if force or _stale(lib, lib_objs):
            tmp = lib + f".tmp{os.getpid()}"
            cmd = [NVCC, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *lib_objs, "-ldl"]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
            os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv))
