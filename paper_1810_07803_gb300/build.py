"""In-tree build of liblbc.so (CUDA kernels + C ABI) for sm_103a with nvcc.

Translation units compile in parallel, then link into one shared library next
to this file. Host code uses no machine-specific flags, so the same command
builds on x86_64 and aarch64 hosts.

build(checked=True) makes the range-checked variant liblbc_checked.so: the
kernels' translation unit compiled with LBC_CHECKED (every computed index
checked before its access; a failed check skips the access and is reported as
LBC_EBOUNDS), linked with the other objects of the normal build.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "liblbc.so")
LIB_CHECKED = os.path.join(HERE, "liblbc_checked.so")
CHECKED_TU = "lbc_kernels.cu"   # the translation unit that holds the range checks
BUILD = os.path.join(HERE, "_build")
SOURCES = ["lbc_api.cu", "lbc_setup.cu", "lbc_pool.cu", "lbc_kernels.cu", "lbc_host.cpp", "lbc_noalloc.cu",
           "lbc_peak.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblbc.so")


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "lbc.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(cc: str, src: str, obj: str, extra: list[str], verbose: bool) -> str:
    cmd = [cc, *FLAGS, *extra, *ARCH, "-c", os.path.join(CSRC, src), "-o", obj]
    if verbose:
        print(" ".join(cmd))
    subprocess.check_call(cmd)
    return obj


def _link(cc: str, lib: str, objs: list[str]) -> None:
    tmp = lib + f".tmp{os.getpid()}"
    subprocess.check_call([cc, *ARCH, "-shared", "-o", tmp, *objs])
    os.replace(tmp, lib)


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    if checked:
        return build_checked(force, verbose)
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    with cf.ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(lambda f: _compile(cc, f, os.path.join(BUILD, f + ".o"), [], verbose), SOURCES))
    _link(cc, LIB, objs)
    return LIB


def build_checked(force: bool = False, verbose: bool = False) -> str:
    """liblbc_checked.so: the normal build's objects with the kernels recompiled under LBC_CHECKED."""
    build(force, verbose)
    if any(not os.path.exists(os.path.join(BUILD, f + ".o")) for f in SOURCES if f != CHECKED_TU):
        build(True, verbose)   # the library exists but its objects do not
    if not force and not _stale(LIB_CHECKED):
        return LIB_CHECKED
    cc = nvcc()
    ck = _compile(cc, CHECKED_TU, os.path.join(BUILD, CHECKED_TU + ".checked.o"), ["-DLBC_CHECKED"], verbose)
    objs = [ck if f == CHECKED_TU else os.path.join(BUILD, f + ".o") for f in SOURCES]
    _link(cc, LIB_CHECKED, objs)
    return LIB_CHECKED


if __name__ == "__main__":
    import sys

    print(build(force=True, verbose=True, checked="--checked" in sys.argv[1:]))
