"""In-tree build of libpradmm.so for sm_103a (nvcc + g++, no cmake).

The CUDA translation units and the host C++ translation unit compile in
parallel; nvcc links them into `paper_2601_15684_gb300/_lib/libpradmm.so`
with the CUDA runtime linked statically.

build(debug=True) also links `_lib/libpradmm_debug.so`: the plain sweeps and
the host code recompiled with -DPRADMM_DEBUG_CHECKS=1 (every neighbour index
and CSR row bound a sweep reads is range-checked on the device and the run
fails with PRADMM_ERR_INDEX if one is out of range), the other objects
shared with the release build.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libpradmm.so")
LIB_DEBUG = os.path.join(LIBDIR, "libpradmm_debug.so")
BUILD_DEBUG = os.path.join(HERE, "_build_debug")
# translation units that carry the index checks of the debug build
DEBUG_UNITS = ["pradmm_kernels.cu", "pradmm_api.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

CU_SOURCES = ["pradmm_kernels.cu", "pradmm_batch.cu", "pradmm_batch_inert.cu", "pradmm_adjoint.cu", "pradmm_sigma.cu",
              "pradmm_noalloc.cu", "pradmm_setup.cu", "pradmm_forest.cu"]
# sources compiled once per set of defines (object name suffix, defines): the
# batched general-Sigma kernels, one object per precision and inertial flag
CU_SPLIT = {"pradmm_batch_sigma.cu": [(f"{r}{'_inert' if i else ''}",
                                       [f"-DPRADMM_BATCH_SIGMA_R={r}", f"-DPRADMM_BATCH_SIGMA_INERT={str(i).lower()}"])
                                      for r in ("float", "double") for i in (False, True)]}
CPP_SOURCES = ["pradmm_api.cpp"]
HEADERS = [os.path.join(CSRC, "pradmm_internal.h"), os.path.join(CSRC, "pradmm_device.cuh"),
           os.path.join(CSRC, "pradmm_batch.cuh"), os.path.join(CSRC, "pradmm_sigma.cuh"),
           os.path.join(INCLUDE, "pradmm.h")]


def _cuda_home() -> str:
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    return os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _nvcc() -> str:
    return shutil.which("nvcc") or os.path.join(_cuda_home(), "bin", "nvcc")


def _stale(out: str, deps: list[str]) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    cuda_inc = os.path.join(_cuda_home(), "include")
    jobs = []
    objs = []
    for src in CU_SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src + ".o")
        objs.append(o)
        if force or _stale(o, [s] + HEADERS):
            jobs.append([_nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                         "-I", INCLUDE, "-I", CSRC, "-c", s, "-o", o])
    for src, variants in CU_SPLIT.items():
        s = os.path.join(CSRC, src)
        for tag, defs in variants:
            o = os.path.join(BUILD, f"{src}.{tag}.o")
            objs.append(o)
            if force or _stale(o, [s] + HEADERS):
                jobs.append([_nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", *defs,
                             "-I", INCLUDE, "-I", CSRC, "-c", s, "-o", o])
    for src in CPP_SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src + ".o")
        objs.append(o)
        if force or _stale(o, [s] + HEADERS):
            # no contraction into fused multiply-adds: the host arithmetic that the
            # device repeats (quaternion normalisation) rounds the same on both
            jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", "-Wall", "-pthread", "-ffp-contract=off", "-I", INCLUDE,
                         "-I", CSRC, "-I", cuda_inc, "-c", s, "-o", o])
    procs = [(j, subprocess.Popen(j, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)) for j in jobs]
    errors = []
    for j, p in procs:
        out, _ = p.communicate()
        if verbose and out:
            sys.stdout.write(out)
        if p.returncode != 0:
            errors.append(" ".join(j) + "\n" + (out or ""))
    if errors:
        raise RuntimeError("libpradmm build failed:\n" + "\n".join(errors))
    if force or jobs or _stale(LIB, objs):
        _link(LIB, objs)
    if debug:
        _build_debug(objs, force, cuda_inc)
    return LIB


def _link(out: str, objs: list[str]) -> None:
    tmp = out + f".tmp{os.getpid()}"
    cmd = [_nvcc(), *ARCH, "-shared", "-Xcompiler", "-fPIC", "-o", tmp, *objs, "-cudart", "static", "-lpthread"]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("libpradmm link failed:\n" + " ".join(cmd) + "\n" + r.stdout)
    os.replace(tmp, out)


def _build_debug(release_objs: list[str], force: bool, cuda_inc: str) -> None:
    os.makedirs(BUILD_DEBUG, exist_ok=True)
    objs, procs = [], []
    for o in release_objs:
        src = os.path.basename(o)[:-2]
        if src not in DEBUG_UNITS:
            objs.append(o)
            continue
        s = os.path.join(CSRC, src)
        od = os.path.join(BUILD_DEBUG, os.path.basename(o))
        objs.append(od)
        if not (force or _stale(od, [s] + HEADERS)):
            continue
        if src.endswith(".cu"):
            cmd = [_nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-DPRADMM_DEBUG_CHECKS=1",
                   "-I", INCLUDE, "-I", CSRC, "-c", s, "-o", od]
        else:
            cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-Wall", "-pthread", "-ffp-contract=off", "-DPRADMM_DEBUG_CHECKS=1",
                   "-I", INCLUDE, "-I", CSRC, "-I", cuda_inc, "-c", s, "-o", od]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError("libpradmm debug build failed:\n" + " ".join(cmd) + "\n" + (out or ""))
    if force or procs or _stale(LIB_DEBUG, objs):
        _link(LIB_DEBUG, objs)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
