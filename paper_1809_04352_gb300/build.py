"""Build libeses.so in-tree with nvcc for sm_103a (GB300).

Each CUDA translation unit is compiled in parallel to an object file under
``_build/`` and linked into ``libeses.so`` next to this file.  The build is
skipped when the library is newer than every source.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libeses.so")
PEAKS_LIB = os.path.join(HERE, "libpeaks.so")  # FMA-rate microbenchmark (measurement only, not part of libeses)
SOURCES = ["eses_api.cu", "eses_scan.cu", "eses_model.cu", "eses_classify.cu", "eses_edges.cu", "eses_noalloc.cu",
           "eses_mlp.cu", "eses_exterior.cu", "eses_mesh.cu"]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libeses")


def _flags():
    return [ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-Wno-deprecated-declarations",
            "-diag-suppress", "1444", "-I", INCLUDE, "-I", CSRC,
            "--expt-relaxed-constexpr"]


def _deps():
    out = [os.path.join(INCLUDE, "eses.h")]
    for f in os.listdir(CSRC):
        if f.endswith((".cu", ".cuh", ".h")):
            out.append(os.path.join(CSRC, f))
    out.append(os.path.abspath(__file__))
    return out


def up_to_date() -> bool:
    for lib in (LIB, PEAKS_LIB):
        if not os.path.exists(lib):
            return False
        t = os.path.getmtime(lib)
        if not all(os.path.getmtime(d) <= t for d in _deps()):
            return False
    return True


def build(force: bool = False, verbose: bool = False, ptxas_verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    objs = []

    def compile_one(src):
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [nvcc] + _flags() + (["-Xptxas", "-v"] if ptxas_verbose else []) + ["-c", os.path.join(CSRC, src),
                                                                               "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose or ptxas_verbose:
            print(r.stdout + r.stderr)
        return obj

    def build_peaks():
        tmp = PEAKS_LIB + f".tmp{os.getpid()}"
        cmd = [nvcc] + _flags() + ["-shared", os.path.join(CSRC, "peaks.cu"), "-o", tmp]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for peaks.cu:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, PEAKS_LIB)

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES) + 1) as ex:
        peaks = ex.submit(build_peaks)
        objs = list(ex.map(compile_one, SOURCES))
        peaks.result()
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, ARCH, "-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
