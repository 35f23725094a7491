"""Compile the CUDA sources into the in-tree C-ABI library ``_build/libbfpfft.so``.

Every translation unit is compiled for sm_103a only, in parallel, with nvcc
directly (no cmake, no torch extension machinery); the objects are linked
with the static CUDA runtime into one shared library that exports the
functions of include/bfpfft.h.
"""

from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB_NAME = "libbfpfft.so"
LIB_PATH = os.path.join(BUILD, LIB_NAME)

SOURCES = [
    "runtime.cu",
    "rows_f32.cu",
    "rows_f16.cu",
    "rows_fp8.cu",
    "sar_nn.cu",
    "sar_nt.cu",
    "sar_tt.cu",
    "metrics.cu",
    "autofocus.cu",
    "metrics_noalloc.cu",
    "uneven.cu",
    "pt_metrics.cu",
    "transpose.cu",
    "rows_adaptive.cu",
    "rows16.cu",
    "rda.cu",
    "twopass.cu",
    "af_tc.cu",
    "rows_tc8.cu",
]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-I" + INCLUDE, "-I" + CSRC]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libbfpfft.so")


def _inputs():
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    deps.append(os.path.abspath(__file__))
    return deps


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _run(cmd):
    p = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if p.returncode != 0:
        raise RuntimeError("command failed:\n" + " ".join(cmd) + "\n" + p.stdout)
    return p.stdout


def build(force: bool = False, jobs: int | None = None, extra_flags=()) -> str:
    """Build (if stale) and return the path of libbfpfft.so."""
    os.makedirs(BUILD, exist_ok=True)
    deps = _inputs()
    if not force and not _stale(LIB_PATH, deps):
        return LIB_PATH
    nvcc = _nvcc()
    objs = []
    cmds = []
    for src in SOURCES:
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(obj)
        if force or _stale(obj, deps):
            cmds.append([nvcc] + NVCC_FLAGS + list(extra_flags) + ["-c", os.path.join(CSRC, src), "-o", obj])
    jobs = jobs or min(len(SOURCES), os.cpu_count() or 4)
    with ThreadPoolExecutor(max_workers=jobs) as ex:
        list(ex.map(_run, cmds))
    tmp = LIB_PATH + ".tmp"
    _run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    print(build(force=True))
