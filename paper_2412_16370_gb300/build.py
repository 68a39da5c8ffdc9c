"""Build the package's CUDA libraries in-tree with nvcc (sm_103a only).

``libpospopcnt.so``: the counting kernels and the C ABI of
``include/pospopcnt.h``.  ``libpospop_synth.so``: the device input
generator of ``include/pospop_synth.h``.  Translation units compile in
parallel; a library is rebuilt only when a source or header is newer.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")

LIB = os.path.join(PKG, "libpospopcnt.so")
SYNTH_LIB = os.path.join(PKG, "libpospop_synth.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-I", INCLUDE, "-I", CSRC]

LIB_SOURCES = ["pospop_stream.cu", "pospop_batch.cu", "pospop_desc.cu", "pospop_api.cu",
               "pospop_tune.cu", "pospop_serve.cu", "pospop_noalloc.cu", "pospop_gather.cu",
               "pospop_select.cu", "pospop_roofline.cu", "pospop_multi.cu", "pospop_resident.cu"]
SYNTH_SOURCES = ["synth.cu"]


def nvcc() -> str:
    exe = shutil.which("nvcc")
    if exe:
        return exe
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpospopcnt")


def _deps() -> list[str]:
    out = []
    for d in (CSRC, INCLUDE):
        for f in os.listdir(d):
            if f.endswith((".h", ".cuh")):
                out.append(os.path.join(d, f))
    return out


def _stale(target: str, sources: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in sources + _deps())


def _run(cmd: list[str]) -> None:
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"build failed: {' '.join(cmd)}\n{r.stdout}")


def _plan(target: str, sources: list[str]):
    srcs = [os.path.join(CSRC, s) for s in sources if os.path.exists(os.path.join(CSRC, s))]
    if not _stale(target, srcs):
        return None
    objs = [os.path.join(BUILD, os.path.basename(s) + ".o") for s in srcs]
    return srcs, objs


def build(force: bool = False) -> list[str]:
    """Compile both libraries (if stale, or always with ``force``); return their paths."""
    if force:
        for p in (LIB, SYNTH_LIB):
            if os.path.exists(p):
                os.remove(p)
    libs = [(LIB, LIB_SOURCES, ["-ldl", "-lpthread"]), (SYNTH_LIB, SYNTH_SOURCES, [])]
    todo = []
    for target, sources, link in libs:
        plan = _plan(target, sources)
        if plan is not None:
            todo.append((target, plan[0], plan[1], link))
    if not todo:
        return [LIB, SYNTH_LIB]
    os.makedirs(BUILD, exist_ok=True)
    compiles = [(s, o) for _, srcs, objs, _ in todo for s, o in zip(srcs, objs)]
    with ThreadPoolExecutor(max_workers=max(1, min(len(compiles), os.cpu_count() or 1))) as pool:
        for f in [pool.submit(_run, [nvcc(), *NVCC_FLAGS, "-c", s, "-o", o]) for s, o in compiles]:
            f.result()
    for target, _, objs, link in todo:
        tmp = target + f".tmp{os.getpid()}"
        _run([nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs, *link])
        os.replace(tmp, target)
    return [LIB, SYNTH_LIB]


if __name__ == "__main__":
    for p in build(force="--force" in sys.argv):
        print(p)
