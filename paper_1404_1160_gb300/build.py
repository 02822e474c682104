"""Builds libpic.so (the CUDA library) in-tree with nvcc for sm_103a.

Each translation unit compiles in parallel; the link step produces
``paper_1404_1160_gb300/libpic.so``.  FP contraction is off (--fmad=false):
the kernels write every fused multiply-add explicitly.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libpic.so")
SOURCES = ["api.cu", "mesh.cu", "window.cu", "window32.cu", "sort.cu", "mlp.cu"]
# window_coop.cu compiles once per (histogram form, fine solver): its kernel
# instantiations build in parallel
VARIANTS = [("window_coop.cu", f"window_coop_h{h}_s{s}", [f"-DPIC_WINDOW_HIST={h}", f"-DPIC_WINDOW_SOLVER={s}"])
            for h in (0, 1, 2) for s in (0, 1)]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpic.so")


def _flags():
    return ARCH + [
        "-O3", "-lineinfo", "-std=c++17", "--fmad=false", "-Xcompiler", "-fPIC,-ffp-contract=off",
        "-I", os.path.join(ROOT, "include"), "-I", CSRC,
    ]


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(ROOT, "include", "pic.h"))
    objs = []
    jobs = []
    units = [(src, src.replace(".cu", ""), []) for src in SOURCES] + VARIANTS
    for src, name, defs in units:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, name + ".o")
        objs.append(o)
        if force or _stale(o, [s] + headers):
            jobs.append([nvcc(), *_flags(), *defs, *(extra or []), "-c", s, "-o", o])
    if jobs:
        with cf.ThreadPoolExecutor(len(jobs)) as ex:
            res = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs))
        for cmd, r in zip(jobs, res):
            if verbose or r.returncode:
                print(" ".join(cmd))
                print(r.stdout, r.stderr)
            if r.returncode:
                raise RuntimeError(f"nvcc failed for {cmd[-3]}")
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + f".{os.getpid()}.tmp"
        link = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static"]
        r = subprocess.run(link, capture_output=True, text=True)
        if r.returncode:
            print(" ".join(link))
            print(r.stdout, r.stderr)
            raise RuntimeError("link of libpic.so failed")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys

    print(build(force="--force" in sys.argv, verbose=True))
