"""Build the CUDA library ``libopmos.so`` in-tree for sm_103a (GB300).

Each translation unit under ``csrc/`` is compiled by nvcc in parallel, then
linked into one shared library whose exported symbols are exactly the C ABI
of ``include/opmos.h``. The search kernels (``search_inst.cu``) are compiled
once per group of objective counts, so the 16 instantiations build side by
side.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libopmos.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "-I", INCLUDE, "-I", CSRC]


# one object per objective count: its single-query kernels (both grid
# shapes) and its multi-query kernel, the objects compiled side by side
D_GROUPS = tuple((d, d) for d in range(1, 17))
INST = "search_inst.cu"


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def units():
    """(source, extra flags, object name) for every object of the library."""
    out = []
    for src in sources():
        name = os.path.basename(src)
        if name == INST:
            for a, b in D_GROUPS:
                out.append((src, [f"-DOPMOS_D_FIRST={a}", f"-DOPMOS_D_LAST={b}"], f"{name}.d{a}_{b}.o"))
        else:
            out.append((src, [], name + ".o"))
    return out


def _deps_mtime():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    return max(os.path.getmtime(f) for f in files)


def _compile(src: str, extra: list[str], objname: str) -> str:
    obj = os.path.join(BUILD, objname)
    cmd = [NVCC, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    """Compile and link; returns the library path. Skips work when up to date."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps_mtime() and not verbose_ptxas:
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    extra = ["-Xptxas", "-v"] if verbose_ptxas else []
    jobs = units()
    # the instantiation groups first: they are the long ones
    jobs.sort(key=lambda u: os.path.basename(u[0]) != INST)
    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda u: _compile(u[0], extra + u[1], u[2]), jobs))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose_ptxas="-v" in sys.argv))
