"""Build libzm.so (the CUDA C-ABI library) in-tree for sm_103a.

Each translation unit under csrc/ is compiled in parallel with nvcc into _build/, then linked
into paper_2406_05490_gb300/_lib/libzm.so.  The checked build of the same sources (-DZM_CHECKS=1:
kernels test their computed indices and count violations instead of accessing out of range)
goes through _build_checked/ into _lib/libzm_checked.so, in the same pool of compile jobs.
Rebuilds only what changed (source or header newer than its object).
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OBJDIR = os.path.join(PKG, "_build")
OBJDIR_CHECKED = os.path.join(PKG, "_build_checked")
LIBDIR = os.path.join(PKG, "_lib")
LIB = os.path.join(LIBDIR, "libzm.so")
LIB_CHECKED = os.path.join(LIBDIR, "libzm_checked.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _headers():
    return glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))


def _compile(src: str, verbose_ptxas: bool, checked: bool = False) -> str:
    obj = os.path.join(OBJDIR_CHECKED if checked else OBJDIR, os.path.basename(src) + ".o")
    newest = max([os.path.getmtime(src)] + [os.path.getmtime(h) for h in _headers()])
    if os.path.exists(obj) and os.path.getmtime(obj) >= newest and not verbose_ptxas:
        return obj
    flags = NVCC_FLAGS + (["-DZM_CHECKS=1"] if checked else [])
    cmd = [_nvcc(), *ARCH, *flags, "-c", src, "-o", obj + ".tmp"]
    if src.endswith(".cpp"):
        cmd = [_nvcc(), *flags, "-x", "c++", "-c", src, "-o", obj + ".tmp"]
    if verbose_ptxas:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if verbose_ptxas and r.stderr:
        sys.stderr.write(r.stderr)
    os.replace(obj + ".tmp", obj)
    return obj


def _link(lib: str, objs) -> None:
    if not os.path.exists(lib) or os.path.getmtime(lib) < max(os.path.getmtime(o) for o in objs):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [_nvcc(), *ARCH, "-shared", "-o", tmp, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)


def build(verbose_ptxas: bool = False, checked: bool = True) -> str:
    """Build libzm.so (and, unless checked=False, libzm_checked.so); returns libzm.so's path."""
    for d in (OBJDIR, OBJDIR_CHECKED, LIBDIR):
        os.makedirs(d, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))
    jobs = [(s, False) for s in srcs] + ([(s, True) for s in srcs] if checked else [])
    # the slowest units first, so that the pool's tail is short
    jobs.sort(key=lambda j: -os.path.getsize(j[0]))
    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda j: (j[1], _compile(j[0], verbose_ptxas and not j[1], j[1])), jobs))
    _link(LIB, sorted(o for c, o in objs if not c))
    if checked:
        _link(LIB_CHECKED, sorted(o for c, o in objs if c))
    return LIB


if __name__ == "__main__":
    print(build(verbose_ptxas="-v" in sys.argv))
