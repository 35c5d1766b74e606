"""Compile the CUDA library ``libfg_lattice.so`` in-tree for sm_103a.

Each translation unit under ``csrc/`` is compiled by nvcc in parallel into
``_build/`` and linked into ``paper_0910_2950_gb300/libfg_lattice.so``.  No
CMake and no torch extension machinery: the library exposes a plain C ABI
(``include/fg_lattice.h``) and links only the CUDA runtime.

    python -m paper_0910_2950_gb300.build [--verbose-ptxas]
"""

from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libfg_lattice.so")
SOURCES = ["fg_lattice.cu", "backend.cu", "gauge.cu", "fermion.cu", "batch.cu", "noalloc.cu", "forcegrad.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_path() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libfg_lattice.so")


def _flags(verbose_ptxas: bool) -> list:
    f = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2", "--expt-relaxed-constexpr",
         "-I", os.path.join(ROOT, "include")] + ARCH
    if verbose_ptxas:
        f += ["-Xptxas", "-v"]
    return f


def _compile(nvcc, src, obj, verbose_ptxas, extra=()):
    cmd = [nvcc, "-c", os.path.join(CSRC, src), "-o", obj] + _flags(verbose_ptxas) + list(extra)
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{res.stdout}\n{res.stderr}")
    return res.stdout + res.stderr


def _stale(objs) -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [
        os.path.join(ROOT, "include", "fg_lattice.h"), os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose_ptxas: bool = False, quiet: bool = True,
          extra_flags=(), out: str = None) -> str:
    """Build (if stale) and return the path of libfg_lattice.so.

    `extra_flags` are appended to every nvcc compile (e.g. -D tuning macros)
    and `out` writes the library elsewhere (both imply a fresh build).
    """
    lib = out or LIB
    bdir = BUILD if out is None else os.path.join(os.path.dirname(os.path.abspath(out)), "_build")
    os.makedirs(bdir, exist_ok=True)
    sources = [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]
    objs = [os.path.join(bdir, os.path.splitext(s)[0] + ".o") for s in sources]
    if not force and not verbose_ptxas and not extra_flags and out is None and not _stale(objs):
        return LIB
    nvcc = nvcc_path()
    with cf.ThreadPoolExecutor(max_workers=len(sources)) as ex:
        logs = list(ex.map(lambda so: _compile(nvcc, so[0], so[1], verbose_ptxas, extra_flags),
                           zip(sources, objs)))
    tmp = lib + ".tmp"
    cmd = [nvcc, "-shared", "-o", tmp] + objs + ARCH + ["-cudart=static"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, lib)
    if not quiet or verbose_ptxas:
        for log in logs:
            if log.strip():
                print(log, file=sys.stderr)
    return lib


if __name__ == "__main__":
    path = build(force=True, verbose_ptxas="--verbose-ptxas" in sys.argv, quiet=False)
    print(path)
