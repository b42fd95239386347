"""Builds the gbdart shared libraries in-tree with nvcc for sm_103a.

Two variants are built from the same sources:
  _build/libgbdart.so          the production library
  _build/libgbdart_checked.so  compiled with -DGBD_CHECKED: every gather
                               checks its cell and epoch index and records a
                               violation in an error word instead of loading

Translation units are compiled in parallel, each with one -gencode.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
SOURCES = ["api.cpp", "runtime.cpp", "serve.cpp", "tune.cpp", "stream.cpp", "march.cu", "pack.cu", "noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the gbdart library needs the CUDA toolkit to build")


def lib_path(checked: bool = False) -> str:
    return os.path.join(BUILD, "libgbdart_checked.so" if checked else "libgbdart.so")


def _sources():
    return [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]


def _deps_mtime() -> float:
    paths = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "gbdart.h"), __file__]
    return max(os.path.getmtime(p) for p in paths if os.path.exists(p))


def _compile(src: str, obj: str, defines: list[str], verbose_ptxas: bool) -> tuple[str, str]:
    cmd = [nvcc(), *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE,
           *defines, "-c", os.path.join(CSRC, src), "-o", obj]
    if verbose_ptxas and src.endswith(".cu"):
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    return src, r.stderr


def build(force: bool = False, checked: bool | None = None, verbose_ptxas: bool = False, jobs: int = 0) -> list[str]:
    """Compile the libraries; returns their paths.  ``checked=None`` builds
    both variants."""
    os.makedirs(BUILD, exist_ok=True)
    variants = [False, True] if checked is None else [checked]
    todo = []
    for chk in variants:
        out = lib_path(chk)
        if force or not os.path.exists(out) or os.path.getmtime(out) < _deps_mtime():
            todo.append(chk)
    logs = {}
    if todo:
        jobs = jobs or min(16, (os.cpu_count() or 4))
        with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
            futs = []
            for chk in todo:
                tag = "chk" if chk else "rel"
                defines = ["-DGBD_CHECKED"] if chk else []
                for src in _sources():
                    obj = os.path.join(BUILD, f"{tag}_{os.path.splitext(src)[0]}.o")
                    futs.append(ex.submit(_compile, src, obj, defines, verbose_ptxas))
            for f in futs:
                src, log = f.result()
                if log.strip():
                    logs[src] = log
        for chk in todo:
            tag = "chk" if chk else "rel"
            objs = [os.path.join(BUILD, f"{tag}_{os.path.splitext(s)[0]}.o") for s in _sources()]
            tmp = lib_path(chk) + f".tmp{os.getpid()}"
            cmd = [nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
            os.replace(tmp, lib_path(chk))
    if verbose_ptxas:
        for src, log in logs.items():
            print(f"--- {src}\n{log}")
    return [lib_path(c) for c in variants]


if __name__ == "__main__":
    import sys
    print("\n".join(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv)))
