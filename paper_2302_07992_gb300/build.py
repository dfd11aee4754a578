"""Build the sm_103a shared library ``_build/librdhei.so`` from ``csrc/*.cu``.

Plain nvcc, one ``-gencode`` (compute_103a / sm_103a), translation units compiled in
parallel, then linked with ``-shared``.  Nothing is installed outside this folder.

``build(checked=True)`` makes the checked library ``_build/librdhei_check.so``
(``-DRDHEI_CHECK``: device index checks that report ``RDHEI_EBOUNDS`` instead of
touching memory out of range); ``rdhei`` loads it when ``RDHEI_CHECKED=1``.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "librdhei.so")
LIB_CHECKED = os.path.join(OUT, "librdhei_check.so")
GENCODE = "arch=compute_103a,code=sm_103a"


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources():
    return sorted(glob.glob(os.path.join(SRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(SRC, "*.cuh")) + [os.path.join(HERE, "..", "include", "rdhei.h")]


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None,
          checked: bool = False) -> str:
    lib = LIB_CHECKED if checked else LIB
    if not force and up_to_date(lib):
        return lib
    objdir = os.path.join(OUT, "check") if checked else OUT
    os.makedirs(objdir, exist_ok=True)
    nv = nvcc()
    flags = ["-gencode", GENCODE, "-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xptxas", "-v"]
    flags += ["-DRDHEI_CHECK"] if checked else []
    flags += list(extra or [])
    objs = []

    def one(src):
        obj = os.path.join(objdir, os.path.basename(src)[:-3] + ".o")
        cmd = [nv] + flags + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
        for obj, log in ex.map(one, _sources()):
            objs.append(obj)
            if verbose:
                sys.stderr.write(log)
    tmp = lib + f".{os.getpid()}.tmp"
    cmd = [nv, "-shared", "-gencode", GENCODE, "-cudart", "static", "-o", tmp] + objs + ["-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, checked="--checked" in sys.argv))
