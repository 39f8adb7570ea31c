"""Builds libfpo.so (the CUDA library behind include/fpo.h) in-tree with nvcc.

Each translation unit is compiled for sm_103a only, in parallel, then linked
into paper_2202_08614_gb300/_build/libfpo.so.
"""

from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
SRC = os.path.join(PKG, "csrc")
OUT = os.path.join(PKG, "_build")
LIB = os.path.join(OUT, "libfpo.so")
SOURCES = ["fpo_api.cu", "fpo_kernels.cu", "fpo_pack.cpp", "fpo_noalloc.cu", "fpo_union.cpp", "fpo_latent.cu", "fpo_train.cu",
           "fpo_diag.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _inputs():
    deps = [os.path.join(SRC, f) for f in os.listdir(SRC)]
    deps.append(os.path.join(ROOT, "include", "fpo.h"))
    deps.append(os.path.abspath(__file__))
    return deps


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in _inputs())


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False,
          defines: tuple = (), lib: str | None = None) -> str:
    """Compiles libfpo.so.  `defines` (e.g. ("FPO_TRAV_MIN_BLOCKS=4",)) and
    `lib` (an output path) build tuning variants next to the default library."""
    target = lib or LIB
    if not force and not defines and lib is None and up_to_date():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    common = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]
    common += [f"-D{d}" for d in defines]
    tag = "" if lib is None else "_" + os.path.splitext(os.path.basename(lib))[0]
    if ptxas_info:
        common += ["-Xptxas", "-v"]

    def compile_one(src):
        obj = os.path.join(OUT, os.path.splitext(src)[0] + tag + ".o")
        cmd = [nvcc()] + ARCH + common + ["-c", os.path.join(SRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose:
        for _, log in results:
            if log.strip():
                print(log)
    tmp = target + f".tmp{os.getpid()}"
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + [o for o, _ in results]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stderr}")
    os.replace(tmp, target)
    return target


if __name__ == "__main__":
    import sys
    build(force="--force" in sys.argv, verbose=True, ptxas_info="-v" in sys.argv)
    print(LIB)
