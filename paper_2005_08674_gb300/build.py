"""Build the sm_103a CUDA library ``liblbm.so`` in-tree with nvcc.

Every translation unit under ``csrc/`` is compiled in parallel for
``-gencode arch=compute_103a,code=sm_103a`` and linked into one shared
library next to this file.  ``python -m paper_2005_08674_gb300.build``
does the same from the command line.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "liblbm.so")
BUILD_DIR = os.path.join(HERE, "_build")
# bounds-checked build (-DLBM_CHECK): every step-kernel access checked against
# the registered buffers, failures counted instead of made (lbm_check_read)
LIB_CHECK = os.path.join(HERE, "liblbm_check.so")
BUILD_DIR_CHECK = os.path.join(BUILD_DIR, "check")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblbm.so")
    return p


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = (_sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
            + glob.glob(os.path.join(INCLUDE, "*.h")))
    return any(os.path.getmtime(d) > t for d in deps)


def build_id() -> str:
    """Hash of the library's sources: part of the autotuner cache's key, so
    that choices recorded by another build of the kernels are not reused."""
    h = hashlib.sha256()
    for path in sorted(glob.glob(os.path.join(CSRC, "*")) + glob.glob(os.path.join(INCLUDE, "*.h"))):
        if path.endswith((".cu", ".cuh", ".h")):
            h.update(os.path.basename(path).encode())
            with open(path, "rb") as f:
                h.update(f.read())
    return h.hexdigest()[:16]


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False, check: bool = False) -> str:
    """Build liblbm.so (or, with check=True, the bounds-checked liblbm_check.so)."""
    lib, bdir = (LIB_CHECK, BUILD_DIR_CHECK) if check else (LIB, BUILD_DIR)
    if not force and not _stale(lib):
        return lib
    os.makedirs(bdir, exist_ok=True)
    cc = nvcc()
    # the checked build is a test instrument: its device code goes through the
    # NVVM optimiser at -O1 (ptxas keeps -O3), which cuts its compile time about
    # threefold; the ordinary library is built at full optimisation
    extra = (["-Xptxas", "-v"] if ptxas_info else []) + (["-DLBM_CHECK", "-Xcicc", "-O1"] if check else [])
    extra += [f"-DLBM_BUILD_ID=\"{build_id()}{'-check' if check else ''}\""]

    def compile_one(src):
        obj = os.path.join(bdir, os.path.basename(src) + ".o")
        cmd = [cc, *ARCH, *FLAGS, *extra, "-I", INCLUDE, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        if verbose or ptxas_info:
            sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        objs = list(ex.map(compile_one, _sources()))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv,
                check="--check" in sys.argv))
