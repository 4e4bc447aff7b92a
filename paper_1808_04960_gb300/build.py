"""Build the in-tree CUDA library ``libgpweno.so`` for sm_103a.

Every translation unit is compiled in parallel with nvcc (one -gencode,
sm_103a only), then linked into a shared library next to this file.  A
rebuild happens only when a source or header is newer than the library.

``build(checked=True)`` builds ``libgpweno_checked.so`` instead, with
-DGPWENO_CHECKED: the stage kernels check every shared-memory and global
access against its array's extent and record a violation in the plan's
flag word (bit = access site) instead of making it.  The tests build and
use it; the product path loads ``libgpweno.so``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libgpweno.so")
OUT_DIR_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(HERE, "libgpweno_checked.so")
SOURCES = ["api.cu", "stage_f32.cu", "stage_f64.cu", "gp_precompute.cpp", "noalloc.cu", "batch_f32.cu",
           "batch_f64.cu"] + ["stage_%s_var%d.cu" % (t, v) for t in ("f32", "f64") for v in (1, 2, 3, 4, 5, 8)]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgpweno")
    return cand


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(ROOT, "include", "gpweno.h"))
    return files


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    lib, out_dir = (LIB_CHECKED, OUT_DIR_CHECKED) if checked else (LIB, OUT_DIR)
    deps = _deps()
    if not force and not _stale(lib, deps):
        return lib
    os.makedirs(out_dir, exist_ok=True)
    nvcc = _nvcc()
    common = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]
    if checked:
        common.append("-DGPWENO_CHECKED")

    def compile_one(src):
        obj = os.path.join(out_dir, src + ".o")
        path = os.path.join(CSRC, src)
        if src.endswith(".cu"):
            cmd = [nvcc, *ARCH, *common, "-Xptxas", "-v" if verbose else "-O3", "-c", path, "-o", obj]
        else:
            cmd = [nvcc, *common, "-Xcompiler", "-ffp-contract=off", "-c", path, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose:
        for _, log in results:
            print(log)
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *[o for o, _ in results], "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, checked="--checked" in sys.argv))
