"""Build libsr.so (the C ABI of include/sr.h) for sm_103a with nvcc.

Each .cu file under csrc/ is compiled on its own (in parallel) and the objects
are linked into paper_1807_07433_gb300/libsr.so.  Objects go to _build/ at the
repository root; both are git-ignored.  Rebuilds only what changed (by mtime
of the source and the headers).
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OBJ = os.path.join(ROOT, "_build", "sr")
LIB = os.path.join(PKG, "libsr.so")
# bounds-checked build (SR_BOUNDS_CHECK: checked indices, sr_bounds_report);
# built on request, not by build()
OBJ_CHECK = os.path.join(ROOT, "_build", "sr_check")
LIB_CHECK = os.path.join(PKG, "libsr_check.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "-I", INCLUDE, "-I", CSRC] + ARCH


def nvcc() -> str:
    cand = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found (set NVCC or put CUDA's bin on PATH)")
    return cand


def _headers_mtime() -> float:
    hs = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))
    return max((os.path.getmtime(h) for h in hs), default=0.0)


def _compile(src: str, obj: str, extra: list[str]) -> tuple[str, str]:
    cmd = [nvcc(), "-c", src, "-o", obj] + NVCC_FLAGS + extra
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stderr}")
    return src, r.stderr


def build(force: bool = False, verbose_ptxas: bool = False, jobs: int | None = None,
          check: bool = False) -> str:
    """Compile every translation unit under csrc/ and link libsr.so (with
    check=True: the bounds-checked libsr_check.so); return its path."""
    obj_dir, lib = (OBJ_CHECK, LIB_CHECK) if check else (OBJ, LIB)
    os.makedirs(obj_dir, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    hdr_t = _headers_mtime()
    todo, objs = [], []
    for s in srcs:
        o = os.path.join(obj_dir, os.path.splitext(os.path.basename(s))[0] + ".o")
        objs.append(o)
        if force or verbose_ptxas or not os.path.exists(o) or \
                os.path.getmtime(o) < max(os.path.getmtime(s), hdr_t):
            todo.append((s, o))
    extra = (["-Xptxas", "-v"] if verbose_ptxas else []) + (["-DSR_BOUNDS_CHECK"] if check else [])
    logs = []
    if todo:
        n = jobs or min(len(todo), os.cpu_count() or 4)
        with cf.ThreadPoolExecutor(max_workers=n) as ex:
            for src, err in ex.map(lambda so: _compile(so[0], so[1], extra), todo):
                logs.append((src, err))
    if verbose_ptxas:
        for src, err in logs:
            sys.stderr.write(f"== {os.path.basename(src)}\n{err}")
    if todo or not os.path.exists(lib):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc(), "-shared", "-o", tmp] + objs + ARCH + ["-Xcompiler", "-fPIC"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv,
                check="--check" in sys.argv))
