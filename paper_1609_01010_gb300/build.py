"""Builds libpolymul.so (the C-ABI CUDA library) in place with nvcc for sm_103a.

Each translation unit under csrc/ is compiled in parallel to _build/*.o and
linked into paper_1609_01010_gb300/libpolymul.so (CUDA runtime linked
statically).  Rebuilds only what changed.  With --debug it builds
libpolymul_debug.so instead (objects in _build_debug/): the kernels'
range and index checks compiled in.  Usage: python -m
paper_1609_01010_gb300.build [--force] [--debug].
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
BUILD = os.path.join(PKG, "_build")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libpolymul.so")
LIB_DEBUG = os.path.join(PKG, "libpolymul_debug.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
         f"-I{INCLUDE}", f"-I{CSRC}"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpolymul.so")


def _deps() -> list[str]:
    return glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        [os.path.join(INCLUDE, "polymul.h")]


def _stale(target: str, sources: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in sources)


# Sources compiled once per variant (preprocessor defines), so their many
# template instantiations build in parallel.
def _variants() -> dict[str, list[tuple[str, list[str]]]]:
    cols = []
    for fwd in (1, 0):
        for lazy in (1, 0):
            for c in (8, 128):  # 32-column tiles run the TMA-fed kernels of k_cols_tma.cu
                name = f"launch_col{'f' if fwd else 'i'}_{'lazy' if lazy else 'strict'}_c{c}"
                cols.append((name, [f"-DPM_FWD={fwd}", f"-DPM_LAZY={lazy}", f"-DPM_C={c}", f"-DPM_COL_FN={name}"]))
    tcols = []
    for fwd in (1, 0):
        for lazy in (1, 0):
            name = f"launch_tcol{'f' if fwd else 'i'}_{'lazy' if lazy else 'strict'}"
            tcols.append((name, [f"-DPM_FWD={fwd}", f"-DPM_LAZY={lazy}", f"-DPM_TCOL_FN={name}"]))
    return {"k_cols.cu": cols, "k_cols_tma.cu": tcols}


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Builds libpolymul.so, or with debug=True libpolymul_debug.so: the same
    library with the kernels' range and index checks compiled in
    (PM_DEBUG_CHECKS; failures land in the device status word)."""
    build_dir = BUILD + ("_debug" if debug else "")
    lib_path = LIB_DEBUG if debug else LIB
    extra = ["-DPM_DEBUG_CHECKS=1"] if debug else []
    os.makedirs(build_dir, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    deps = _deps()
    cc = nvcc()
    variants = _variants()
    jobs = []
    objs = []
    for src in srcs:
        base = os.path.basename(src)[:-3]
        for tag, defs in variants.get(os.path.basename(src), [(None, [])]):
            obj = os.path.join(build_dir, base + (f".{tag}" if tag else "") + ".o")
            objs.append(obj)
            if force or _stale(obj, [src] + deps):
                jobs.append([cc, *ARCH, *FLAGS, *extra, *defs, "-c", src, "-o", obj])
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            results = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs))
        for cmd, r in zip(jobs, results):
            if verbose or r.returncode:
                sys.stderr.write(r.stdout + r.stderr)
            if r.returncode:
                raise RuntimeError(f"nvcc failed ({r.returncode}): {' '.join(cmd)}")
    if force or jobs or _stale(lib_path, objs):
        tmp = lib_path + f".tmp{os.getpid()}"
        cmd = [cc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs, "-lpthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError(f"link failed: {' '.join(cmd)}")
        os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, debug="--debug" in sys.argv))
