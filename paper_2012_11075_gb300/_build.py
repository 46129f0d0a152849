"""Build of the CUDA library ``libwblbe.so`` (sm_103a, C ABI of include/wblbe.h).

The library is built in-tree, next to this file, with plain nvcc; it links the
CUDA runtime statically and needs nothing from PyTorch.
"""
from __future__ import annotations

import os
import platform
import subprocess
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
LIB_DIR = PKG / "_lib"
LIB_PATH = LIB_DIR / f"libwblbe_{platform.machine()}.so"
# the same sources built with -DWBLBE_DEBUG_BOUNDS (checked accesses, a debugging aid)
DEBUG_LIB_PATH = LIB_DIR / f"libwblbe_bounds_{platform.machine()}.so"
SOURCES = [CSRC / "batch.cu", CSRC / "wblbe.cu", CSRC / "strip_variants.cu",
           CSRC / "wblbe_noalloc.cu", CSRC / "probe.cu", CSRC / "slabs.cu", CSRC / "d3q19.cu"]
DEPENDS = SOURCES + [CSRC / "lbm_kernels.cuh", CSRC / "strip_launch.cuh",
                     ROOT / "include" / "wblbe.h"]

NVCC_FLAGS = [
    "-gencode", "arch=compute_103a,code=sm_103a",
    "-O3", "-lineinfo", "-std=c++17",
    "-Xcompiler", "-fPIC",
    "--expt-relaxed-constexpr",
]


def nvcc() -> str:
    cand = os.environ.get("NVCC") or "/usr/local/cuda/bin/nvcc"
    return cand if os.path.exists(cand) else "nvcc"


def needs_build(target: Path = LIB_PATH) -> bool:
    if not target.exists():
        return True
    t = target.stat().st_mtime
    return any(p.stat().st_mtime > t for p in DEPENDS if p.exists())


def build(force: bool = False, verbose: bool = False, extra_flags=(),
          debug_bounds: bool = False) -> Path:
    """Compile libwblbe.so if it is missing or older than its sources.
    ``debug_bounds`` builds the bounds-checked variant instead (its own file)."""
    target = DEBUG_LIB_PATH if debug_bounds else LIB_PATH
    if debug_bounds:
        extra_flags = (*extra_flags, "-DWBLBE_DEBUG_BOUNDS")
    if not force and not needs_build(target):
        return target
    from concurrent.futures import ThreadPoolExecutor
    LIB_DIR.mkdir(exist_ok=True)
    obj_dir = LIB_DIR / f"obj_{platform.machine()}"
    obj_dir.mkdir(exist_ok=True)
    tag = os.getpid()
    objs = [obj_dir / f"{src.stem}.{tag}{'.bounds' if debug_bounds else ''}.o"
            for src in SOURCES]

    def compile_one(src, obj):
        cmd = [nvcc(), *NVCC_FLAGS, *extra_flags, "-c", "-o", str(obj), str(src)]
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.check_call(cmd)

    # the translation units compile in parallel, then one link
    with ThreadPoolExecutor(len(SOURCES)) as ex:
        for j in [ex.submit(compile_one, s, o) for s, o in zip(SOURCES, objs)]:
            j.result()
    tmp = target.with_suffix(f".{tag}.tmp")
    cmd = [nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-shared",
           "-o", str(tmp), *map(str, objs)]
    if verbose:
        print(" ".join(cmd), flush=True)
    subprocess.check_call(cmd)
    for o in objs:
        o.unlink()
    os.replace(tmp, target)
    return target
