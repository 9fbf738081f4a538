"""Builds the package's native code in-tree.

librelo.so: the sm_103a CUDA library behind include/relo.h (nvcc, one -gencode, translation
units compiled in parallel, static CUDA runtime).  _scene_sampler.so: the seeded input
generator's C helper (gcc).  Both are git-ignored build products.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "librelo.so")
CHECKED_LIB = os.path.join(HERE, "librelo_checked.so")
SOURCES = ["scene.cu", "forest.cu", "ransac.cu", "regressor.cu", "conv_tc.cu", "api.cu", "server.cu", "posegraph.cu",
           "fusion.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]
# occupancy bounds of the raycast, forest and hypothesis-search kernels (tuning knobs; the defaults come from sweeps)
NVCC_FLAGS += [f"-D{k}={os.environ[k]}" for k in ("RELO_RAYCAST_MIN_BLOCKS", "RELO_RAYCAST_COLOUR_MIN_BLOCKS",
                                                  "RELO_SEARCH_MIN_BLOCKS", "RELO_FOREST_MIN_BLOCKS",
                                                  "RELO_REFINE_MIN_BLOCKS", "RELO_FEW_HYPS",
                                                  "RELO_REFINE_FEW_MIN_BLOCKS", "RELO_ENERGY_MIN_BLOCKS")
               if k in os.environ]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _stale(out: str, deps: list[str]) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build_cuda(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """librelo.so; with checked=True the bounds-checked variant librelo_checked.so (RELO_CHECKED:
    guarded accesses count their failed index checks, relo_debug_check_failures)."""
    hdrs = [os.path.join(CSRC, "relo_internal.cuh"), os.path.join(CSRC, "regressor.cuh"), os.path.join(ROOT, "include", "relo.h")]
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    bdir = os.path.join(ROOT, "_build", "relo_checked" if checked else "relo")
    lib_path = CHECKED_LIB if checked else LIB
    nvcc_flags = NVCC_FLAGS + (["-DRELO_CHECKED=1"] if checked else [])
    # the objects depend on the compile flags too: a change of flags rebuilds everything
    stamp = os.path.join(bdir, "flags")
    flags = " ".join(nvcc_flags)
    try:
        with open(stamp) as f:
            force = force or f.read() != flags
    except OSError:
        force = True
    if not force and not _stale(lib_path, srcs + hdrs):
        return lib_path
    os.makedirs(bdir, exist_ok=True)
    nvcc = _nvcc()
    procs, objs = [], []
    for s in srcs:
        o = os.path.join(bdir, os.path.basename(s).replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + hdrs):
            cmd = [nvcc] + nvcc_flags + ["-c", s, "-o", o]
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError("nvcc failed: " + " ".join(cmd) + "\n" + out.decode(errors="replace"))
    tmp = lib_path + f".tmp{os.getpid()}"
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs
    subprocess.check_call(cmd)
    os.replace(tmp, lib_path)
    with open(stamp, "w") as f:
        f.write(flags)
    return lib_path


def build(force: bool = False, verbose: bool = False) -> None:
    from .synth import build as build_synth
    build_cuda(force=force, verbose=verbose)
    build_synth(force=force)


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
