"""Build libqmc_gb300.so in-tree: every translation unit compiled for sm_103a
by its own nvcc process (in parallel), then linked into one shared library.

    python -m paper_1811_11722_gb300.build [--jobs N] [--force]
"""
from __future__ import annotations

import argparse
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
BUILD = os.path.join(ROOT, "_build", "qmc")
LIB = os.path.join(PKG, "libqmc_gb300.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", f"-I{INCLUDE}"]
SECTOR_DIMS = range(1, 9)


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found; the CUDA toolkit is required to build libqmc_gb300.so")


def _units():
    """(object name, source, extra flags) for every translation unit."""
    units = []
    for real in ("float", "double"):
        for d in SECTOR_DIMS:
            units.append((f"sector_{real}_{d}.o", "kernels_sector.cu", [f"-DQMC_REAL={real}", f"-DQMC_D={d}"]))
    for real in ("float", "double"):
        units.append((f"misc_{real}.o", "kernels_misc.cu", [f"-DQMC_REAL={real}"]))
    for d in SECTOR_DIMS:
        units.append((f"cv_{d}.o", "cv_inst.cu", [f"-DQMC_D={d}"]))
    for src in ("finalize.cu", "api.cu", "deformed.cu", "batch.cu", "cbc.cpp", "cv.cu", "noalloc.cu", "jit.cu", "probe.cu", "multi.cu", "persist.cu"):
        if os.path.exists(os.path.join(CSRC, src)):
            units.append((os.path.splitext(src)[0] + ".o", src, []))
    return units


def _deps_mtime() -> float:
    files = glob.glob(os.path.join(CSRC, "*")) + glob.glob(os.path.join(INCLUDE, "*.h"))
    return max(os.path.getmtime(f) for f in files)


def _compile(nvcc, obj, src, extra, verbose):
    out = os.path.join(BUILD, obj)
    cmd = [nvcc] + ARCH + NVCC_FLAGS + extra
    if src.endswith(".cpp"):
        # host-only unit; no FMA contraction so its floating point matches the
        # same expressions evaluated elsewhere term by term
        cmd += ["-x", "cu", "-Xcompiler", "-ffp-contract=off"]
    cmd += ["-c", os.path.join(CSRC, src), "-o", out]
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src} {' '.join(extra)}:\n{r.stderr[-4000:]}")
    return out


def build_library(jobs: int | None = None, force: bool = False, verbose: bool = False) -> str:
    """Compile and link the CUDA library; returns the .so path."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps_mtime():
        return LIB
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    units = _units()
    jobs = jobs or max(1, min(len(units), os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        objs = list(ex.map(lambda u: _compile(nvcc, u[0], u[1], u[2], verbose), units))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart", "-lnvrtc", "-ldl", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr[-4000:]}")
    os.replace(tmp, LIB)
    return LIB


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=None)
    ap.add_argument("--force", action="store_true")
    ap.add_argument("-v", "--verbose", action="store_true")
    a = ap.parse_args(argv)
    print(build_library(a.jobs, a.force, a.verbose))


if __name__ == "__main__":
    sys.exit(main())
