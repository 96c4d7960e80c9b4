"""Builds libqmcfft.so in-tree for sm_103a with nvcc (no torch extension,
no cmake): every .cu under csrc/ is compiled in parallel, then linked into
one shared library exporting the C ABI of include/qmc.h."""

from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT_DIR = os.path.join(PKG, "_lib")
BUILD_DIR = os.path.join(ROOT, "_build")
LIB_NAME = "libqmcfft.so"
# the same sources with every table index checked in the kernels
# (-DQMC_CHECK_BOUNDS: out-of-range indices latch QMC_ERR_BOUNDS)
CHECKED_LIB_NAME = "libqmcfft_checked.so"
CHECKED_BUILD_DIR = os.path.join(ROOT, "_build_checked")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    exe = shutil.which("nvcc")
    if exe:
        return exe
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found")


def sources() -> list[str]:
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def lib_path(checked: bool = False) -> str:
    return os.path.join(OUT_DIR, CHECKED_LIB_NAME if checked else LIB_NAME)


def _newest_input() -> float:
    paths = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    inc = os.path.join(ROOT, "include")
    paths.extend(os.path.join(inc, h) for h in os.listdir(inc))
    return max(os.path.getmtime(p) for p in paths)


def build(force: bool = False, verbose: bool = False, extra_flags: list[str] | None = None,
          checked: bool = False) -> str:
    """Compiles and links the library (the bounds-checked variant with
    checked=True); skipped when it is newer than every source."""
    out = lib_path(checked)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= _newest_input():
        return out
    bdir = CHECKED_BUILD_DIR if checked else BUILD_DIR
    os.makedirs(bdir, exist_ok=True)
    os.makedirs(OUT_DIR, exist_ok=True)
    exe = nvcc()
    extra = list(extra_flags or []) + (["-DQMC_CHECK_BOUNDS"] if checked else [])

    def compile_one(src: str) -> str:
        obj = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
        cmd = [exe, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{res.stderr}")
        if verbose and res.stderr:
            sys.stderr.write(res.stderr)
        return obj

    srcs = sources()
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = out + ".tmp"
    cmd = [exe, *ARCH, "-shared", "-o", tmp, *objs]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stderr}")
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, checked="--checked" in sys.argv))
