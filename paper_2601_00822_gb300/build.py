"""Builds libbfcs.so (the C-ABI library) in-tree with nvcc for sm_103a.

Each translation unit is compiled in parallel; the per-precision kernel files
are compiled per arithmetic type (BFCS_R = float / double, and ff = float-float
for the FFT and defect kernels of the precision ladder).  No cmake, no torch headers.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_build")
LIB_PATH = os.path.join(OUT_DIR, "libbfcs.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2", "--expt-relaxed-constexpr",
         "-I" + INCLUDE, "-I" + CSRC]

# (source, extra defines, object name)
UNITS = [
    ("k_fft.cu", ["-DBFCS_R=float"], "k_fft_f32.o"),
    ("k_fft.cu", ["-DBFCS_R=double"], "k_fft_f64.o"),
    ("k_green.cu", ["-DBFCS_R=float"], "k_green_f32.o"),
    ("k_green.cu", ["-DBFCS_R=double"], "k_green_f64.o"),
    ("k_fft.cu", ["-DBFCS_R=ff"], "k_fft_ff.o"),
    ("k_green.cu", ["-DBFCS_R=ff", "-DBFCS_FF"], "k_green_ff.o"),
    ("k_cg.cu", ["-DBFCS_R=float"], "k_cg_f32.o"),
    ("k_cg.cu", ["-DBFCS_R=double"], "k_cg_f64.o"),
    ("k_cd.cu", ["-DBFCS_R=float"], "k_cd_f32.o"),
    ("k_cd.cu", ["-DBFCS_R=double"], "k_cd_f64.o"),
    ("k_misc.cu", [], "k_misc.o"),
    ("rve.cu", [], "rve.o"),
    ("k_nonlocal.cu", [], "k_nonlocal.o"),
    ("solver.cu", [], "solver.o"),
    ("noalloc.cu", [], "noalloc.o"),
    ("unet.cu", [], "unet.o"),
]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources_digest() -> str:
    h = hashlib.sha256()
    for d in (CSRC, INCLUDE):
        for name in sorted(os.listdir(d)):
            if name.endswith((".cu", ".cuh", ".h")):
                with open(os.path.join(d, name), "rb") as f:
                    h.update(name.encode() + f.read())
    h.update(" ".join(ARCH + FLAGS).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False, jobs: int | None = None) -> str:
    """Compile (if sources changed) and return the path of libbfcs.so."""
    os.makedirs(OUT_DIR, exist_ok=True)
    stamp = os.path.join(OUT_DIR, "stamp.txt")
    digest = _sources_digest()
    if not force and os.path.exists(LIB_PATH) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == digest:
                return LIB_PATH
    cc = nvcc()

    def compile_unit(u):
        src, defs, obj = u
        cmd = [cc, *ARCH, *FLAGS, *defs, "-c", os.path.join(CSRC, src), "-o", os.path.join(OUT_DIR, obj)]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src} {defs}:\n{r.stderr}")
        return r.stderr

    with cf.ThreadPoolExecutor(max_workers=jobs or min(len(UNITS), os.cpu_count() or 4)) as ex:
        for msg in ex.map(compile_unit, UNITS):
            if verbose and msg:
                print(msg, file=sys.stderr)
    objs = [os.path.join(OUT_DIR, u[2]) for u in UNITS]
    tmp = LIB_PATH + ".tmp"
    r = subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB_PATH)
    with open(stamp, "w") as f:
        f.write(digest)
    return LIB_PATH


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
