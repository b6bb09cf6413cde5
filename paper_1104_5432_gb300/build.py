"""In-tree build of the CUDA library ``libsu2gb300.so`` for sm_103a.

Each translation unit is compiled by nvcc in parallel, then linked into one
shared library with a plain C ABI (``include/su2.h``).  No PyTorch headers
are involved.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libsu2gb300.so")
SOURCES = ["heatbath.cu", "observables.cu", "links.cu", "api.cu", "plaquette_static.cu",
           "selftest.cu", "cluster.cu"]
# heatbath_shapes.cu once per pair of launch shapes and row of the 14-entry
# table in csrc/su2_internal.h (FP32, FP64, FP32 site pairs): (object name,
# defines, flags).
# The FP32 phase kernels flush denormals to zero: none can occur on their
# path (links, staple sums and uniforms are >= 2^-24 in magnitude or exactly
# 0, the log series is evaluated in Horner form, alpha and 1/(2 alpha) stay
# normal down to beta = 1e-9), and without denormal handling the division
# and square-root sequences are shorter (2% at 64^4).
ROW_NAMES = ("f32", "f64", "f32pairs")
SHAPE_UNITS = [(f"heatbath_shapes_{ROW_NAMES[row]}_{k}",
                (f"SU2_ROW={row}", f"SU2_FIRST={k}"), ("-ftz=true",) if row != 1 else ())
               for row in (0, 1, 2) for k in range(0, 14, 2)]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                   "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC, *extra]


def _deps_mtime() -> float:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files += [os.path.join(INCLUDE, h) for h in os.listdir(INCLUDE)]
    files.append(os.path.abspath(__file__))
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False,
          defines=(), lib_path: str = LIB, build_dir: str = BUILD) -> str:
    """Compile to lib_path; `defines` are extra -D tuning macros (SU2_TPB,
    SU2_HB_MIN_BLOCKS) for building variants side by side."""
    if not force and os.path.exists(lib_path) and os.path.getmtime(lib_path) >= _deps_mtime():
        return lib_path
    os.makedirs(build_dir, exist_ok=True)
    cc = nvcc()
    extra = ["-Xptxas", "-v"] if ptxas_info else []
    extra += [f"-D{d}" for d in defines]

    units = [(src, src.replace(".cu", ""), (), ()) for src in SOURCES]
    units += [("heatbath_shapes.cu", name, defs, fl) for name, defs, fl in SHAPE_UNITS]

    def one(unit):
        src, name, defs, fl = unit
        obj = os.path.join(build_dir, name + ".o")
        cmd = [cc, *flags(extra + list(fl) + [f"-D{d}" for d in defs]), "-c",
               os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {name}:\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=min(len(units), os.cpu_count() or 8)) as ex:
        results = list(ex.map(one, units))
    if verbose or ptxas_info:
        for _, err in results:
            if err:
                sys.stderr.write(err)
    tmp = lib_path + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *[o for o, _ in results]]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv)
    print(LIB)
