"""Build libmck.so in-tree with nvcc for sm_103a (GB300).

Each translation unit under csrc/ compiles in parallel into _build/, then
they link into paper_1702_08159_gb300/libmck.so (CUDA runtime linked
statically, so the library loads without a GPU). Up-to-date objects are
reused. Run directly (``python -m paper_1702_08159_gb300.build [-v]``) or via
``__graft_entry__.build()``.
"""

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libmck.so")
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE,
          "--expt-relaxed-constexpr"]
# Per-file extra flags. plan.cu evaluates float64 formulas exactly as written
# (no fused multiply-add contraction) so its tables round like a plain IEEE
# float64 evaluation.
EXTRA = {"plan.cu": ["--fmad=false"]}
SOURCES = ["api.cu", "plan.cu", "fwht.cu", "fwht_mma.cu", "features.cu", "features_mma.cu",
           "chunks.cu", "large.cu", "train.cu", "grouped.cu"]


def nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmck.so")
    return exe


def _deps_mtime():
    paths = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "mck.h")]
    return max(os.path.getmtime(p) for p in paths) if paths else 0.0


def _compile(src, verbose):
    obj = os.path.join(BUILD, src.replace(".cu", ".o"))
    if os.path.exists(obj) and os.path.getmtime(obj) >= _deps_mtime():
        return obj, ""
    cmd = [nvcc(), *ARCH, *COMMON, *EXTRA.get(src, []), "-c", os.path.join(CSRC, src), "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
    return obj, r.stderr


def build(verbose=False, force=False):
    """Compile and link libmck.so; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    if force:
        for f in os.listdir(BUILD):
            os.remove(os.path.join(BUILD, f))
    if (not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps_mtime()):
        return LIB
    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(lambda s: _compile(s, verbose), SOURCES))
    if verbose:
        for _, log in results:
            if log:
                sys.stderr.write(log)
    objs = [o for o, _ in results]
    tmp = LIB + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
