"""Plain FP32 multi-core CPU Fastfood feature map (``fastfood_fp32.c``).

The CPU comparison point that the benchmark times beside the GPU kernels: an
iterative in-place FP32 Walsh-Hadamard transform and the feature map, samples
split over POSIX threads on every host core. It is built with gcc into this
directory (``build()``) and called through ctypes. It is not the oracle (that
is float64 and test infrastructure) and not part of the GPU library; it
shares no code with either. The tables B, Pi, G and Cs are inputs.
"""

import ctypes
import os
import shutil
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "fastfood_fp32.c")
LIB = os.path.join(HERE, "libff32.so")

_lib = None


def build(force=False):
    """Compile libff32.so with gcc (portable flags: no -march); returns its path."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        raise RuntimeError("no C compiler found for the CPU baseline")
    tmp = LIB + ".tmp"
    r = subprocess.run([cc, "-O3", "-std=c11", "-shared", "-fPIC", "-pthread", "-o", tmp, SRC, "-lm"],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"gcc failed on fastfood_fp32.c:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


def load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(LIB)
        P, I64, I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        lib.ff32_features.restype = ctypes.c_int
        lib.ff32_features.argtypes = [P, I64, I64, I64, I64, I32, P, P, P, P, P, I64, I32]
        _lib = lib
    return _lib


def _c(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, ctypes.c_void_p(a.ctypes.data)


def features(x, B, perm, G, Cs, threads=None, out=None):
    """phi (n x 2Ed float32) of x (n x in_dim) with tables of shape (E, d).

    ``out``: an (out_rows, 2Ed) float32 array that receives sample i in row
    i % out_rows (a smaller buffer lets a timing run write every feature of a
    large batch without holding them all); default a fresh (n, 2Ed) array.
    """
    lib = load()
    x, xp = _c(x, np.float32)
    n, in_dim = x.shape
    E, d = np.shape(B)
    B, Bp = _c(B, np.float32)
    perm, pp = _c(perm, np.uint32)
    G, Gp = _c(G, np.float32)
    Cs, Cp = _c(Cs, np.float32)
    if out is None:
        out = np.empty((n, 2 * E * d), np.float32)
    if out.dtype != np.float32 or not out.flags.c_contiguous or out.shape[1] != 2 * E * d:
        raise ValueError("out must be a C-contiguous float32 array with 2Ed columns")
    threads = threads or os.cpu_count() or 1
    st = lib.ff32_features(xp, n, in_dim, in_dim, d, E, Bp, pp, Gp, Cp,
                           ctypes.c_void_p(out.ctypes.data), out.shape[0], threads)
    if st != 0:
        raise RuntimeError(f"ff32_features failed with status {st}")
    return out


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), or None."""
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
        for line in r.stdout.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return None
