"""The C ABI library loads, exports every declared entry point, and rejects bad
arguments on the host before any device work (these checks need no GPU)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import shutil

    from paper_1702_08159_gb300 import _lib, build

    if not os.path.exists(_lib.LIB_PATH):
        if not (shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc")):
            pytest.skip("nvcc unavailable and libmck.so not built")
        build.build()
    return _lib.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "mck.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mck_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    from paper_1702_08159_gb300 import _lib

    names = declared_functions()
    assert len(names) >= 13
    for name in names:
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, f"{name} has no ctypes signature in the binding"


def test_status_strings(lib):
    for code in (0, -1, -2, -3, -4, -5):
        assert lib.mck_status_string(code).startswith(b"MCK_")
    assert b"unknown" in lib.mck_status_string(42)


def _plan(lib, d=1024, E=1, kernel=0, sigma=1.0, t=40, seed=1, device=-1, out=True):
    h = ctypes.c_void_p()
    return lib.mck_plan_ex(ctypes.byref(h) if out else None, d, E, kernel, sigma, t, seed, device)


@pytest.mark.parametrize("kw,status", [
    (dict(d=3), -1), (dict(d=0), -1), (dict(d=1), -1), (dict(d=-8), -1),
    (dict(d=1 << 21), -5), (dict(d=1 << 16, kernel=1), -5), (dict(E=0), -1), (dict(E=70000), -1), (dict(kernel=3), -1), (dict(kernel=-1), -1),
    (dict(sigma=0.0), -1), (dict(sigma=-1.0), -1), (dict(sigma=float("inf")), -1),
    (dict(sigma=float("nan")), -1), (dict(kernel=1, t=0), -1), (dict(device=-2), -1),
    (dict(out=False), -1), (dict(d=1 << 15, E=1 << 14), -1),
])
def test_plan_argument_validation(lib, kw, status):
    assert _plan(lib, **kw) == status
    assert lib.mck_last_error()


def test_calls_reject_null_plan_and_arguments(lib):
    v = ctypes.c_void_p
    assert lib.mck_plan_info(None, None, None, None, None, None, None, None) == -1
    assert lib.mck_plan_tables(None, None, None, None, None) == -1
    assert lib.mck_features(None, v(16), 1, 1, 1, None, None, v(16), None) == -1
    assert lib.mck_features_backward(None, v(16), 1, 1, 1, None, None, v(16), None, None, None,
                                     None) == -1
    assert lib.mck_fused_logits(None, v(16), 1, 1, 1, None, None, v(16), None, 10, v(16),
                                None) == -1
    for prec in (0, 4, 3):  # FP32, the tensor-core split, and an unbuilt contraction precision
        assert lib.mck_fused_logits_ex(None, v(16), 1, 1, 1, None, None, v(16), None, 10, v(16),
                                       prec, None) == -1
        assert lib.mck_features_ex(None, v(16), 1, 1, 1, None, None, v(16), prec, None) == -1
    assert lib.mck_fwht(v(16), 1, 3, 0, None) == -1          # d not a power of two
    assert lib.mck_fwht(v(16), 1, 1 << 21, 0, None) == -5    # beyond 2^20
    assert lib.mck_fwht(v(16), 1, 8, 7, None) == -5          # unknown precision
    assert lib.mck_fwht(v(16), 4, 8, 1, None) == -5          # tensor-core form needs d >= 256
    assert lib.mck_fwht(v(16), 3, 256, 1, None) == -1        # n * d not a multiple of 1024
    assert lib.mck_fwht(None, 1, 8, 0, None) == -1
    assert lib.mck_fwht(None, 0, 8, 0, None) == 0            # empty: no storage needed
    assert lib.mck_fwht(v(16), -1, 8, 0, None) == -1
    assert lib.mck_fwht(v(16), 0, 8, 0, None) == 0           # empty batch: no-op
    assert lib.mck_softmax_xent(v(16), v(16), -1, 10, None, None, None) == -1
    assert lib.mck_softmax_xent(v(16), v(16), 1, 0, None, None, None) == -1
    lib.mck_plan_destroy(None)  # ignored


def test_no_gpu_reports_cuda_error_not_crash(lib):
    # Without a usable device a valid request must fail cleanly with MCK_ECUDA.
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    assert _plan(lib) == -3
    assert b"cuda" in lib.mck_last_error().lower()


def test_binding_refuses_missing_library(tmp_path, monkeypatch):
    from paper_1702_08159_gb300 import _lib

    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "libmck.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(RuntimeError, match="no fallback"):
        _lib.load()


C_CALLER = r"""
#include <stdio.h>
#include <string.h>
#include "mck.h"

int main(void) {
  mck_plan_t p = 0;
  /* argument checks run on the host before any device work */
  mck_status_t s = mck_plan(&p, 3, 1, MCK_RBF, 1.0, 1u);
  if (s != MCK_EINVAL || p != 0) return 1;
  s = mck_plan_ex(&p, 1024, 1, MCK_LAPLACE + 1, 1.0, 40, 1u, -1);
  if (s != MCK_EINVAL) return 2;
  if (strncmp(mck_status_string(MCK_EUNSUPPORTED), "MCK_", 4) != 0) return 3;
  if (mck_last_error() == 0 || mck_last_error()[0] == 0) return 4;
  mck_plan_destroy(0);
  printf("ok\n");
  return 0;
}
"""


def test_header_is_plain_c_and_links(lib, tmp_path):
    """A C99 program includes mck.h, links libmck.so and gets the host-side
    argument errors: the boundary needs neither C++ nor Python."""
    import shutil
    import subprocess

    from paper_1702_08159_gb300 import _lib

    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    src = tmp_path / "caller.c"
    src.write_text(C_CALLER)
    exe = tmp_path / "caller"
    libdir = os.path.dirname(_lib.LIB_PATH)
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                        str(src), "-o", str(exe), "-L", libdir, "-l:libmck.so",
                        "-Wl,-rpath," + libdir], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert run.returncode == 0 and run.stdout.strip() == "ok", (run.returncode, run.stderr)
