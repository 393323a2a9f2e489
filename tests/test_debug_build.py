"""The bounds-checked debug library builds from the same sources (nvcc, -DLISA_DEBUG_BOUNDS) and
reports its index checks as compiled in; no GPU is needed (nothing here calls CUDA).  The GPU
side of the debug build is tests/test_gpu_debug_bounds.py."""
import os
import shutil
import subprocess
import sys

import pytest


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="needs nvcc")
def test_debug_library_builds_with_checks_enabled():
    from paper_2507_06300_gb300 import build
    path = build.build(debug=True)
    assert path.endswith("liblisa_psd_debug.so") and os.path.exists(path)
    # loaded in a child process: the release library of this process is left alone
    code = ("import ctypes, sys; l = ctypes.CDLL(sys.argv[1]); "
            "l.lisa_debug_bounds_enabled.restype = ctypes.c_int32; print(l.lisa_debug_bounds_enabled())")
    r = subprocess.run([sys.executable, "-c", code, path], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == "1"

