"""Host-side logic compiled and run on the CPU: the memory rectangles the
dataflow capture orders launches by (paper_0707_2347_gb300/csrc/flow.cpp)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_0707_2347_gb300", "csrc")


def _cuda_include():
    for d in ("/usr/local/cuda/include", os.path.join(os.environ.get("CUDA_HOME", ""), "include")):
        if d and os.path.exists(os.path.join(d, "cuda_runtime.h")):
            return d
    return None


def test_dependency_rectangles(tmp_path):
    cxx = shutil.which("g++")
    inc = _cuda_include()
    if not cxx or not inc:
        pytest.skip("g++ or the CUDA headers are missing")
    exe = tmp_path / "rects_test"
    # flow.cpp's rectangle functions need no CUDA library; the Flow class is
    # compiled but not linked in (only rect_of / rect_bytes / overlaps run)
    src = os.path.join(ROOT, "tests", "host", "rects_test.cpp")
    obj = tmp_path / "flow_rects.o"
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, "-I", inc, "-c", os.path.join(CSRC, "flow.cpp"), "-o",
                    str(obj)], check=True)
    r = subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, "-I", inc, src, str(obj), "-o", str(exe),
                        "-Wl,--unresolved-symbols=ignore-all"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout
