"""The column rule of the x-face traces at lane-group ends, checked on the
host with the kernels' own functions.

An element stores its low x face when its left neighbour (periodic along x)
is not the previous lane of its group of E elements, and its high face when
its right neighbour is not the next lane; the fused kernel reads exactly
those faces of the neighbours it cannot reach by a shuffle.  x_col
(csrc/xface_layout.h, no CUDA types) must give every stored face of one side
a column of its own below the row pitch, and the reader must find the
writer's column.  This test compiles tests/cpp/xface_layout_test.cpp against
that header with the system C++ compiler and runs it over n_x = 1..200,
1..5 rows and E = 4, 8, 16, 32 (every n_x < E, multiple of E and neither).
The GPU tests run the kernels on meshes of each kind.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_stored_x_faces_have_their_own_columns(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = tmp_path / "xface_layout_test"
    src = os.path.join(ROOT, "tests", "cpp", "xface_layout_test.cpp")
    inc = os.path.join(ROOT, "paper_2107_14027_gb300", "csrc")
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", inc, src, "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
