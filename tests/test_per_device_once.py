"""The launchers raise a kernel's shared-memory limit once per device.

cudaFuncSetAttribute acts on the current device's context, so a flag kept
once per process would skip the call on a second GPU.  The launchers use
PerDeviceOnce (csrc/per_device_once.h, header-only, no CUDA types); this
test compiles a host program against it with the system C++ compiler and
runs it with a fake device query (no GPU needed).
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_set_up_runs_once_per_device(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = tmp_path / "per_device_once_test"
    src = os.path.join(ROOT, "tests", "cpp", "per_device_once_test.cpp")
    inc = os.path.join(ROOT, "paper_2107_14027_gb300", "csrc")
    subprocess.run([cxx, "-std=c++17", "-O1", "-pthread", "-I", inc, src, "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
